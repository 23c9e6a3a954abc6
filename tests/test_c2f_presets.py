"""The package's C2F presets are the paper's FME-settings table (the golden
fixture), and their scheduled pixel-candidate counts at the paper's
1024 x 2048 resolution reproduce the table's GFLOPs column (RAW counting)."""
import json
import os

import pytest

from paper_2508_05990_b300 import bayer_me as bm

GOLDEN = os.path.join(os.path.dirname(__file__), "golden", "fme_settings_gflops.json")


@pytest.mark.parametrize("mode", ["standard", "mode1", "mode2", "mode3", "mode4"])
def test_presets_match_the_table(mode):
    tab = json.load(open(GOLDEN))
    m = tab["modes"][mode]
    p = bm.C2F_PRESETS[mode]
    assert list(p.levels) == m["levels"]
    assert [list(s) for s in p.stages] == m["stages"]
    H, W = tab["resolution"]
    gflops = bm.c2f_pixel_candidates(p, H, W, even=False) / 1e9
    assert abs(gflops - m["gflops"]) <= 0.011


def test_even_mapping_keeps_the_reach():
    p = bm.C2FSetting((32,), ((2, 1),))
    # (2, 1) becomes (1, 2): 9 candidates instead of 25, same +-2 reach
    assert bm.c2f_pixel_candidates(p, 64, 64, even=True) == 4 * 32 * 32 * 9
    assert bm.c2f_pixel_candidates(p, 64, 64, even=False) == 4 * 32 * 32 * 25
