"""What the trained proposal network gains over the search without it.

On held-out 1080p clips (the scene generator with the evaluation seeds
2*10^6 + k, never seen in training), three searches of the same pairs:

* exhaustive +-32 search (no network): the reference for SAD regret, 1089
  candidates per block;
* the +-4 refine around the zero MV for every block (the seeded search with no
  network: proposal (0, 0), confidence 1): 25 candidates per block;
* the learned-seeded search with the committed trained weights: 25 candidates
  per confident block, 1089 for the fallback blocks.

The trained network must keep the SAD regret at or below 1 % while evaluating
at most a third of the exhaustive search's candidates, and its regret must be a
small fraction of the zero-proposal refine's.  The same check with untrained
(He-initialised) weights shows that the gain comes from training.
"""
import os

import numpy as np
import pytest

from paper_2508_05990_b300 import bayer_me as bm
from paper_2508_05990_b300 import synth

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

H, W, T, RANGE = 1088, 1920, 8, 32
EVAL_SEED = 2_000_000
WEIGHTS = os.path.join(os.path.dirname(os.path.dirname(os.path.abspath(__file__))), "paper_2508_05990_b300",
                       "weights", "proposal_1080p_r32.npz")
N_CAND_FULL = (RANGE + 1) ** 2
N_CAND_REFINE = 25


@pytest.fixture(scope="module")
def handle():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2508_05990_b300 import build
    build.build()
    h = bm.Handle(0)
    yield h
    h.close()


@pytest.fixture(scope="module")
def heldout(handle):
    """Two held-out 8-frame clips (14 pairs) on the device and their exhaustive-search fields."""
    clips = [torch.from_numpy(synth.pan_clip(EVAL_SEED + k, H, W, n_frames=T).view(np.int16)).cuda() for k in (0, 1)]
    kw = dict(batch=T - 1, ref_batch_stride=H * W, cur_batch_stride=H * W)
    full = [handle.estimate_ex(d, d[1:], search_range=RANGE, **kw) for d in clips]
    return clips, full, kw


def _sad(rec):
    return bm.records_to_numpy(rec)["sad"].astype(np.int64)


def _learned(handle, heldout, wbf):
    clips, full, kw = heldout
    sad_l = sad_f = 0
    n_fb = n_blk = 0
    for d, f in zip(clips, full):
        fb = torch.empty((T - 1, H // 16, W // 16), dtype=torch.uint8, device="cuda")
        out = handle.estimate_learned(d, d[1:], wbf, RANGE, 0.5, fallback=fb, **kw)
        sad_l += int(_sad(out).sum())
        sad_f += int(_sad(f).sum())
        n_fb += int(fb.sum().item())
        n_blk += fb.numel()
    rate = n_fb / n_blk
    return (sad_l - sad_f) / sad_f, rate, rate + (1 - rate) * N_CAND_REFINE / N_CAND_FULL


def test_trained_network_gain(handle, heldout):
    clips, full, kw = heldout
    # no network: +-4 refine around the zero MV everywhere
    sad_z = sad_f = 0
    for d, f in zip(clips, full):
        prop = torch.zeros((T - 1, H // 16, W // 16, 2), dtype=torch.float32, device="cuda")
        conf = torch.ones((T - 1, H // 16, W // 16), dtype=torch.float32, device="cuda")
        out = handle.estimate_ex(d, d[1:], mode=bm.MODE_SEEDED, search_range=RANGE, prop_dxdy=prop, conf=conf, **kw)
        sad_z += int(_sad(out).sum())
        sad_f += int(_sad(f).sum())
    regret_zero = (sad_z - sad_f) / sad_f

    theta = torch.from_numpy(np.load(WEIGHTS)["theta"].astype(np.float32)).cuda()
    regret_t, fb_t, cand_t = _learned(handle, heldout, bm.to_bf16_bits(theta).contiguous())
    w_init = torch.from_numpy(synth.he_normal_params(7, bm.CNN_SHAPES)).cuda()
    regret_u, fb_u, cand_u = _learned(handle, heldout, bm.to_bf16_bits(w_init).contiguous())
    print(f"\nzero-proposal refine: regret {regret_zero:.4f} (25 candidates per block)"
          f"\ntrained network: regret {regret_t:.4f}, fallback {fb_t:.3f}, candidates {cand_t:.3f} of exhaustive"
          f"\nuntrained network: regret {regret_u:.4f}, fallback {fb_u:.3f}, candidates {cand_u:.3f} of exhaustive")
    assert 0.0 <= regret_t <= 0.01
    assert cand_t <= 1 / 3
    assert regret_t <= 0.1 * regret_zero
    # untrained weights either fall back far more often or lose far more SAD
    assert cand_u >= 2 * cand_t or regret_u >= 5 * max(regret_t, 1e-3)


def test_configured_scale_weights_on_the_configured_heldout_pairs(handle):
    """The network trained on exactly 2,000 pairs, evaluated on exactly the 200
    held-out pairs of the learned-proposal workload (seeds 2e6 + k, first 200
    pairs of 29 clips): SAD regret at most 1 % against the exhaustive search,
    with at most a quarter of the blocks falling back."""
    import os
    from paper_2508_05990_b300 import train_proposal as tp
    path = os.path.join(os.path.dirname(os.path.dirname(os.path.abspath(__file__))), "paper_2508_05990_b300",
                        "weights", "proposal_1080p_r32_2000pairs.npz")
    theta = torch.from_numpy(np.load(path)["theta"].astype(np.float32)).cuda()
    clips = tp.make_clips(tp.EVAL_SEED, 29, max(1, (os.cpu_count() or 2) - 1))
    clips_d = torch.from_numpy(clips.view(np.int16)).cuda()
    labels = tp.label_clips(handle, clips_d)
    res = tp.evaluate(handle, clips_d, labels, bm.to_bf16_bits(theta).contiguous(), reps=2, n_pairs=200)
    print(f"\nconfigured scale: {res}")
    assert res["pairs"] == 200
    assert 0.0 <= res["sad_regret"] <= 0.01
    assert res["fallback_rate"] <= 0.25
