"""Pins of the CPU oracle's feature propagation z_pred = Warp(z_R, MV) (Sec. 3.3).

Pinned against: the identity (zero MV), a plain shifted copy (MVs that are
multiples of the feature stride), torch's float64 grid_sample (a library
routine computing the same bilinear sampling), ramps whose warp has a closed
form, and the float32 rounding bound.
"""
import numpy as np
import pytest
import torch

from paper_2508_05990_b300 import synth


def random_valid_mv(rng, h, w, B, H, W, multiple=2, mag=16):
    """Per-block MVs that are multiples of ``multiple`` and keep each displaced
    block inside the H x W frame (so every bilinear tap with weight > 0 is in
    range)."""
    import oracle
    mv = np.zeros((h, w), oracle.MV_DTYPE)
    for i in range(h):
        for j in range(w):
            lo_x, hi_x = max(-mag, -j * B), min(mag, W - B - j * B)
            lo_y, hi_y = max(-mag, -i * B), min(mag, H - B - i * B)
            dx = multiple * int(rng.integers(-(-lo_x // multiple), hi_x // multiple + 1))
            dy = multiple * int(rng.integers(-(-lo_y // multiple), hi_y // multiple + 1))
            mv[i, j] = (dx, dy, 0)
    return mv


@pytest.mark.parametrize("layout", [0, 1])
@pytest.mark.parametrize("interp", [0, 1])
def test_zero_mv_is_identity(oracle_mod, layout, interp):
    feat = synth.features(1, 8, 16, 24, layout="NCHW" if layout == 0 else "NHWC")[0]
    mv = np.zeros((4, 6), oracle_mod.MV_DTYPE)
    out = oracle_mod.propagate(feat, mv, 16, 4, interp=interp, layout=layout)
    np.testing.assert_array_equal(out, feat)


@pytest.mark.parametrize("stride", [2, 4, 8])
def test_stride_multiple_mv_is_plain_copy(oracle_mod, stride):
    """MVs that are multiples of the stride move whole feature cells: bilinear
    equals nearest equals out[c, y, x] = feat[c, y + dy/s, x + dx/s]."""
    B = 16
    Hf, Wf, C = 24, 32, 5
    H, W = Hf * stride, Wf * stride
    h, w = H // B, W // B
    rng = np.random.default_rng(stride)
    mv = random_valid_mv(rng, h, w, B, H, W, multiple=stride, mag=4 * stride)
    feat = synth.features(2, C, Hf, Wf)[0]
    near = oracle_mod.propagate(feat, mv, B, stride, interp=0)
    bil = oracle_mod.propagate(feat, mv, B, stride, interp=1)
    cells = B // stride
    expect = np.empty_like(feat)
    for y in range(Hf):
        for x in range(Wf):
            m = mv[y // cells, x // cells]
            expect[:, y, x] = feat[:, y + m["dy"] // stride, x + m["dx"] // stride]
    np.testing.assert_array_equal(near, expect)
    assert np.array_equal(bil, expect)  # value equality (+0.0 == -0.0)


@pytest.mark.parametrize("stride", [4, 8])
def test_bilinear_f64_matches_grid_sample(oracle_mod, stride):
    """torch.nn.functional.grid_sample (float64, align_corners=True, border
    padding) samples the same positions (y + dy/s, x + dx/s)."""
    B = 16
    Hf, Wf, C = 20, 28, 3
    H, W = Hf * stride, Wf * stride
    h, w = -(-H // B), -(-W // B)
    rng = np.random.default_rng(10 + stride)
    mv = random_valid_mv(rng, h, w, B, H, W, multiple=2, mag=12)
    feat = synth.features(3, C, Hf, Wf)[0]
    ours = oracle_mod.propagate_bilinear_f64(feat, mv, B, stride)
    cells = B // stride
    yy, xx = np.mgrid[0:Hf, 0:Wf].astype(np.float64)
    dx = mv["dx"].astype(np.float64)[np.arange(Hf)[:, None] // cells, np.arange(Wf)[None, :] // cells]
    dy = mv["dy"].astype(np.float64)[np.arange(Hf)[:, None] // cells, np.arange(Wf)[None, :] // cells]
    sx, sy = xx + dx / stride, yy + dy / stride
    grid = np.stack([2 * sx / (Wf - 1) - 1, 2 * sy / (Hf - 1) - 1], axis=-1)[None]
    ref = torch.nn.functional.grid_sample(torch.from_numpy(feat.astype(np.float64))[None],
                                          torch.from_numpy(grid), mode="bilinear",
                                          padding_mode="border", align_corners=True)[0].numpy()
    np.testing.assert_allclose(ours, ref, rtol=0, atol=1e-12)


def test_half_cell_rounding_and_ramp(oracle_mod):
    """On the ramp feat[c, y, x] = x, an MV of dx = 2 at stride 4 (half a cell)
    gives bilinear x + 0.5 exactly and nearest x + 1 (half away from zero);
    dx = -2 gives x - 0.5 and x - 1."""
    B, s = 16, 4
    Hf, Wf = 8, 16
    feat = np.broadcast_to(np.arange(Wf, dtype=np.float32)[None, None, :], (2, Hf, Wf)).copy()
    for d, near_off, bil_off in ((2, 1.0, 0.5), (-2, -1.0, -0.5), (6, 2.0, 1.5), (-6, -2.0, -1.5)):
        mv = np.zeros((2, 4), oracle_mod.MV_DTYPE)
        mv["dx"] = d
        near = oracle_mod.propagate(feat, mv, B, s, interp=0)
        bil = oracle_mod.propagate(feat, mv, B, s, interp=1)
        x = np.arange(Wf, dtype=np.float32)
        inner = slice(2, Wf - 2)
        np.testing.assert_array_equal(near[0, 0, inner], (x + near_off)[inner])
        np.testing.assert_array_equal(bil[0, 0, inner], (x + bil_off)[inner])


@pytest.mark.parametrize("stride", [4, 8])
def test_bilinear_f32_within_rounding_bound(oracle_mod, stride):
    """float32 evaluation differs from the float64 one by at most the rounding
    of six operations on a convex combination: 8 * 2^-24 * sum_i w_i |a_i|."""
    B = 16
    Hf, Wf, C = 34, 60, 16
    H, W = Hf * stride, Wf * stride
    h, w = -(-H // B), -(-W // B)
    mv = random_valid_mv(np.random.default_rng(7), h, w, B, H, W, multiple=2, mag=32)
    feat = synth.features(4, C, Hf, Wf)[0]
    f32 = oracle_mod.propagate(feat, mv, B, stride, interp=1)
    f64 = oracle_mod.propagate_bilinear_f64(feat, mv, B, stride)
    bound = 8 * 2.0 ** -24 * oracle_mod.propagate_bilinear_f64(np.abs(feat), mv, B, stride)
    assert (np.abs(f32.astype(np.float64) - f64) <= bound).all()


def test_nhwc_equals_nchw(oracle_mod):
    B, s = 16, 4
    Hf, Wf, C = 12, 20, 7
    mv = random_valid_mv(np.random.default_rng(1), 3, 5, B, Hf * s, Wf * s, multiple=2, mag=8)
    feat = synth.features(5, C, Hf, Wf)[0]
    for interp in (0, 1):
        a = oracle_mod.propagate(feat, mv, B, s, interp=interp, layout=0)
        b = oracle_mod.propagate(np.ascontiguousarray(feat.transpose(1, 2, 0)), mv, B, s, interp=interp, layout=1)
        np.testing.assert_array_equal(a, b.transpose(2, 0, 1))
