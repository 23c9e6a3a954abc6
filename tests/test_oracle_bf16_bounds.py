"""Pins of the refine oracle's bfloat16 form and of the per-element error
measures the GPU tests use (tests/fp_bounds.py).

* ``refine(..., act_round="bf16")`` against closed forms: a one-channel chain
  whose roundings can be worked out by hand, and data exactly representable in
  bfloat16 (no rounding, so it equals the exact refine).
* Its rounding against torch's float32 -> bfloat16 conversion.
* The per-element tolerances of tests/fp_bounds.py hold, with margin, for the
  bfloat16-rounded oracle, whose roundings are the GPU's (it differs from the
  GPU only in the order of its float32 sums): against the exact oracle (max
  relative error 2e-2 of the terms' absolute sum), and against itself with
  float32 sums in another order (2^-8); the latter rejects an output with one
  element moved by 5 % of the output's RMS, the former one moved by 25 %.
"""
import numpy as np
import pytest
import torch

from oracle import cnn, refine
from paper_2508_05990_b300 import bayer_me as bm
from paper_2508_05990_b300 import synth

import fp_bounds as fb


def one_channel(v):
    """A 1 x 1 x 1 map and 1 -> 1 -> 1 -> 1 weights whose centre tap is v."""
    w = np.zeros((1, 1, 3, 3))
    w[0, 0, 1, 1] = v
    return w


def test_refine_bf16_closed_form():
    # x = 1 + 2^-9 rounds to 1 (below half an ulp); w = 1 + 2^-8 is a tie and
    # rounds to even, 1; the hidden values 1 + 2^-9 (bias 2^-9) round to 1 again
    x = np.full((1, 1, 1), 1 + 2.0 ** -9)
    w = one_channel(1 + 2.0 ** -8)
    b = np.array([2.0 ** -9])
    got = refine.refine(x, w, b, w, b, w, b, act_round="bf16")
    # layer 1: 1*1 + 2^-9 -> round -> 1; layer 2 the same; layer 3: 1*1 + 2^-9, not rounded
    assert got.shape == (1, 1, 1) and got[0, 0, 0] == 1 + 2.0 ** -9
    exact = refine.refine(x, w, b, w, b, w, b)
    a1 = (1 + 2.0 ** -9) * (1 + 2.0 ** -8) + 2.0 ** -9
    a2 = a1 * (1 + 2.0 ** -8) + 2.0 ** -9
    assert exact[0, 0, 0] == pytest.approx(a2 * (1 + 2.0 ** -8) + 2.0 ** -9, rel=1e-15)
    # 1 + 3 * 2^-8 is not a tie: it rounds up to 1 + 2^-6
    got = refine.refine(np.ones((1, 1, 1)), one_channel(1 + 3 * 2.0 ** -8), np.zeros(1), one_channel(1.0),
                        np.zeros(1), one_channel(1.0), np.zeros(1), act_round="bf16")
    assert got[0, 0, 0] == 1 + 2.0 ** -6


def test_refine_bf16_exact_on_representable_data():
    """Small integers times powers of two, sparse weights: every operand and
    hidden value is a bfloat16 number, so no rounding happens anywhere."""
    rng = np.random.default_rng(3)
    x = rng.integers(-3, 4, (6, 7, 4)).astype(np.float64)
    ws = [np.where(rng.random((o, i, 3, 3)) < 0.15, rng.integers(-2, 3, (o, i, 3, 3)) / 4.0, 0.0)
          for o, i in ((5, 4), (5, 5), (4, 5))]
    bs = [rng.integers(-2, 3, 5) / 2.0, rng.integers(-2, 3, 5) / 2.0, np.zeros(4)]
    args = (x, ws[0], bs[0], ws[1], bs[1], ws[2], bs[2])
    exact = refine.refine(*args)
    h1 = np.maximum(refine.conv3x3(x, ws[0], bs[0]), 0)
    h2 = np.maximum(refine.conv3x3(h1, ws[1], bs[1]), 0)
    for v in (h1, h2):  # the hidden values really are bfloat16 numbers
        np.testing.assert_array_equal(refine.round_bf16(v), v)
    np.testing.assert_array_equal(refine.refine(*args, act_round="bf16"), exact)


def test_refine_round_bf16_matches_torch():
    rng = np.random.default_rng(2)
    x = np.concatenate([rng.normal(size=1000) * 10.0 ** rng.integers(-5, 5, 1000), [0.0, 1 + 2 ** -8, 1 + 3 * 2 ** -8]])
    want = torch.from_numpy(x).float().bfloat16().double().numpy()
    np.testing.assert_array_equal(refine.round_bf16(x), want)


REFINE_SHAPES = [("w", (64, 128, 3, 3)), ("b", (64,)), ("w", (64, 64, 3, 3)), ("b", (64,)),
                 ("w", (128, 64, 3, 3)), ("b", (128,))]


def refine_params(seed):
    theta = synth.he_normal_params(seed, REFINE_SHAPES)
    rng = np.random.default_rng(seed + 1)
    out, o = [], 0
    for kind, shape in REFINE_SHAPES:
        n = int(np.prod(shape))
        v = theta[o:o + n].reshape(shape)
        if kind == "b":
            v = rng.normal(0, 0.1, shape).astype(np.float32)
        out.append(np.ascontiguousarray(v, np.float32))
        o += n
    return out


def test_refine_tolerances_hold_for_the_bf16_oracle_and_catch_a_planted_error():
    feat = synth.features(67, 128, 12, 40, n=1, layout="NHWC")[0]
    p = refine_params(5)
    exact, m = fb.refine_exact(feat, *p)
    emu = refine.refine(feat, *p, act_round="bf16")
    err = np.abs(emu - exact)
    assert np.all(err <= fb.TOL_BF16 * m)
    assert (err / m).max() < fb.TOL_BF16 / 4  # the tolerance has margin
    # the same roundings with float32 sums in torch's order stay within 2^-8 m of the oracle's
    bf = lambda v: torch.from_numpy(np.asarray(v, np.float32)).bfloat16().float()  # noqa: E731
    t = bf(feat).permute(2, 0, 1)[None]
    for k, relu in ((0, True), (2, True), (4, False)):
        t = torch.nn.functional.conv2d(t, bf(p[k]), torch.from_numpy(p[k + 1]), padding=1)
        t = bf(torch.relu(t).numpy()) if relu else t
    o32 = t[0].permute(1, 2, 0).double().numpy()
    assert np.all(np.abs(o32 - emu) <= fb.TOL_BF16_SAME_ROUNDING * m)
    assert (np.abs(o32 - emu) / m).max() < fb.TOL_BF16_SAME_ROUNDING / 4
    # one element moved by 5 % of the output's RMS fails the same-rounding check, by 25 % the exact one
    rms = np.sqrt((exact ** 2).mean())
    i = np.unravel_index(np.argmin(m), m.shape)
    bad = emu.copy()
    bad[i] += 0.05 * rms
    assert not np.all(np.abs(bad - emu) <= fb.TOL_BF16_SAME_ROUNDING * m)
    bad[i] += 0.20 * rms
    assert not np.all(np.abs(bad - exact) <= fb.TOL_BF16 * m)
    # FP32: float32 operands and sums (torch's float32 conv2d as the stand-in)
    t = torch.from_numpy(feat).permute(2, 0, 1)[None]
    for k, relu in ((0, True), (2, True), (4, False)):
        t = torch.nn.functional.conv2d(t, torch.from_numpy(p[k]), torch.from_numpy(p[k + 1]), padding=1)
        t = torch.relu(t) if relu else t
    f32 = t[0].permute(1, 2, 0).double().numpy()
    assert np.all(np.abs(f32 - exact) <= fb.TOL_FP32 * m)
    bad = f32.copy()
    bad[i] += 1e-3 * rms
    assert not np.all(np.abs(bad - exact) <= fb.TOL_FP32 * m)


def test_cnn_tolerances_hold_for_the_bf16_oracle():
    H, W = 128, 192
    ref, cur = synth.pan_clip(90, H, W, n_frames=2, rect_size=(16, 64))
    theta = torch.from_numpy(synth.he_normal_params(3, bm.CNN_SHAPES)).to(torch.bfloat16).double().numpy()
    z, mz, _ = fb.cnn_logits(theta, ref, cur, 32)
    zb, _, (gx, gy, gc) = fb.cnn_logits(theta, ref, cur, 32, act_round="bf16")
    assert np.all(np.abs(zb - z) <= fb.TOL_BF16 * mz)
    assert (np.abs(zb - z) / mz).max() < fb.TOL_BF16 / 2
    prop = np.stack([gx, gy], -1)
    assert fb.outputs_within(prop, gc, z, fb.TOL_BF16 * mz, 32).all()
    assert fb.outputs_within(prop, gc, zb, fb.TOL_CNN_SAME_ROUNDING * mz, 32).all()
    # a proposal moved by 1 px where the network is confident fails
    i = np.unravel_index(np.argmin(mz[0]), mz[0].shape)
    bad = prop.copy()
    bad[i + (0,)] += 1.0
    assert not fb.outputs_within(bad, gc, z, fb.TOL_BF16 * mz, 32).all()
    # a confidence moved by 0.02 fails the same-rounding check
    bad = gc.copy()
    bad[np.unravel_index(np.argmax(gc * (1 - gc)), gc.shape)] += 0.02
    assert not fb.outputs_within(prop, bad, zb, fb.TOL_CNN_SAME_ROUNDING * mz, 32).all()
