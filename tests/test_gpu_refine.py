"""Refine convolution (3x3, C=128 -> 64 -> 64 -> 128) of propagated features,
BF16 on the tensor cores and FP32 on the SIMT cores, both judged against the
float64 oracle (oracle/refine.py), element by element.

Tolerances (tests/fp_bounds.py states the measure and derives them): every
output element y, with m = |b3| + sum |w3| |h2| the absolute sum of its terms,
  * BF16: |gpu - exact| <= 2e-2 m, and |gpu - bf16-rounded oracle| <= 2^-8 m
    (the oracle rounding input, weights and both hidden maps where the kernels
    do; the two differ only in the order of the float32 sums);
  * FP32: |gpu - exact| <= 1e-5 m.
"""
import numpy as np
import pytest

import fp_bounds as fb
from oracle import refine
from paper_2508_05990_b300 import bayer_me as bm
from paper_2508_05990_b300 import synth

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

SHAPES = [("w", (64, 128, 3, 3)), ("b", (64,)), ("w", (64, 64, 3, 3)), ("b", (64,)), ("w", (128, 64, 3, 3)),
          ("b", (128,))]


@pytest.fixture(scope="module")
def handle():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2508_05990_b300 import build
    build.build()
    h = bm.Handle(0)
    yield h
    h.close()


def params(seed):
    theta = synth.he_normal_params(seed, SHAPES)
    rng = np.random.default_rng(seed + 1)
    out, o = [], 0
    for kind, shape in SHAPES:
        n = int(np.prod(shape))
        v = theta[o:o + n].reshape(shape)
        if kind == "b":  # non-zero biases exercise the epilogue
            v = rng.normal(0, 0.1, shape).astype(np.float32)
        out.append(np.ascontiguousarray(v, np.float32))
        o += n
    return out


def check_elements(ob, of, feat, p):
    """Every element of the BF16 output ob and the FP32 output of against the
    oracle (one map, NHWC)."""
    exact, m = fb.refine_exact(feat, *p)
    emu = refine.refine(feat, *p, act_round="bf16")
    assert np.isfinite(ob).all() and np.isfinite(of).all()
    worst = np.unravel_index(np.argmax(np.abs(ob - exact) / m), m.shape)
    assert np.all(np.abs(ob - exact) <= fb.TOL_BF16 * m), ("bf16 vs exact", worst)
    worst = np.unravel_index(np.argmax(np.abs(ob - emu) / m), m.shape)
    assert np.all(np.abs(ob - emu) <= fb.TOL_BF16_SAME_ROUNDING * m), ("bf16 vs bf16-rounded oracle", worst)
    worst = np.unravel_index(np.argmax(np.abs(of - exact) / m), m.shape)
    assert np.all(np.abs(of - exact) <= fb.TOL_FP32 * m), ("fp32 vs exact", worst)


@pytest.mark.parametrize("shape", [(1, 20, 40), (2, 37, 150), (1, 136, 240)])
def test_refine_bf16_and_fp32_vs_float64(handle, shape):
    n, Hf, Wf = shape
    feat = synth.features(30 + Hf, 128, Hf, Wf, n=n, layout="NHWC")
    p = params(5)
    d = [torch.from_numpy(x).cuda() for x in p]
    f = torch.from_numpy(feat).cuda()
    ob = handle.refine_conv(f, d, bm.PREC_BF16).cpu().numpy()
    of = handle.refine_conv(f, d, bm.PREC_FP32).cpu().numpy()
    assert handle.sync_status() == bm.OK
    for i in range(n):
        check_elements(ob[i], of[i], feat[i], p)


def test_refine_4k_full_map(handle):
    """The 4K form (540 x 960 x 128 at stride 4): every output element of the
    whole map -- first and last rows, every column strip, every row where a
    CTA's run of rows starts or ends and where the ring of staged rows wraps."""
    Hf, Wf = 540, 960
    feat = synth.features(1002, 128, Hf, Wf, n=1, layout="NHWC")
    p = params(6)
    d = [torch.from_numpy(x).cuda() for x in p]
    f = torch.from_numpy(feat).cuda()
    ob = handle.refine_conv(f, d, bm.PREC_BF16).cpu().numpy()[0]
    of = handle.refine_conv(f, d, bm.PREC_FP32).cpu().numpy()[0]
    assert handle.sync_status() == bm.OK
    check_elements(ob, of, feat[0], p)


def test_refine_rejects_unsupported(handle):
    f = torch.zeros((1, 8, 8, 96), device="cuda")
    w = [torch.zeros(1, device="cuda")] * 6
    with pytest.raises(bm.BayerError) as e:
        handle.refine_conv(f, w)
    assert e.value.status == bm.ERR_UNSUPPORTED
