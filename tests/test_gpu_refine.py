"""Refine convolution (3x3, C=128 -> 64 -> 64 -> 128) of propagated features,
BF16 on the tensor cores and FP32 on the SIMT cores, both judged against the
float64 oracle (oracle/refine.py).

Tolerances (normwise relative): BF16 2e-2 (inputs, weights and two hidden
activations rounded to bfloat16, relative 2^-9 each, float32 accumulation);
FP32 1e-5 (float32 products and sums over 9 * 128 terms).
"""
import numpy as np
import pytest

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


def rel(a, b):
    return float(np.linalg.norm(np.asarray(a, np.float64) - b) / np.linalg.norm(b))


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
        want = refine.refine(feat[i], *p)
        assert rel(ob[i], want) < 2e-2
        assert rel(of[i], want) < 1e-5


def test_refine_4k_sampled(handle):
    """The 4K form (540 x 960 x 128 at stride 4): full-frame outputs, a row band
    checked against the oracle (rows 255..264, every column)."""
    Hf, Wf = 540, 960
    feat = synth.features(1002, 128, Hf, Wf, n=1, layout="NHWC")
    p = params(6)
    d = [torch.from_numpy(x).cuda() for x in p]
    f = torch.from_numpy(feat).cuda()
    ob = handle.refine_conv(f, d, bm.PREC_BF16).cpu().numpy()[0]
    of = handle.refine_conv(f, d, bm.PREC_FP32).cpu().numpy()[0]
    y0, y1 = 255, 265
    # a band 3 rows deeper on each side reproduces the band exactly (3 stacked 3x3 convs)
    band = refine.refine(feat[0][y0 - 3:y1 + 3], *p)[3:-3]
    assert rel(ob[y0:y1], band) < 2e-2
    assert rel(of[y0:y1], band) < 1e-5
    assert np.isfinite(ob).all() and np.isfinite(of).all()


def test_refine_rejects_unsupported(handle):
    f = torch.zeros((1, 8, 8, 96), device="cuda")
    w = [torch.zeros(1, device="cuda")] * 6
    with pytest.raises(bm.BayerError) as e:
        handle.refine_conv(f, w)
    assert e.value.status == bm.ERR_UNSUPPORTED
