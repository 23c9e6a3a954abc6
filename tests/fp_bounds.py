"""Per-element error measures for the BF16 and FP32 convolution paths.

Test helper: evaluates the oracle's own functions (on absolute values, for the
magnitudes below); it holds no arithmetic of the method beyond what
``oracle/`` computes.

Measure.  An output element y = b + sum_k w_k x_k of a convolution is judged
against m = |b| + sum_k |w_k| |x_k|, the sum of the absolute values of the
terms that make it.  This is the denominator of the componentwise error bounds
of floating-point inner products (Higham, "Accuracy and Stability of Numerical
Algorithms", 2nd ed., Sec. 3.1): a sum of n terms computed with unit roundoff u
satisfies |fl(y) - y| <= gamma_n m, gamma_n = n u / (1 - n u), whatever |y|
is -- near a zero crossing |y| can be arbitrarily smaller than its error, so a
relative error |got - exact| / |exact| has no bound there.  "Max relative
error t" is therefore stated and tested per element as

    |got - exact| <= t * m.

The tolerances and why they hold (the numbers in brackets were measured on
the CPU with the oracle's bfloat16-rounded form, which rounds exactly where
the GPU does):
  * BF16 vs the exact float64 oracle: t = 2e-2.  The last layer's own
    roundings (its input and weights in bfloat16, relative error u_b = 2^-8
    each) move y by at most 2 u_b m = 7.8e-3 m; the earlier layers' rounding
    errors enter through the last layer's weights as a sum of many terms of
    independent sign [refine: 2.2e-3 m; proposal network logits: 8.9e-3 m at
    1080p].
  * BF16 vs the oracle's bfloat16-rounded form: t = 2^-8 for the refine's
    three layers, 2^-7 for the proposal network's five.  Both round the same
    operands at the same points; they differ in the order of the float32 sums
    (gamma_n m at each layer, 1.4e-4 m for n = 1153), which can also flip the
    bfloat16 rounding of a hidden value that lies that close to a rounding
    boundary; a flip early in the network travels through every later layer
    [float32 sums in torch's order: refine 5.1e-4 m; proposal network logits
    at 1080p 2.9e-3 m, 99.99th percentile 2.5e-3 m].
  * FP32 vs the exact float64 oracle: t = 1e-5 (float32 operands are exact;
    each layer's sum has gamma_n m = 6.9e-5 m in the worst case and about
    sqrt(n) u m = 2e-6 m typically [1.6e-7 m]).
A worst-case bound carried through all the layers (every error of one sign)
grows by the ratio m / |y| at each layer -- about 10 for these random-weight
maps -- and exceeds the output itself after three layers, so it would accept
anything; it is not used.
"""
from __future__ import annotations

import numpy as np

from oracle import cnn, refine

TOL_BF16 = 2e-2
TOL_BF16_SAME_ROUNDING = 2.0 ** -8
TOL_CNN_SAME_ROUNDING = 2.0 ** -7
TOL_FP32 = 1e-5


def refine_exact(x, w1, b1, w2, b2, w3, b3):
    """Exact float64 outputs of the three refine convolutions and their term
    magnitudes m = |b3| + |W3| * |h2| (h2 the exact second hidden map)."""
    h1 = np.maximum(refine.conv3x3(x, w1, b1), 0.0)
    h2 = np.maximum(refine.conv3x3(h1, w2, b2), 0.0)
    y = refine.conv3x3(h2, w3, b3)
    m = refine.conv3x3(h2, np.abs(np.asarray(w3, np.float64)), np.abs(np.asarray(b3, np.float64)))
    return y, m


def _to_blocks(zh):
    """Head outputs [12, h4, w4] -> [3, 2 h4, 2 w4] (depth-to-space x 2, the
    network's own channel order)."""
    h4, w4 = zh.shape[1:]
    z = np.zeros((3, 2 * h4, 2 * w4))
    for sy in range(2):
        for sx in range(2):
            for q in range(3):
                z[q, sy::2, sx::2] = zh[3 * (2 * sy + sx) + q]
    return z


def cnn_logits(theta, ref, cur, search_range, act_round=None):
    """The proposal network's head outputs z [3, h, w] (dx, dy, confidence
    logits) from the oracle, their term magnitudes m_z = |b_h| + |W_h| |x4|
    (x4 the exact last hidden map), and the oracle's (dx, dy, conf)."""
    dx, dy, conf, c = cnn.forward(theta, ref, cur, search_range, act_round=act_round)
    p = c["p"]
    x4 = c["acts"][-1]
    mh = np.einsum("jc,chw->jhw", np.abs(p["wh"]), np.abs(x4)) + np.abs(p["bh"])[:, None, None]
    return c["z"], _to_blocks(mh), (dx, dy, conf)


def cnn_grad_magnitudes(theta, ref, cur, label_dx, label_dy, search_range, neg_weight=1.0, act_round=None,
                        grad_round=None):
    """(gradient, M): the oracle's gradient and, per parameter, the sum of the
    absolute values of every term of its expansion -- the oracle's own
    backward pass run on |dL/dz|, |weights| and |activations| (the ReLU masks
    unchanged), so that every product and sum of the chain rule adds
    magnitudes."""
    _, cache, dz = cnn.loss_and_dz(theta, ref, cur, label_dx, label_dy, search_range, act_round, neg_weight)
    g = cnn.backward(cache, dz, grad_round)
    cache_abs = dict(cache, p={k: np.abs(v) for k, v in cache["p"].items()}, acts=[np.abs(a) for a in cache["acts"]])
    return g, cnn.backward(cache_abs, np.abs(dz), grad_round)


# The GPU evaluates tanhf and expf in float32: a few units in the last place.
OUT_SLACK = 2.0 ** -18


def tanh_interval(z, t, search_range):
    """range * tanh over [z - t, z + t], widened by the float32 evaluation slack:
    an output lies in it iff some logit within t of z gives it (tanh is monotone)."""
    return (search_range * np.tanh(z - t) - search_range * OUT_SLACK,
            search_range * np.tanh(z + t) + search_range * OUT_SLACK)


def sigmoid_interval(z, t):
    return 1.0 / (1.0 + np.exp(-(z - t))) - OUT_SLACK, 1.0 / (1.0 + np.exp(-(z + t))) + OUT_SLACK


def inside(v, lo_hi) -> np.ndarray:
    lo, hi = lo_hi
    v = np.asarray(v, np.float64)
    return (v >= lo) & (v <= hi)


def outputs_within(prop, conf, z, t, search_range) -> np.ndarray:
    """Per block: the GPU's (dx, dy, conf) all come from logits within t of z
    (t per element)."""
    return (inside(prop[..., 0], tanh_interval(z[0], t[0], search_range))
            & inside(prop[..., 1], tanh_interval(z[1], t[1], search_range))
            & inside(conf, sigmoid_interval(z[2], t[2])))
