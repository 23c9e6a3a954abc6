"""CPU oracle (float64) of the refine convolution of propagated features.

TEST INFRASTRUCTURE ONLY (see ``oracle/__init__.py``).

The paper corrects propagated features with a learned residual (Sec. 3.3,
z_C = z_pred + z_Res); the refine form here is its dense-convolution core:
three 3x3 convolutions, stride 1, zero padding 1, on NHWC maps,
C -> hidden (ReLU) -> hidden (ReLU) -> C (linear), biases added:

    y[o, i, k] = b[o] + sum_{c, ky, kx} w[o, c, ky, kx] * x[c, i + ky - 1, k + kx - 1]

Each tap's channel contraction is one library matrix product (tensordot).

``act_round="bf16"`` evaluates the same three convolutions with the operands
the BF16 form stores in bfloat16 rounded to it (round to nearest, ties to
even, of the float32 value): the input map, the three weight tensors and the
two hidden activations (after ReLU); biases stay float32 and every sum is
exact (float64).  ``act_round=None`` is the exact reference.
"""
from __future__ import annotations

import numpy as np


def conv3x3(x, w, b):
    """x [H, W, Cin] (NHWC, one map), w [Cout, Cin, 3, 3], b [Cout] -> [H, W, Cout], float64."""
    x = np.asarray(x, np.float64)
    H, W, _ = x.shape
    xp = np.zeros((H + 2, W + 2, x.shape[2]))
    xp[1:H + 1, 1:W + 1] = x
    y = np.zeros((H, W, w.shape[0])) + np.asarray(b, np.float64)
    w = np.asarray(w, np.float64)
    for ky in range(3):
        for kx in range(3):
            y += np.tensordot(xp[ky:ky + H, kx:kx + W], w[:, :, ky, kx], axes=([2], [1]))
    return y


def round_bf16(x) -> np.ndarray:
    """float64 -> float32 -> bfloat16 (round to nearest, ties to even) -> float64:
    keep the top 16 bits of the float32 pattern after adding half of the
    dropped 16 bits' range, minus one unless the kept part is odd."""
    b = np.asarray(x, np.float32).view(np.uint32).astype(np.uint64)
    b = (b + 0x7FFF + ((b >> 16) & 1)) & 0xFFFF0000
    return b.astype(np.uint32).view(np.float32).astype(np.float64)


def refine(x, w1, b1, w2, b2, w3, b3, act_round=None):
    """Three convolutions: ReLU after the first two, the last linear."""
    r = round_bf16 if act_round == "bf16" else (lambda v: np.asarray(v, np.float64))
    a = np.maximum(conv3x3(r(x), r(w1), b1), 0.0)
    a = np.maximum(conv3x3(r(a), r(w2), b2), 0.0)
    return conv3x3(r(a), r(w3), b3)
