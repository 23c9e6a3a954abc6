"""CPU oracle (float64) of the refine convolution of propagated features.

TEST INFRASTRUCTURE ONLY (see ``oracle/__init__.py``).

The paper corrects propagated features with a learned residual (Sec. 3.3,
z_C = z_pred + z_Res); the refine form here is its dense-convolution core:
three 3x3 convolutions, stride 1, zero padding 1, on NHWC maps,
C -> hidden (ReLU) -> hidden (ReLU) -> C (linear), biases added:

    y[o, i, k] = b[o] + sum_{c, ky, kx} w[o, c, ky, kx] * x[c, i + ky - 1, k + kx - 1]

Each tap's channel contraction is one library matrix product (tensordot).
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


def refine(x, w1, b1, w2, b2, w3, b3):
    """Three convolutions: ReLU after the first two, the last linear."""
    a = np.maximum(conv3x3(x, w1, b1), 0.0)
    a = np.maximum(conv3x3(a, w2, b2), 0.0)
    return conv3x3(a, w3, b3)
