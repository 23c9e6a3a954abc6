"""CPU oracle (float64, numpy) of the learned MV-proposal network and its loss.

TEST INFRASTRUCTURE ONLY (see ``oracle/__init__.py``).

The paper has no proposal network; this is the small CNN that seeds the +-4
refine of the learned-seeded search (a proposal per 16x16 block and a
confidence).  Its only link to the paper is the training recipe (AdamW,
lr 1e-4 -> 1e-6 cosine, batch 16; Sec. 4.1 "Training Details") and the BerHu
regression loss the paper uses for PRNet (Sec. 3.3), reused here for the MV
regression.  Written out plainly so that it can be read against the
definitions below:

* input: the four RGGB planes (R at (0, 0), then G on the R row, G on the B
  row, B) of the reference frame and of the current frame at half
  resolution, 8 channels, each sample scaled as v / 2048 - 1;
* four layers y = ReLU(conv3x3(x, stride 2, zero padding 1) + b), 32 channels;
* head: 1x1 conv 32 -> 12 + bias; channel j = 3 * (2 * sy + sx) + q of cell
  (i, k) gives quantity q (0: dx, 1: dy, 2: confidence) of block
  (2 i + sy, 2 k + sx) (depth-to-space x 2);
* dx = range * tanh(z_0), dy = range * tanh(z_1), conf = sigmoid(z_2);
* loss (mean over blocks): BerHu_c(dx - dx*) + BerHu_c(dy - dy*) with
  c = 4 px (|e| below c, (e^2 + c^2) / (2c) above), plus the weighted binary
  cross entropy -t log(conf) - w_neg (1 - t) log(1 - conf) against t = 1 if
  the proposal rounded to the nearest even integer lies within +-4 of the
  label in both components, else 0 (t is a constant of the prediction, no
  gradient flows through it).

Activations: the network's definition stores each post-ReLU activation in
bfloat16 (weights are bfloat16 too).  ``act_round="bf16"`` applies that
rounding (round to nearest, ties to even, of the float32 value) at the same
points; ``act_round=None`` keeps every activation in float64, the exact
reference.  Training stores each layer's pre-activation gradient in bfloat16
too (the operand of that layer's weight- and input-gradient products);
``grad_round="bf16"`` rounds it there.

Parameters are one flat vector (``param_layout``); the CUDA path uses the same
order.  Every function below is plain numpy; the convolution uses einsum over
the nine kernel taps, a library primitive for each tap's channel contraction.
"""
from __future__ import annotations

import numpy as np

CH = 32
N_LAYERS = 4
IN_CH = 8
BERHU_C = 4.0


def param_layout():
    """[(name, shape)] in flat order: conv1..conv4 weight [32, Cin, 3, 3] and
    bias [32], then head weight [12, 32] and bias [12]."""
    lay = []
    cin = IN_CH
    for l in range(N_LAYERS):
        lay.append((f"w{l + 1}", (CH, cin, 3, 3)))
        lay.append((f"b{l + 1}", (CH,)))
        cin = CH
    lay.append(("wh", (12, CH)))
    lay.append(("bh", (12,)))
    return lay


def n_params() -> int:
    return int(sum(np.prod(s) for _, s in param_layout()))


def unflatten(theta):
    out, o = {}, 0
    for name, shape in param_layout():
        n = int(np.prod(shape))
        out[name] = np.asarray(theta[o:o + n], np.float64).reshape(shape)
        o += n
    return out


def flatten(grads) -> np.ndarray:
    return np.concatenate([np.asarray(grads[name], np.float64).ravel() for name, _ in param_layout()])


def pack(ref, cur) -> np.ndarray:
    """[8, H/2, W/2]: R, G(R row), G(B row), B planes of ref then cur, v/2048 - 1."""
    planes = []
    for f in (ref, cur):
        f = np.asarray(f, np.float64)
        for py, px in ((0, 0), (0, 1), (1, 0), (1, 1)):
            planes.append(f[py::2, px::2] / 2048.0 - 1.0)
    return np.stack(planes)


def conv_out(n: int) -> int:
    return (n - 1) // 2 + 1


def conv3x3s2(x, w, b):
    """y[o, i, k] = b[o] + sum_{c, ky, kx} w[o, c, ky, kx] x[c, 2i + ky - 1, 2k + kx - 1]
    (zero outside the map)."""
    C, H, W = x.shape
    Ho, Wo = conv_out(H), conv_out(W)
    xp = np.zeros((C, H + 2, W + 2))
    xp[:, 1:H + 1, 1:W + 1] = x
    y = np.zeros((w.shape[0], Ho, Wo))
    for ky in range(3):
        for kx in range(3):
            tap = xp[:, ky:ky + 2 * Ho:2, kx:kx + 2 * Wo:2]
            y += np.einsum("oc,chw->ohw", w[:, :, ky, kx], tap)
    return y + b[:, None, None]


def conv3x3s2_backward(x, w, dy):
    """Gradients of conv3x3s2 w.r.t. x, w, b given dL/dy."""
    C, H, W = x.shape
    Ho, Wo = dy.shape[1:]
    xp = np.zeros((C, H + 2, W + 2))
    xp[:, 1:H + 1, 1:W + 1] = x
    dxp = np.zeros_like(xp)
    dw = np.zeros_like(w)
    for ky in range(3):
        for kx in range(3):
            tap = xp[:, ky:ky + 2 * Ho:2, kx:kx + 2 * Wo:2]
            dw[:, :, ky, kx] = np.einsum("ohw,chw->oc", dy, tap)
            dxp[:, ky:ky + 2 * Ho:2, kx:kx + 2 * Wo:2] += np.einsum("oc,ohw->chw", w[:, :, ky, kx], dy)
    return dxp[:, 1:H + 1, 1:W + 1], dw, dy.sum(axis=(1, 2))


def round_bf16(x) -> np.ndarray:
    """float64 -> float32 -> bfloat16 (round to nearest, ties to even) -> float64."""
    b = np.asarray(x, np.float32).view(np.uint32).astype(np.uint64)
    b = (b + 0x7FFF + ((b >> 16) & 1)) & 0xFFFF0000
    return b.astype(np.uint32).view(np.float32).astype(np.float64)


def forward(theta, ref, cur, search_range: int, act_round=None):
    """Returns (dx, dy, conf) each [h, w] and the cache for ``backward``."""
    p = unflatten(theta)
    acts = [pack(ref, cur)]
    pre = []
    for l in range(N_LAYERS):
        z = conv3x3s2(acts[-1], p[f"w{l + 1}"], p[f"b{l + 1}"])
        pre.append(z)
        a = np.maximum(z, 0.0)
        acts.append(round_bf16(a) if act_round == "bf16" else a)
    x4 = acts[-1]
    zh = np.einsum("jc,chw->jhw", p["wh"], x4) + p["bh"][:, None, None]
    h4, w4 = x4.shape[1:]
    z = np.zeros((3, 2 * h4, 2 * w4))
    for sy in range(2):
        for sx in range(2):
            for q in range(3):
                z[q, sy::2, sx::2] = zh[3 * (2 * sy + sx) + q]
    dx = search_range * np.tanh(z[0])
    dy = search_range * np.tanh(z[1])
    conf = 1.0 / (1.0 + np.exp(-z[2]))
    cache = dict(p=p, acts=acts, pre=pre, z=z, range=search_range)
    return dx, dy, conf, cache


def round_even(v):
    """Nearest even integer, halves away from zero (the seeded refine's centre)."""
    return 2.0 * np.sign(v / 2.0) * np.floor(np.abs(v / 2.0) + 0.5)


def berhu(e, c=BERHU_C):
    a = np.abs(e)
    return np.where(a <= c, a, (e * e + c * c) / (2 * c))


def berhu_grad(e, c=BERHU_C):
    return np.where(np.abs(e) <= c, np.sign(e), e / c)


def loss_and_grad(theta, ref, cur, label_dx, label_dy, search_range: int, act_round=None, neg_weight=1.0,
                  grad_round=None):
    """Mean loss over blocks and its gradient w.r.t. theta (float64)."""
    loss, cache, dz = loss_and_dz(theta, ref, cur, label_dx, label_dy, search_range, act_round, neg_weight)
    return loss, backward(cache, dz, grad_round)


def loss_and_dz(theta, ref, cur, label_dx, label_dy, search_range: int, act_round=None, neg_weight=1.0):
    """Mean loss over blocks, the forward cache and dL/dz for ``backward``."""
    dx, dy, conf, cache = forward(theta, ref, cur, search_range, act_round)
    n = dx.size
    ex, ey = dx - label_dx, dy - label_dy
    t = ((np.abs(round_even(dx) - label_dx) <= 4) & (np.abs(round_even(dy) - label_dy) <= 4)).astype(np.float64)
    eps = 1e-12
    bce = -(t * np.log(conf + eps) + neg_weight * (1 - t) * np.log(1 - conf + eps))
    loss = float((berhu(ex) + berhu(ey) + bce).sum() / n)
    z = cache["z"]
    R = cache["range"]
    dz = np.zeros_like(z)
    dz[0] = berhu_grad(ex) * R * (1 - np.tanh(z[0]) ** 2) / n
    dz[1] = berhu_grad(ey) * R * (1 - np.tanh(z[1]) ** 2) / n
    dz[2] = (conf * (t + neg_weight * (1 - t)) - t) / n
    return loss, cache, dz


def backward(cache, dz, grad_round=None):
    """Gradient w.r.t. theta.  ``grad_round="bf16"``: each layer's
    pre-activation gradient is rounded to bfloat16 (as the network's training
    definition stores it) before it enters that layer's weight and input
    gradients; otherwise it stays float64."""
    p, acts, pre = cache["p"], cache["acts"], cache["pre"]
    rnd = round_bf16 if grad_round == "bf16" else (lambda v: v)
    x4 = acts[-1]
    h4, w4 = x4.shape[1:]
    dzh = np.zeros((12, h4, w4))
    for sy in range(2):
        for sx in range(2):
            for q in range(3):
                dzh[3 * (2 * sy + sx) + q] = dz[q, sy::2, sx::2]
    g = {"wh": np.einsum("jhw,chw->jc", dzh, x4), "bh": dzh.sum(axis=(1, 2))}
    da = np.einsum("jc,jhw->chw", p["wh"], dzh)
    for l in reversed(range(N_LAYERS)):
        dpre = rnd(da * (pre[l] > 0))
        dxin, g[f"w{l + 1}"], g[f"b{l + 1}"] = conv3x3s2_backward(acts[l], p[f"w{l + 1}"], dpre)
        da = dxin
    return flatten(g)
