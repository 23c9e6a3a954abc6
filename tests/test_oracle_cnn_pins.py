"""Pins of the float64 proposal-network oracle (oracle/cnn.py): its convolution
against torch's float64 conv2d, its whole forward and gradient against torch
autograd in float64 (library routines computing the same functions), and its
gradient against central finite differences."""
import numpy as np
import pytest
import torch
import torch.nn.functional as F

from oracle import cnn
from paper_2508_05990_b300 import synth


def shapes():
    return [("b" if n.startswith("b") else "w", s) for n, s in cnn.param_layout()]


@pytest.mark.parametrize("C,H,W", [(8, 17, 24), (32, 16, 9), (3, 5, 5)])
def test_conv_matches_torch(C, H, W):
    rng = np.random.default_rng(C + H)
    x = rng.normal(size=(C, H, W))
    w = rng.normal(size=(32, C, 3, 3))
    b = rng.normal(size=32)
    want = F.conv2d(torch.from_numpy(x)[None], torch.from_numpy(w), torch.from_numpy(b), stride=2, padding=1)[0]
    np.testing.assert_allclose(cnn.conv3x3s2(x, w, b), want.numpy(), rtol=1e-12, atol=1e-12)


def torch_forward(theta, ref, cur, R):
    p = {k: torch.from_numpy(v).requires_grad_(True) for k, v in cnn.unflatten(theta).items()}
    x = torch.from_numpy(cnn.pack(ref, cur))[None]
    for l in range(4):
        x = F.relu(F.conv2d(x, p[f"w{l + 1}"], p[f"b{l + 1}"], stride=2, padding=1))
    zh = torch.einsum("jc,bchw->bjhw", p["wh"], x) + p["bh"][None, :, None, None]
    # channel j = 3 * (2 sy + sx) + q  ->  [q, 2h, 2w]
    h4, w4 = zh.shape[2:]
    z = zh[0].reshape(2, 2, 3, h4, w4).permute(2, 3, 0, 4, 1).reshape(3, 2 * h4, 2 * w4)
    return R * torch.tanh(z[0]), R * torch.tanh(z[1]), torch.sigmoid(z[2]), p


@pytest.mark.parametrize("H,W", [(40, 96), (72, 64)])
def test_forward_matches_torch_off_multiples_of_32(H, W):
    """Heights that are no multiple of 32 (the learned search's 1080-row and
    720-row case in small): every layer takes its natural ceil(n / 2) size,
    torch's stride-2 conv with padding 1 included, and the depth-to-space
    output has 2 ceil(H / 32) >= ceil(H / 16) block rows."""
    ref, cur = synth.pan_clip(5, H, W, n_frames=2, rect_size=(8, 16))
    theta = synth.he_normal_params(14, shapes()).astype(np.float64)
    dx, dy, conf, _ = cnn.forward(theta, ref, cur, 32)
    tdx, tdy, tconf, _ = torch_forward(theta, ref, cur, 32)
    assert dx.shape == (2 * (-(-H // 32)), W // 16) and dx.shape[0] >= -(-H // 16)
    np.testing.assert_allclose(dx, tdx.detach().numpy(), rtol=1e-10, atol=1e-10)
    np.testing.assert_allclose(dy, tdy.detach().numpy(), rtol=1e-10, atol=1e-10)
    np.testing.assert_allclose(conf, tconf.detach().numpy(), rtol=1e-10, atol=1e-12)


def test_forward_and_gradient_match_torch_autograd():
    ref, cur = synth.pan_clip(3, 64, 96, n_frames=2, rect_size=(8, 24))
    theta = synth.he_normal_params(11, shapes()).astype(np.float64)
    R = 32
    dx, dy, conf, _ = cnn.forward(theta, ref, cur, R)
    tdx, tdy, tconf, p = torch_forward(theta, ref, cur, R)
    np.testing.assert_allclose(dx, tdx.detach().numpy(), rtol=1e-10, atol=1e-10)
    np.testing.assert_allclose(conf, tconf.detach().numpy(), rtol=1e-10, atol=1e-12)
    rng = np.random.default_rng(4)
    ldx = 2.0 * rng.integers(-16, 17, dx.shape)
    ldy = 2.0 * rng.integers(-16, 17, dx.shape)
    loss, g = cnn.loss_and_grad(theta, ref, cur, ldx, ldy, R)
    # same loss in torch; the confidence target is a constant of the prediction
    t = ((np.abs(cnn.round_even(dx) - ldx) <= 4) & (np.abs(cnn.round_even(dy) - ldy) <= 4)).astype(np.float64)
    c = cnn.BERHU_C

    def bh(e):
        a = e.abs()
        return torch.where(a <= c, a, (e * e + c * c) / (2 * c))
    tt = torch.from_numpy(t)
    tl = (bh(tdx - torch.from_numpy(ldx)) + bh(tdy - torch.from_numpy(ldy))
          - (tt * torch.log(tconf + 1e-12) + (1 - tt) * torch.log(1 - tconf + 1e-12))).mean()
    tl.backward()
    assert abs(tl.item() - loss) < 1e-10
    tg = np.concatenate([p[n].grad.numpy().ravel() for n, _ in cnn.param_layout()])
    np.testing.assert_allclose(g, tg, rtol=1e-8, atol=1e-12)


@pytest.mark.parametrize("neg_weight", [1.0, 6.0])
def test_gradient_matches_finite_differences(neg_weight):
    ref, cur = synth.pan_clip(5, 64, 64, n_frames=2, rect_size=(8, 24))
    theta = synth.he_normal_params(12, shapes()).astype(np.float64)
    rng = np.random.default_rng(6)
    ldx = 2.0 * rng.integers(-8, 9, (4, 4))
    ldy = 2.0 * rng.integers(-8, 9, (4, 4))
    _, g = cnn.loss_and_grad(theta, ref, cur, ldx, ldy, 16, neg_weight=neg_weight)
    idx = np.concatenate([rng.choice(2304, 6, replace=False), 2304 + rng.choice(32, 3, replace=False),
                          rng.choice(np.arange(2336, cnn.n_params()), 12, replace=False)])
    h = 1e-6
    for i in idx:
        tp, tm = theta.copy(), theta.copy()
        tp[i] += h
        tm[i] -= h
        fd = (cnn.loss_and_grad(tp, ref, cur, ldx, ldy, 16, neg_weight=neg_weight)[0]
              - cnn.loss_and_grad(tm, ref, cur, ldx, ldy, 16, neg_weight=neg_weight)[0]) / (2 * h)
        assert abs(fd - g[i]) <= 1e-6 + 1e-5 * abs(g[i]), (i, fd, g[i])


def test_pack_planes():
    f = np.arange(16, dtype=np.uint16).reshape(4, 4)
    x = cnn.pack(f, f + 100)
    assert x.shape == (8, 2, 2)
    np.testing.assert_allclose(x[0], f[0::2, 0::2] / 2048 - 1)
    np.testing.assert_allclose(x[2], f[1::2, 0::2] / 2048 - 1)
    np.testing.assert_allclose(x[7], (f[1::2, 1::2] + 100) / 2048 - 1)
    assert cnn.n_params() == 30476


def test_round_bf16_matches_torch():
    rng = np.random.default_rng(1)
    x = np.concatenate([rng.normal(size=1000) * 10.0 ** rng.integers(-5, 5, 1000), [0.0, -0.0, 1.0, 3.0, 1 + 2 ** -8]])
    want = torch.from_numpy(x).float().bfloat16().double().numpy()
    np.testing.assert_array_equal(cnn.round_bf16(x), want)


def test_refine_conv_matches_torch():
    """oracle/refine.py: stride-1 3x3 convolution (NHWC) against torch's float64 conv2d."""
    from oracle import refine
    rng = np.random.default_rng(12)
    x = rng.normal(size=(9, 13, 16))
    w = rng.normal(size=(8, 16, 3, 3))
    b = rng.normal(size=8)
    want = F.conv2d(torch.from_numpy(x.transpose(2, 0, 1))[None], torch.from_numpy(w), torch.from_numpy(b),
                    padding=1)[0].numpy().transpose(1, 2, 0)
    np.testing.assert_allclose(refine.conv3x3(x, w, b), want, rtol=1e-12, atol=1e-12)
    w2, w3 = rng.normal(size=(8, 8, 3, 3)), rng.normal(size=(16, 8, 3, 3))
    t = torch.from_numpy(x.transpose(2, 0, 1))[None]
    t = F.relu(F.conv2d(t, torch.from_numpy(w), torch.from_numpy(b), padding=1))
    t = F.relu(F.conv2d(t, torch.from_numpy(w2), torch.zeros(8, dtype=torch.float64), padding=1))
    t = F.conv2d(t, torch.from_numpy(w3), torch.zeros(16, dtype=torch.float64), padding=1)
    np.testing.assert_allclose(refine.refine(x, w, b, w2, np.zeros(8), w3, np.zeros(16)),
                               t[0].numpy().transpose(1, 2, 0), rtol=1e-11, atol=1e-11)


def test_gradient_rounding_matches_torch_hooks():
    """grad_round="bf16" rounds each layer's pre-activation gradient: the same
    network in torch float64 with a backward hook on every pre-activation that
    rounds its gradient to bfloat16 (float32 first) gives the same gradient."""
    ref, cur = synth.pan_clip(7, 64, 96, n_frames=2, rect_size=(8, 24))
    theta = synth.he_normal_params(13, shapes()).astype(np.float64)
    R = 32
    rng = np.random.default_rng(9)
    ldx = 2.0 * rng.integers(-16, 17, (4, 6))
    ldy = 2.0 * rng.integers(-16, 17, (4, 6))
    _, g = cnn.loss_and_grad(theta, ref, cur, ldx, ldy, R, grad_round="bf16")
    _, g_exact = cnn.loss_and_grad(theta, ref, cur, ldx, ldy, R)
    assert not np.allclose(g, g_exact, rtol=1e-6, atol=0)  # the rounding is there

    def rnd(t):
        return torch.from_numpy(cnn.round_bf16(t.detach().numpy()))

    p = {k: torch.from_numpy(v).requires_grad_(True) for k, v in cnn.unflatten(theta).items()}
    x = torch.from_numpy(cnn.pack(ref, cur))[None]
    for l in range(4):
        z = F.conv2d(x, p[f"w{l + 1}"], p[f"b{l + 1}"], stride=2, padding=1)
        z.register_hook(rnd)
        x = F.relu(z)
    zh = torch.einsum("jc,bchw->bjhw", p["wh"], x) + p["bh"][None, :, None, None]
    h4, w4 = zh.shape[2:]
    z = zh[0].reshape(2, 2, 3, h4, w4).permute(2, 3, 0, 4, 1).reshape(3, 2 * h4, 2 * w4)
    tdx, tdy, tconf = R * torch.tanh(z[0]), R * torch.tanh(z[1]), torch.sigmoid(z[2])
    dx = tdx.detach().numpy()
    dy = tdy.detach().numpy()
    t = ((np.abs(cnn.round_even(dx) - ldx) <= 4) & (np.abs(cnn.round_even(dy) - ldy) <= 4)).astype(np.float64)
    c = cnn.BERHU_C

    def bh(e):
        a = e.abs()
        return torch.where(a <= c, a, (e * e + c * c) / (2 * c))
    tt = torch.from_numpy(t)
    tl = (bh(tdx - torch.from_numpy(ldx)) + bh(tdy - torch.from_numpy(ldy))
          - (tt * torch.log(tconf + 1e-12) + (1 - tt) * torch.log(1 - tconf + 1e-12))).mean()
    tl.backward()
    tg = np.concatenate([p[n].grad.numpy().ravel() for n, _ in cnn.param_layout()])
    np.testing.assert_allclose(g, tg, rtol=1e-9, atol=1e-13)
