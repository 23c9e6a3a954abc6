"""Learned proposal network and learned-seeded search on the GPU vs the oracle.

The network's weights and activations are bfloat16 with float32 accumulation.
The oracle (oracle/cnn.py) evaluates the same bf16 weights in float64, either
keeping activations exact (act_round=None) or rounding them to bfloat16 at the
points the network's definition stores them (act_round="bf16").

Forward, per block (tests/fp_bounds.py states the measure): with z the exact
head logits and m_z = |b_h| + sum |w_h| |x4| the absolute sum of their terms,
every output (dx, dy, conf) must come from logits within 2e-2 m_z of the exact
oracle's and within 2^-7 m_z of the bfloat16-rounded oracle's (tanh and the
sigmoid are monotone, so this is an interval test on the outputs).

Gradient, per parameter: within 2^-8 M (+ a floor of 2^-8 * 1e-3 * max M) of
the oracle with the network's training roundings modelled (bf16 activations
and bf16 pre-activation gradients, the operands of the tensor-core backward),
M being the sum of the absolute values of every term of the parameter's
chain-rule expansion; the two differ only in the order of the float32 sums
(and where that flips the bfloat16 rounding or the ReLU mask of a value at a
boundary).  Against the exact float64 oracle the
gradient is compared normwise (5e-2): rounding the activations to bfloat16
moves the loss surface itself, ReLU masks included, so no per-parameter bound
against the exact gradient exists (measured: 3.2 %, identical for the GPU and
for the bf16-activation oracle).
Integer outputs (MV fields) are compared bit for bit.
"""
import numpy as np
import pytest

import fp_bounds as fb
import oracle
from oracle import cnn
from paper_2508_05990_b300 import bayer_me as bm
from paper_2508_05990_b300 import synth

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def handle():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2508_05990_b300 import build
    build.build()
    h = bm.Handle(0)
    yield h
    h.close()


def dev(a):
    return torch.from_numpy(np.ascontiguousarray(a)).cuda()


def weights(seed):
    theta = synth.he_normal_params(seed, bm.CNN_SHAPES)
    w32 = torch.from_numpy(theta).cuda()
    wbf = bm.to_bf16_bits(w32)
    theta_bf = w32.to(torch.bfloat16).double().cpu().numpy()  # the values the GPU uses, exactly
    return w32, wbf, theta_bf


def rel(a, b):
    return float(np.linalg.norm(np.asarray(a, np.float64) - b) / max(np.linalg.norm(b), 1e-30))


def check_forward(prop, conf, theta, ref, cur, R=32):
    """Every block's outputs against both oracles (see the module docstring).
    The network's 2 ceil(H/32) block rows are cropped to the block grid's
    ceil(H/16) (the header's definition), which the GPU's outputs have."""
    h, w = conf.shape
    assert h == -(-ref.shape[0] // 16) and w == ref.shape[1] // 16
    z, mz, _ = fb.cnn_logits(theta, ref, cur, R)
    zb, _, _ = fb.cnn_logits(theta, ref, cur, R, act_round="bf16")
    z, mz, zb = z[:, :h, :w], mz[:, :h, :w], zb[:, :h, :w]
    ok = fb.outputs_within(prop, conf, z, fb.TOL_BF16 * mz, R)
    assert ok.all(), ("vs exact", np.argwhere(~ok)[:5])
    ok = fb.outputs_within(prop, conf, zb, fb.TOL_CNN_SAME_ROUNDING * mz, R)
    assert ok.all(), ("vs bf16-rounded", np.argwhere(~ok)[:5])


@pytest.mark.parametrize("shape", [(128, 192), (1088, 1920), (64, 2048), (96, 2080), (1080, 1920), (720, 1280),
                                   (72, 2080)])
def test_cnn_forward_matches_oracle(handle, shape):
    """128x192 and 1088x1920: layers 3, 4 and the head in one kernel; 64x2048:
    its widest case (layer-3 rows of 128 pixels); 96x2080: layer-3 rows of 130
    pixels, so the per-tile layer-3 and layer-4 kernels run instead (and H4 = 3
    leaves the last layer-4 row pair half outside the map).  Heights that are
    no multiple of 32: 1080 (layer 2's 135 rows make layer 3 read its zero pad
    row; 68 block rows, the last 8 pixels high), 720 (46 network block rows
    cropped to 45) and 72 with the per-tile kernels (6 rows cropped to 5)."""
    H, W = shape
    ref, cur = synth.pan_clip(90, H, W, n_frames=2, rect_size=(16, 64))
    _, wbf, theta = weights(3)
    prop, conf = handle.cnn_forward(dev(ref), dev(cur), wbf, 32)
    check_forward(prop[0].cpu().numpy(), conf[0].cpu().numpy(), theta, ref, cur)


def test_cnn_forward_batched_strides(handle):
    H, W = 96, 128
    frames = synth.pan_clip(91, H, W, n_frames=4, rect_size=(8, 32))
    _, wbf, theta = weights(4)
    d = dev(frames)
    prop, conf = handle.cnn_forward(d, d[1:], wbf, 16, batch=3, ref_batch_stride=H * W, cur_batch_stride=H * W)
    for t in range(3):
        check_forward(prop[t].cpu().numpy(), conf[t].cpu().numpy(), theta, frames[t], frames[t + 1], 16)


@pytest.mark.parametrize("shape,neg_weight,offset", [((128, 192), 1.0, 0), ((128, 192), 8.0, 0),
                                                     ((64, 1088), 5.0, 0), ((1088, 1920), 5.0, 0),
                                                     ((128, 192), 1.0, 2), ((128, 192), 1.0, 1)])
def test_cnn_loss_and_gradient_match_oracle(handle, shape, neg_weight, offset):
    """Loss and gradient of a batch of 2 pairs.  128x192: every backward
    launch covers a ragged tail (a layer's last row segment of 64 pixels
    partly past the row; input gradients: one partial 128-column tile) and the
    layer-1 weight gradient runs 4 pipelined chunks per CTA.  64x1088: the
    input gradient of layer 2 spans two column tiles (136 = 128 + 8).
    1088x1920, the training resolution: every CTA loops over several tiles
    and chunks.  offset: the frames start `offset` samples into their buffer,
    so that the layer-1 weight gradient loads the samples itself (4-byte loads
    at offset 2, 2-byte loads at offset 1) instead of copying 16-byte pieces
    of raw rows."""
    H, W = shape
    frames = synth.pan_clip(92, H, W, n_frames=3, rect_size=(16, 48))
    _, wbf, theta = weights(5)
    rng = np.random.default_rng(8)
    h, w = H // 16, W // 16
    labels = np.zeros((2, h, w), oracle.MV_DTYPE)
    labels["dx"] = 2 * rng.integers(-16, 17, (2, h, w))
    labels["dy"] = 2 * rng.integers(-16, 17, (2, h, w))
    d = dev(frames)
    if offset:
        flat = torch.zeros(d.numel() + 8, dtype=d.dtype, device="cuda")
        flat[offset:offset + d.numel()].copy_(d.reshape(-1))
        d = flat[offset:offset + d.numel()].view(d.shape)
    lab = dev(labels.view(np.int32).reshape(2, h, w, 2))
    grad, loss = handle.cnn_loss_grad(d, d[1:], wbf, lab, 32, batch=2, ref_batch_stride=H * W, cur_batch_stride=H * W,
                                      neg_weight=neg_weight)
    assert handle.sync_status() == bm.OK
    g = grad.cpu().numpy()
    losses, grads = [], []
    for t in range(2):
        l, gr = cnn.loss_and_grad(theta, frames[t], frames[t + 1], labels["dx"][t].astype(np.float64),
                                  labels["dy"][t].astype(np.float64), 32, neg_weight=neg_weight)
        losses.append(l)
        grads.append(gr)
    want_loss, want_grad = np.mean(losses), np.mean(grads, axis=0)
    assert abs(float(loss.item()) - want_loss) <= fb.TOL_BF16 * abs(want_loss)
    assert rel(g, want_grad) < 5e-2
    # per parameter against the same network with its bfloat16 activation and
    # pre-activation-gradient roundings modelled
    gb, Mb = zip(*[fb.cnn_grad_magnitudes(theta, frames[t], frames[t + 1], labels["dx"][t].astype(np.float64),
                                          labels["dy"][t].astype(np.float64), 32, neg_weight=neg_weight,
                                          act_round="bf16", grad_round="bf16") for t in range(2)])
    gb, Mb = np.mean(gb, axis=0), np.mean(Mb, axis=0)
    t = fb.TOL_BF16_SAME_ROUNDING
    bound = t * Mb + t * 1e-3 * Mb.max()
    worst = int(np.argmax(np.abs(g - gb) - bound))
    assert np.all(np.abs(g - gb) <= bound), (worst, g[worst], gb[worst], Mb[worst])


def test_adamw_matches_formula(handle):
    rng = np.random.default_rng(2)
    n = bm.CNN_NPARAMS
    w0, g, m0, v0 = (rng.normal(size=n).astype(np.float32) for _ in range(4))
    v0 = np.abs(v0)
    w, m, v = dev(w0.copy()), dev(m0.copy()), dev(v0.copy())
    wb = torch.empty(n, dtype=torch.int16, device="cuda")
    lr, b1, b2, eps, wd, step = 1e-3, 0.9, 0.999, 1e-8, 0.01, 7
    handle.cnn_adamw(w, wb, dev(g), m, v, step, lr, b1, b2, eps, wd)
    mm = b1 * m0.astype(np.float64) + (1 - b1) * g
    vv = b2 * v0.astype(np.float64) + (1 - b2) * g.astype(np.float64) ** 2
    ww = w0 - lr * ((mm / (1 - b1 ** step)) / (np.sqrt(vv / (1 - b2 ** step)) + eps) + wd * w0)
    np.testing.assert_allclose(w.cpu().numpy(), ww, rtol=1e-5, atol=1e-7)
    np.testing.assert_allclose(m.cpu().numpy(), mm, rtol=1e-5, atol=1e-7)
    assert torch.equal(wb, bm.to_bf16_bits(w))


def test_learned_equals_seeded_mode_on_network_proposals(handle):
    H, W = 256, 384
    frames = synth.pan_clip(93, H, W, n_frames=3, rect_size=(16, 64))
    _, wbf, _ = weights(6)
    d = dev(frames)
    kw = dict(batch=2, ref_batch_stride=H * W, cur_batch_stride=H * W)
    fb = torch.empty((2, H // 16, W // 16), dtype=torch.uint8, device="cuda")
    nfb = torch.zeros(1, dtype=torch.int32, device="cuda")
    got = handle.estimate_learned(d, d[1:], wbf, 32, 0.5, fallback=fb, n_fallback=nfb, **kw)
    prop, conf = handle.cnn_forward(d, d[1:], wbf, 32, **kw)
    fb2 = torch.empty_like(fb)
    want = handle.estimate_ex(d, d[1:], mode=bm.MODE_SEEDED, search_range=32, prop_dxdy=prop, conf=conf,
                              fallback=fb2, **kw)
    torch.cuda.synchronize()
    assert torch.equal(got, want) and torch.equal(fb, fb2)
    assert int(nfb.item()) == int(fb.sum().item())


@pytest.mark.parametrize("H", [224, 216, 210])
@pytest.mark.parametrize("mode", ["all_fallback", "at_optimum", "mixed", "mixed_odd_pitch"])
def test_seeded_fast_path_vs_oracle(handle, mode, H):
    """SEEDED mode (block 16, EVEN, +-32) vs the oracle on a 14 x 20-block frame
    (the second CTA of 256 blocks is partial); "mixed_odd_pitch" stores the
    frames with a row pitch of 321 samples, which rules out paired loads.
    H = 216 and 210: the last block row is clipped to 8 and 2 rows (the
    refine's and the fallback list kernel's clipped forms)."""
    W = 320
    frames = synth.pan_clip(94, H, W, n_frames=2, rect_size=(16, 64))
    h, w = -(-H // 16), W // 16
    full, _ = oracle.me_full(frames[0], frames[1], 16, 32, even=True)
    if mode == "all_fallback":
        pdx = pdy = np.zeros((h, w), np.float32)
        conf = np.zeros((h, w), np.float32)
    elif mode == "at_optimum":
        pdx, pdy = full["dx"].astype(np.float32), full["dy"].astype(np.float32)
        conf = np.ones((h, w), np.float32)
    else:
        pdx, pdy, conf = synth.proposals(95, h, w, 32, true_mv=np.stack([full["dx"], full["dy"]], -1), jitter=4.0)
    prop = np.stack([pdx, pdy], -1)
    if mode == "mixed_odd_pitch":
        padded = np.zeros((2, H, W + 1), np.uint16)
        padded[:, :, :W] = frames
        d = dev(padded)
        out = handle.estimate_ex(d[0], d[1], mode=bm.MODE_SEEDED, search_range=32, prop_dxdy=dev(prop),
                                 conf=dev(conf), W=W, H=H, pitch=W + 1)
    else:
        out = handle.estimate_ex(dev(frames[0]), dev(frames[1]), mode=bm.MODE_SEEDED, search_range=32,
                                 prop_dxdy=dev(prop), conf=dev(conf))
    want, _, _ = oracle.me_seeded(frames[0], frames[1], 16, 32, pdx, pdy, conf)
    g = bm.records_to_numpy(out[0])
    for k in ("dx", "dy", "sad"):
        np.testing.assert_array_equal(g[k], want[k])
    if mode in ("all_fallback", "at_optimum"):
        for k in ("dx", "dy", "sad"):
            np.testing.assert_array_equal(g[k], full[k])


def test_learned_1080p_clip_as_benchmarked(handle):
    """The benchmark's learned-seeded step: the 7 pairs of the 1080p clip in
    one call with the committed trained weights.  Equals SEEDED mode on the
    network's own proposals bit for bit (fallback flags too), and two pairs
    equal the oracle's seeded search given those proposals."""
    import os
    wl = synth.WORKLOADS["1080p"]
    H, W = wl["H"], wl["W"]
    frames = synth.pan_clip(wl["seed"], H, W, n_frames=wl["frames"])
    d = dev(frames)
    path = os.path.join(os.path.dirname(os.path.dirname(os.path.abspath(__file__))), "paper_2508_05990_b300",
                        "weights", "proposal_1080p_r32.npz")
    wbf = bm.to_bf16_bits(torch.from_numpy(np.load(path)["theta"].astype(np.float32)).cuda()).contiguous()
    kw = dict(batch=7, ref_batch_stride=H * W, cur_batch_stride=H * W)
    fb = torch.empty((7, H // 16, W // 16), dtype=torch.uint8, device="cuda")
    got = handle.estimate_learned(d, d[1:], wbf, 32, 0.5, fallback=fb, **kw)
    prop, conf = handle.cnn_forward(d, d[1:], wbf, 32, **kw)
    fb2 = torch.empty_like(fb)
    want = handle.estimate_ex(d, d[1:], mode=bm.MODE_SEEDED, search_range=32, prop_dxdy=prop, conf=conf,
                              fallback=fb2, **kw)
    torch.cuda.synchronize()
    assert torch.equal(got, want) and torch.equal(fb, fb2)
    p, c = prop.cpu().numpy(), conf.cpu().numpy()
    for t in (0, 6):
        ref_field, ref_fb, _ = oracle.me_seeded(frames[t], frames[t + 1], 16, 32, p[t, ..., 0], p[t, ..., 1], c[t])
        g = bm.records_to_numpy(got[t])
        for k in ("dx", "dy", "sad"):
            np.testing.assert_array_equal(g[k], ref_field[k])
        np.testing.assert_array_equal(fb[t].cpu().numpy(), ref_fb)


def test_learned_1920x1080(handle):
    """The learned-seeded search on real 1080-row frames (the last block row 8
    rows high, the network's layer 3 reading its zero pad row): equal to SEEDED
    mode on the network's own proposals bit for bit, and to the oracle's
    seeded search given those proposals for two pairs; the network's outputs
    for the first pair within the forward bounds."""
    import os
    H, W = 1080, 1920
    frames = synth.pan_clip(synth.WORKLOADS["1080p"]["seed"], H, W, n_frames=4)
    d = dev(frames)
    path = os.path.join(os.path.dirname(os.path.dirname(os.path.abspath(__file__))), "paper_2508_05990_b300",
                        "weights", "proposal_1080p_r32.npz")
    theta32 = torch.from_numpy(np.load(path)["theta"].astype(np.float32)).cuda()
    wbf = bm.to_bf16_bits(theta32).contiguous()
    kw = dict(batch=3, ref_batch_stride=H * W, cur_batch_stride=H * W)
    h, w = 68, 120
    fbk = torch.empty((3, h, w), dtype=torch.uint8, device="cuda")
    got = handle.estimate_learned(d, d[1:], wbf, 32, 0.5, fallback=fbk, **kw)
    assert tuple(got.shape) == (3, h, w, 2)
    prop, conf = handle.cnn_forward(d, d[1:], wbf, 32, **kw)
    fb2 = torch.empty_like(fbk)
    want = handle.estimate_ex(d, d[1:], mode=bm.MODE_SEEDED, search_range=32, prop_dxdy=prop, conf=conf,
                              fallback=fb2, **kw)
    torch.cuda.synchronize()
    assert handle.sync_status() == bm.OK
    assert torch.equal(got, want) and torch.equal(fbk, fb2)
    last = fbk[:, -1].cpu().numpy()
    assert last.any() and not last.all(), "the clipped block row should hold refined and fallback blocks"
    p, c = prop.cpu().numpy(), conf.cpu().numpy()
    for t in (0, 2):
        ref_field, ref_fb, _ = oracle.me_seeded(frames[t], frames[t + 1], 16, 32, p[t, ..., 0], p[t, ..., 1], c[t])
        g = bm.records_to_numpy(got[t])
        for k in ("dx", "dy", "sad"):
            np.testing.assert_array_equal(g[k], ref_field[k])
        np.testing.assert_array_equal(fbk[t].cpu().numpy(), ref_fb)
    theta_bf = theta32.to(torch.bfloat16).double().cpu().numpy()
    check_forward(p[0], c[0], theta_bf, frames[0], frames[1])


def test_network_size_rules(handle):
    """Inference takes H % 8 == 0 and W % 32 == 0; the loss keeps H % 32 == 0;
    other sizes return BAYER_ERR_UNSUPPORTED and launch nothing."""
    _, wbf, _ = weights(6)
    f = torch.zeros((2, 1084, 1920), dtype=torch.int16, device="cuda")  # 1084 % 8 == 4
    for call in (lambda: handle.cnn_forward(f[0], f[1], wbf, 32),
                 lambda: handle.estimate_learned(f[0], f[1], wbf, 32, 0.5)):
        with pytest.raises(bm.BayerError) as e:
            call()
        assert e.value.status == bm.ERR_UNSUPPORTED
    g = torch.zeros((2, 1080, 1936), dtype=torch.int16, device="cuda")  # 1936 % 32 == 16
    with pytest.raises(bm.BayerError) as e:
        handle.cnn_forward(g[0], g[1], wbf, 32)
    assert e.value.status == bm.ERR_UNSUPPORTED
    k = torch.zeros((2, 1080, 1920), dtype=torch.int16, device="cuda")
    labels = torch.zeros((1, 68, 120, 2), dtype=torch.int32, device="cuda")
    with pytest.raises(bm.BayerError) as e:
        handle.cnn_loss_grad(k[0], k[1], wbf, labels, 32)
    assert e.value.status == bm.ERR_UNSUPPORTED
    prop, conf = handle.cnn_forward(k[0], k[1], wbf, 32)  # 1080 rows: accepted, 68 block rows
    assert tuple(conf.shape) == (1, 68, 120)
    torch.cuda.synchronize()
    assert handle.sync_status() == bm.OK
