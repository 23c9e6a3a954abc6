"""CUDA path vs the CPU oracle, through the C ABI, element by element.

Motion vectors and SADs are integers and must match bit for bit; NEAREST
propagation is a copy and must match bit for bit; BILINEAR propagation must
match the oracle's float evaluation (same operation order, each operation
rounded) bit for bit, and the double-precision oracle within a relative error
of 1e-5 (the float32 bound for this op: six roundings of a convex combination
give at most 8 * 2^-24 ~ 4.8e-7 relative to sum |w_i a_i|).
"""
import numpy as np
import pytest

import oracle
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


def assert_fields_equal(gpu_records, oracle_field):
    g = bm.records_to_numpy(gpu_records)
    g = g.reshape(oracle_field.shape)
    for k in ("dx", "dy", "sad"):
        bad = np.argwhere(g[k] != oracle_field[k])
        assert bad.size == 0, f"{k} differs at {bad[:5].tolist()}: gpu {g[bad[0][0]][bad[0][1]] if bad.size else ''}"


# ----------------------------------------------------------------------------
# exhaustive search
# ----------------------------------------------------------------------------

def test_parity_256_planted(handle):
    """The 256x256 planted-shift pair: block 16, +-16 EVEN (fast kernel R = 8)."""
    f0, f1, _ = synth.planted_pair(1000)
    out = handle.estimate(dev(f0), dev(f1), 16, 16)
    torch.cuda.synchronize()
    ref_field, _ = oracle.me_full(f0, f1, 16, 16, even=True)
    assert_fields_equal(out, ref_field)


@pytest.mark.parametrize("rng_px", [0, 8, 16, 24, 32])
def test_full16_ranges_random(handle, rng_px):
    rng = np.random.default_rng(rng_px)
    H, W = 96, 160
    f0 = rng.integers(0, 4096, (H, W)).astype(np.uint16)
    f1 = rng.integers(0, 4096, (H, W)).astype(np.uint16)
    out = handle.estimate(dev(f0), dev(f1), 16, rng_px)
    ref_field, _ = oracle.me_full(f0, f1, 16, rng_px, even=True)
    assert_fields_equal(out, ref_field)


@pytest.mark.parametrize("kind", ["flat", "saturated", "zero", "checker", "identical"])
def test_full16_adversarial(handle, kind):
    H, W = 80, 128
    rng = np.random.default_rng(9)
    if kind == "flat":
        f0 = np.full((H, W), 2000, np.uint16)
        f1 = f0.copy()
    elif kind == "saturated":
        f0 = np.full((H, W), 4095, np.uint16)
        f1 = np.where(rng.random((H, W)) < 0.5, 4095, 0).astype(np.uint16)
    elif kind == "zero":
        f0 = np.zeros((H, W), np.uint16)
        f1 = np.full((H, W), 4095, np.uint16)
    elif kind == "checker":
        yy, xx = np.mgrid[0:H, 0:W]
        f0 = np.where((xx // 2 + yy // 2) % 2 == 0, 4095, 0).astype(np.uint16)
        f1 = np.roll(f0, 2, axis=1)
    else:
        f0 = synth.round_clip(synth.blob_texture_scene(rng, H, W))
        f1 = f0.copy()
    out = handle.estimate(dev(f0), dev(f1), 16, 32)
    ref_field, _ = oracle.me_full(f0, f1, 16, 32, even=True)
    assert_fields_equal(out, ref_field)


@pytest.mark.parametrize("shape", [(16, 16), (34, 50), (136, 200), (72, 1000)])
@pytest.mark.parametrize("block", [8, 16, 32])
def test_full_ragged_and_blocks(handle, shape, block):
    """Partial edge blocks and non-16 blocks take the generic kernel; a frame
    smaller than one block is rejected (W, H >= block is the contract)."""
    H, W = shape
    if W < block or H < block:
        f = dev(np.zeros((H, W), np.uint16))
        with pytest.raises(bm.BayerError):
            handle.estimate(f, f, block, 12)
        return
    f0, f1 = synth.pan_clip(5, H, W, n_frames=2, rect_size=(8, 24))
    out = handle.estimate(dev(f0), dev(f1), block, 12)
    ref_field, _ = oracle.me_full(f0, f1, block, 12, even=True)
    assert_fields_equal(out, ref_field)


@pytest.mark.parametrize("block,rng_px", [(16, 9), (8, 6), (64, 5)])
def test_full_raw_phase(handle, block, rng_px):
    H, W = 128, 192
    f0, f1 = synth.pan_clip(6, H, W, n_frames=2, rect_size=(8, 40))
    out = handle.estimate_ex(dev(f0), dev(f1), mode=bm.MODE_FULL, phase=bm.PHASE_RAW, block=block,
                             search_range=rng_px)
    ref_field, _ = oracle.me_full(f0, f1, block, rng_px, even=False)
    assert_fields_equal(out[0], ref_field)


def test_full_1080p_clip_batched(handle):
    """The 1080p workload as the benchmark launches it: 8 frames, 7 pairs in
    one launch, block 16, +-32 EVEN; every block of every pair vs the oracle."""
    wl = synth.WORKLOADS["1080p"]
    frames = synth.pan_clip(wl["seed"], wl["H"], wl["W"], n_frames=wl["frames"])
    H, W = wl["H"], wl["W"]
    d = dev(frames)
    out = handle.estimate_ex(d, d[1:], batch=7, ref_batch_stride=H * W, cur_batch_stride=H * W,
                             search_range=32)
    torch.cuda.synchronize()
    for t in range(7):
        ref_field, _ = oracle.me_full(frames[t], frames[t + 1], 16, 32, even=True)
        assert_fields_equal(out[t], ref_field)


def test_full_4k_pair_sampled(handle):
    """4K (3840x2160), block 16, +-32: one pair, all 32400 blocks."""
    frames = synth.pan_clip(1002, 2160, 3840, n_frames=2)
    out = handle.estimate(dev(frames[0]), dev(frames[1]), 16, 32)
    ref_field, _ = oracle.me_full(frames[0], frames[1], 16, 32, even=True)
    assert_fields_equal(out, ref_field)


# ----------------------------------------------------------------------------
# coarse-to-fine pyramid and learned-seeded refine
# ----------------------------------------------------------------------------

@pytest.mark.parametrize("even", [False, True])
@pytest.mark.parametrize("shape", [(256, 320), (720, 960)])
def test_c2f_standard(handle, even, shape):
    H, W = shape
    f0, f1 = synth.pan_clip(40, H, W, n_frames=2)
    out = handle.estimate_ex(dev(f0), dev(f1), mode=bm.MODE_C2F,
                             phase=bm.PHASE_EVEN if even else bm.PHASE_RAW)
    ref_field, _ = oracle.me_c2f(f0, f1, even=even)
    assert_fields_equal(out[0], ref_field)


@pytest.mark.parametrize("mode", ["mode1", "mode2", "mode4"])
def test_c2f_settings(handle, mode):
    import json, os
    tab = json.load(open(os.path.join(os.path.dirname(__file__), "golden", "fme_settings_gflops.json")))
    m = tab["modes"][mode]
    f0, f1 = synth.pan_clip(41, 256, 384, n_frames=2)
    setting = bm.C2FSetting(tuple(m["levels"]), tuple(tuple(s) for s in m["stages"]))
    out = handle.estimate_ex(dev(f0), dev(f1), mode=bm.MODE_C2F, phase=bm.PHASE_RAW, c2f=setting)
    ref_field, _ = oracle.me_c2f(f0, f1, levels=m["levels"], stages=[tuple(s) for s in m["stages"]], even=False)
    assert_fields_equal(out[0], ref_field)


def test_seeded_refine(handle):
    frames = synth.pan_clip(50, 272, 480, n_frames=2)
    h, w = 17, 30
    pdx, pdy, conf = synth.proposals(3, h, w, 32)
    prop = np.stack([pdx, pdy], axis=-1).astype(np.float32)
    fb = torch.empty((1, h, w), dtype=torch.uint8, device="cuda")
    out = handle.estimate_ex(dev(frames[0]), dev(frames[1]), mode=bm.MODE_SEEDED, block=16, search_range=32,
                             prop_dxdy=dev(prop), conf=dev(conf), fallback=fb)
    ref_field, ref_fb, _ = oracle.me_seeded(frames[0], frames[1], 16, 32, pdx, pdy, conf)
    assert_fields_equal(out[0], ref_field)
    np.testing.assert_array_equal(fb[0].cpu().numpy(), ref_fb)


# ----------------------------------------------------------------------------
# propagation
# ----------------------------------------------------------------------------

def _mv_field(seed, h, w, B, H, W, mag=32):
    rng = np.random.default_rng(seed)
    mv = np.zeros((h, w), oracle.MV_DTYPE)
    for i in range(h):
        for j in range(w):
            lo_x, hi_x = max(-mag, -j * B), min(mag, W - B - j * B)
            lo_y, hi_y = max(-mag, -i * B), min(mag, H - B - i * B)
            mv[i, j] = (2 * rng.integers(-(-lo_x // 2), hi_x // 2 + 1), 2 * rng.integers(-(-lo_y // 2), hi_y // 2 + 1), 0)
    return mv


def _records(mv):
    return dev(np.ascontiguousarray(mv).view(np.int32).reshape(mv.shape + (2,)))


@pytest.mark.parametrize("C,Hf,Wf,stride", [(64, 64, 64, 4), (256, 136, 240, 8), (7, 20, 36, 2), (3, 9, 13, 4),
                                          (6, 11, 7, 8), (5, 8, 12, 16), (12, 9, 13, 4), (8, 11, 7, 8)])
@pytest.mark.parametrize("interp", [bm.INTERP_NEAREST, bm.INTERP_BILINEAR])
@pytest.mark.parametrize("layout", [bm.LAYOUT_NCHW, bm.LAYOUT_NHWC])
def test_propagate(handle, C, Hf, Wf, stride, interp, layout):
    B = 16
    H, W = Hf * stride, Wf * stride
    h, w = -(-H // B), -(-W // B)
    mv = _mv_field(C + Hf, h, w, B, H, W)
    feat = synth.features(C, C, Hf, Wf, layout="NCHW" if layout == bm.LAYOUT_NCHW else "NHWC")[0]
    out = handle.feat_propagate(dev(feat), _records(mv), B, stride, interp=interp, layout=layout)
    g = out[0].cpu().numpy()
    expect = oracle.propagate(feat, mv, B, stride, interp=interp, layout=layout)
    np.testing.assert_array_equal(g.view(np.uint32), expect.view(np.uint32))
    if interp == bm.INTERP_BILINEAR:
        e64 = oracle.propagate_bilinear_f64(feat, mv, B, stride, layout=layout)
        scale = oracle.propagate_bilinear_f64(np.abs(feat), mv, B, stride, layout=layout)
        assert (np.abs(g - e64) <= 1e-5 * np.maximum(scale, 1e-30)).all()


def test_propagate_batched_1080p(handle):
    """Seven 256 x 136 x 240 maps in one launch, each with its own MV field."""
    B, s, C, Hf, Wf = 16, 8, 256, 136, 240
    mvs = np.stack([_mv_field(100 + t, 68, 120, B, 1088, 1920) for t in range(7)])
    feats = synth.features(1001, C, Hf, Wf, n=7)
    out = handle.feat_propagate(dev(feats), _records(mvs), B, s)
    g = out.cpu().numpy()
    for t in range(7):
        expect = oracle.propagate(feats[t], mvs[t], B, s, interp=bm.INTERP_BILINEAR)
        np.testing.assert_array_equal(g[t].view(np.uint32), expect.view(np.uint32))


@pytest.mark.parametrize("layout", [bm.LAYOUT_NHWC, bm.LAYOUT_NCHW])
def test_propagate_4k_full(handle, layout):
    """The 4K precision form's propagation: one 128 x 540 x 960 float32 map at
    stride 4 (3840 x 2160 frame, 240 x 135 blocks), bilinear, every output bit
    for bit against the oracle."""
    B, s, C, Hf, Wf = 16, 4, 128, 540, 960
    mv = _mv_field(2002, 135, 240, B, 2160, 3840)
    feat = synth.features(2003, C, Hf, Wf, layout="NCHW" if layout == bm.LAYOUT_NCHW else "NHWC")[0]
    out = handle.feat_propagate(dev(feat), _records(mv), B, s, interp=bm.INTERP_BILINEAR, layout=layout)
    g = out[0].cpu().numpy()
    expect = oracle.propagate(feat, mv, B, s, interp=bm.INTERP_BILINEAR, layout=layout)
    np.testing.assert_array_equal(g.view(np.uint32), expect.view(np.uint32))


# ----------------------------------------------------------------------------
# end-to-end host path, argument errors, probe
# ----------------------------------------------------------------------------

@pytest.mark.parametrize("H", [272, 264])
def test_clip_process_host(handle, H):
    """The host-buffer path; 264 rows clip the last block row to 8 (33-row maps)."""
    frames = synth.pan_clip(60, H, 480, n_frames=4)
    feats = synth.features(61, 32, -(-H // 8), 60, n=3)
    mv, fo = handle.clip_process_host(frames, feats, block=16, search_range=32, stride=8)
    for t in range(3):
        ref_field, _ = oracle.me_full(frames[t], frames[t + 1], 16, 32, even=True)
        for k in ("dx", "dy", "sad"):
            np.testing.assert_array_equal(mv[t][k], ref_field[k])
        expect = oracle.propagate(feats[t], ref_field, 16, 8, interp=bm.INTERP_BILINEAR)
        np.testing.assert_array_equal(fo[t].view(np.uint32), expect.view(np.uint32))


def test_invalid_arguments_return_status(handle):
    f = torch.zeros((64, 64), dtype=torch.int16, device="cuda")
    with pytest.raises(bm.BayerError) as e:
        handle.estimate(f, f, 16, 7)  # odd range
    assert e.value.status == bm.ERR_INVALID_ARG
    with pytest.raises(bm.BayerError):
        handle.estimate(f, f, 12, 8)  # block not in {8,16,32,64}
    g = torch.zeros((63, 64), dtype=torch.int16, device="cuda")
    with pytest.raises(bm.BayerError):
        handle.estimate(g, g, 16, 8)  # odd height
    feat = torch.zeros((1, 4, 16, 16), device="cuda")
    mv = torch.zeros((1, 3, 4, 2), dtype=torch.int32, device="cuda")
    with pytest.raises(bm.BayerError):
        handle.feat_propagate(feat, mv, 16, 4)  # mv field 3x4 != 4x4
    with pytest.raises(bm.BayerError):
        handle.feat_propagate(feat, torch.zeros((1, 4, 4, 2), dtype=torch.int32, device="cuda"), 16, 4, out=feat)
    assert handle.sync_status() == bm.OK


def test_probe_alu(handle):
    pc, mhz, nsm = handle.probe_alu(0)
    assert 20 < pc < 140 and 500 < mhz < 2500 and nsm > 0


@pytest.mark.parametrize("block,rng_px,phase", [(8, 32, bm.PHASE_EVEN), (32, 32, bm.PHASE_EVEN),
                                                (64, 32, bm.PHASE_EVEN), (16, 32, bm.PHASE_RAW),
                                                (64, 12, bm.PHASE_RAW)])
def test_full_search_as_one_level(handle, block, rng_px, phase):
    """Exhaustive searches the 16-pixel strip kernel does not take run as a
    one-stage pyramid level on the packed C2F kernel (RAW: both column parities)."""
    H, W = 256, 384
    frames = synth.pan_clip(45, H, W, n_frames=3)
    d = dev(frames)
    out = handle.estimate_ex(d, d[1:], mode=bm.MODE_FULL, phase=phase, block=block, search_range=rng_px, batch=2,
                             ref_batch_stride=H * W, cur_batch_stride=H * W)
    for t in range(2):
        ref_field, _ = oracle.me_full(frames[t], frames[t + 1], block, rng_px, even=phase == bm.PHASE_EVEN)
        assert_fields_equal(out[t], ref_field)
