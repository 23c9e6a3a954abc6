"""The paper's coarse-to-fine presets in the EVEN and RAW phases on the GPU vs
the oracle, bit for bit: levels of whole 8- to 64-pixel blocks run the packed
C2F kernel (me_c2f.cu); levels without a whole-block grid or a shared start
centre, and unaligned frames, the generic one."""
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


def check(got, want):
    g = bm.records_to_numpy(got)
    for k in ("dx", "dy", "sad"):
        np.testing.assert_array_equal(g[k], want[k])


@pytest.mark.parametrize("mode", ["standard", "mode1", "mode2", "mode3", "mode4"])
def test_presets_even_batched(handle, mode):
    H, W = 512, 768
    frames = synth.pan_clip(60, H, W, n_frames=3, rect_size=(16, 96))
    d = torch.from_numpy(frames).cuda()
    setting = bm.C2F_PRESETS[mode]
    out = handle.estimate_ex(d, d[1:], mode=bm.MODE_C2F, phase=bm.PHASE_EVEN, c2f=setting, batch=2,
                             ref_batch_stride=H * W, cur_batch_stride=H * W)
    torch.cuda.synchronize()
    for t in range(2):
        want, _ = oracle.me_c2f(frames[t], frames[t + 1], levels=list(setting.levels),
                                stages=[tuple(s) for s in setting.stages], even=True)
        check(out[t], want)


def test_standard_1080p_clip(handle):
    """Two pairs of the benchmark's 1080p clip with the standard pyramid."""
    wl = synth.WORKLOADS["1080p"]
    H, W = wl["H"], wl["W"]
    frames = synth.pan_clip(wl["seed"], H, W, n_frames=3)
    d = torch.from_numpy(frames).cuda()
    out = handle.estimate_ex(d, d[1:], mode=bm.MODE_C2F, phase=bm.PHASE_EVEN, batch=2, ref_batch_stride=H * W,
                             cur_batch_stride=H * W)
    torch.cuda.synchronize()
    for t in range(2):
        want, _ = oracle.me_c2f(frames[t], frames[t + 1], even=True)
        check(out[t], want)


def test_large_motion_near_borders(handle):
    """Fast global motion: the pyramid's windows reach past every frame edge."""
    H, W = 256, 384
    rng = np.random.default_rng(61)
    base = synth.round_clip(synth.blob_texture_scene(rng, H + 128, W + 128))
    f0 = np.ascontiguousarray(base[64:64 + H, 64:64 + W])
    f1 = np.ascontiguousarray(base[64 - 38:64 - 38 + H, 64 + 52:64 + 52 + W])
    out = handle.estimate_ex(torch.from_numpy(f0).cuda(), torch.from_numpy(f1).cuda(), mode=bm.MODE_C2F,
                             phase=bm.PHASE_EVEN)
    torch.cuda.synchronize()
    want, _ = oracle.me_c2f(f0, f1, even=True)
    check(out[0], want)


def test_odd_pitch_takes_the_generic_kernel(handle):
    H, W, pitch = 256, 320, 321
    f0, f1 = synth.pan_clip(62, H, W, n_frames=2)
    buf = np.zeros((2, H, pitch), np.uint16)
    buf[0, :, :W], buf[1, :, :W] = f0, f1
    d = torch.from_numpy(buf).cuda()
    out = handle.estimate_ex(d[0], d[1], mode=bm.MODE_C2F, phase=bm.PHASE_EVEN, W=W, H=H, pitch=pitch)
    torch.cuda.synchronize()
    want, _ = oracle.me_c2f(f0, f1, even=True)
    check(out[0], want)


@pytest.mark.parametrize("mode", ["standard", "mode3"])
def test_partial_tiles_and_mixed_levels(handle, mode):
    """480 x 800: 15 x 25 blocks of 32 (partial 2 x 2 tiles at the right and
    bottom); 480 is no multiple of 64, so the standard pyramid's first level
    takes the generic kernel and its second the packed one."""
    H, W = 480, 800
    f0, f1 = synth.pan_clip(63, H, W, n_frames=2, rect_size=(16, 96))
    setting = bm.C2F_PRESETS[mode]
    out = handle.estimate_ex(torch.from_numpy(f0).cuda(), torch.from_numpy(f1).cuda(), mode=bm.MODE_C2F,
                             phase=bm.PHASE_EVEN, c2f=setting)
    torch.cuda.synchronize()
    want, _ = oracle.me_c2f(f0, f1, levels=list(setting.levels), stages=[tuple(s) for s in setting.stages], even=True)
    check(out[0], want)


def test_mode4_partial_small_tiles(handle):
    """496 x 816: 31 x 51 blocks of 16 (partial 2 x 2 tiles of the small-block
    path) and 62 x 102 of 8; no whole 32- or 64-pixel grid, so the two coarse
    levels run the generic kernel and hand it their MVs as start centres."""
    H, W = 496, 816
    f0, f1 = synth.pan_clip(64, H, W, n_frames=2, rect_size=(8, 48))
    setting = bm.C2F_PRESETS["mode4"]
    out = handle.estimate_ex(torch.from_numpy(f0).cuda(), torch.from_numpy(f1).cuda(), mode=bm.MODE_C2F,
                             phase=bm.PHASE_EVEN, c2f=setting)
    torch.cuda.synchronize()
    want, _ = oracle.me_c2f(f0, f1, levels=list(setting.levels), stages=[tuple(s) for s in setting.stages], even=True)
    check(out[0], want)


@pytest.mark.parametrize("levels,stages", [((16, 8), ((4, 4), (2, 1))), ((8,), ((8, 8), (4, 4), (2, 1))),
                                           ((16,), ((2, 8), (2, 4), (2, 2)))])
def test_small_block_levels(handle, levels, stages):
    """Pyramids that start at a 16- or 8-pixel level (common start centre 0)."""
    H, W = 256, 384
    frames = synth.pan_clip(65, H, W, n_frames=3, rect_size=(8, 48))
    d = torch.from_numpy(frames).cuda()
    setting = bm.C2FSetting(levels, stages)
    out = handle.estimate_ex(d, d[1:], mode=bm.MODE_C2F, phase=bm.PHASE_EVEN, c2f=setting, batch=2,
                             ref_batch_stride=H * W, cur_batch_stride=H * W)
    torch.cuda.synchronize()
    for t in range(2):
        want, _ = oracle.me_c2f(frames[t], frames[t + 1], levels=list(levels), stages=[tuple(s) for s in stages],
                                even=True)
        check(out[t], want)


def test_mode4_1080p_pair(handle):
    """One pair of the benchmark's 1080p clip through all four mode-4 levels."""
    wl = synth.WORKLOADS["1080p"]
    H, W = wl["H"], wl["W"]
    f0, f1 = synth.pan_clip(wl["seed"], H, W, n_frames=2)
    setting = bm.C2F_PRESETS["mode4"]
    out = handle.estimate_ex(torch.from_numpy(f0).cuda(), torch.from_numpy(f1).cuda(), mode=bm.MODE_C2F,
                             phase=bm.PHASE_EVEN, c2f=setting)
    torch.cuda.synchronize()
    want, _ = oracle.me_c2f(f0, f1, levels=list(setting.levels), stages=[tuple(s) for s in setting.stages], even=True)
    check(out[0], want)


@pytest.mark.parametrize("levels", [(64, 32, 32), (16, 16)])
def test_children_without_a_shared_centre(handle, levels):
    """A repeated level: each block's parent is the same-sized block, so a 2 x 2
    tile would mix start centres; the second 32-pixel level takes one block per
    CTA and the second 16-pixel level the generic kernel."""
    H, W = 288, 384
    f0, f1 = synth.pan_clip(66, H, W, n_frames=2, rect_size=(8, 48))
    stages = ((4, 8), (2, 4), (2, 1))
    out = handle.estimate_ex(torch.from_numpy(f0).cuda(), torch.from_numpy(f1).cuda(), mode=bm.MODE_C2F,
                             phase=bm.PHASE_EVEN, c2f=bm.C2FSetting(levels, stages))
    torch.cuda.synchronize()
    want, _ = oracle.me_c2f(f0, f1, levels=list(levels), stages=list(stages), even=True)
    check(out[0], want)


@pytest.mark.parametrize("mode", ["standard", "mode1", "mode2", "mode3", "mode4"])
def test_presets_raw_batched(handle, mode):
    """RAW phase: steps 8 and 4, then step 1 (both column parities), and start
    centres of either parity below the first level."""
    H, W = 512, 768
    frames = synth.pan_clip(67, H, W, n_frames=3, rect_size=(16, 96))
    d = torch.from_numpy(frames).cuda()
    setting = bm.C2F_PRESETS[mode]
    out = handle.estimate_ex(d, d[1:], mode=bm.MODE_C2F, phase=bm.PHASE_RAW, c2f=setting, batch=2,
                             ref_batch_stride=H * W, cur_batch_stride=H * W)
    torch.cuda.synchronize()
    for t in range(2):
        want, _ = oracle.me_c2f(frames[t], frames[t + 1], levels=list(setting.levels),
                                stages=[tuple(s) for s in setting.stages], even=False)
        check(out[t], want)


def test_raw_large_motion_near_borders(handle):
    """Odd global motion in RAW: the odd-parity windows reach past every frame edge."""
    H, W = 256, 384
    rng = np.random.default_rng(68)
    base = synth.round_clip(synth.blob_texture_scene(rng, H + 128, W + 128))
    f0 = np.ascontiguousarray(base[64:64 + H, 64:64 + W])
    f1 = np.ascontiguousarray(base[64 - 37:64 - 37 + H, 64 + 51:64 + 51 + W])
    out = handle.estimate_ex(torch.from_numpy(f0).cuda(), torch.from_numpy(f1).cuda(), mode=bm.MODE_C2F,
                             phase=bm.PHASE_RAW)
    torch.cuda.synchronize()
    want, _ = oracle.me_c2f(f0, f1, even=False)
    check(out[0], want)


def test_raw_standard_1080p_pair(handle):
    wl = synth.WORKLOADS["1080p"]
    H, W = wl["H"], wl["W"]
    f0, f1 = synth.pan_clip(wl["seed"], H, W, n_frames=2)
    out = handle.estimate_ex(torch.from_numpy(f0).cuda(), torch.from_numpy(f1).cuda(), mode=bm.MODE_C2F,
                             phase=bm.PHASE_RAW)
    torch.cuda.synchronize()
    want, _ = oracle.me_c2f(f0, f1, even=False)
    check(out[0], want)


def test_raw_mode4_partial_small_tiles(handle):
    """RAW mode 4 at 496 x 816: partial 2 x 2 tiles at the 16-pixel level, odd
    start centres from every RAW parent level, step-1 windows at both parities."""
    H, W = 496, 816
    f0, f1 = synth.pan_clip(69, H, W, n_frames=2, rect_size=(8, 48))
    setting = bm.C2F_PRESETS["mode4"]
    out = handle.estimate_ex(torch.from_numpy(f0).cuda(), torch.from_numpy(f1).cuda(), mode=bm.MODE_C2F,
                             phase=bm.PHASE_RAW, c2f=setting)
    torch.cuda.synchronize()
    want, _ = oracle.me_c2f(f0, f1, levels=list(setting.levels), stages=[tuple(s) for s in setting.stages],
                            even=False)
    check(out[0], want)


@pytest.mark.parametrize("block,rng_px,even", [(8, 13, False), (32, 14, True), (64, 7, False), (16, 10, True)])
def test_full_search_other_ranges(handle, block, rng_px, even):
    """Exhaustive searches through the one-stage level path: odd RAW ranges, and
    EVEN ranges the 16-pixel strip kernel does not take (R = range / 2 steps)."""
    H, W = 192, 320
    f0, f1 = synth.pan_clip(70, H, W, n_frames=2)
    out = handle.estimate_ex(torch.from_numpy(f0).cuda(), torch.from_numpy(f1).cuda(), mode=bm.MODE_FULL,
                             phase=bm.PHASE_EVEN if even else bm.PHASE_RAW, block=block, search_range=rng_px)
    torch.cuda.synchronize()
    want, _ = oracle.me_full(f0, f1, block, rng_px, even=even)
    check(out[0], want)
