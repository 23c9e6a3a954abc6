"""Frames whose height is not a multiple of the block size, on the fast kernels.

The last block row of such a frame is clipped to the rows inside the frame
(its SAD covers those rows; a candidate is valid when the clipped block stays
inside the frame).  The exhaustive 16-pixel strip kernel and the packed
coarse-to-fine level kernel serve it directly -- the real 1920 x 1080 frame,
the paper's 720 x 960 runtime resolution at its [64, 32] pyramid, 4K at block
32 and 64 -- and every MV field must equal the oracle's bit for bit.  Widths
that are not a multiple of the block still take the generic kernel (tested in
test_gpu_parity.py).
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


def check(got, want):
    g = bm.records_to_numpy(got).reshape(want.shape)
    for k in ("dx", "dy", "sad"):
        bad = np.argwhere(g[k] != want[k])
        assert bad.size == 0, f"{k} differs at {bad[:5].tolist()} of {want.shape}"


@pytest.mark.parametrize("H,W", [(18, 64), (40, 256), (100, 320), (250, 448)])
@pytest.mark.parametrize("rng_px", [8, 16, 24, 32])
def test_full16_clipped_last_row(handle, H, W, rng_px):
    """Block 16 EVEN on the strip kernel: the last block row keeps H % 16 rows."""
    frames = synth.pan_clip(300 + H, H, W, n_frames=3, rect_size=(8, 32))
    d = dev(frames)
    out = handle.estimate_ex(d, d[1:], search_range=rng_px, batch=2, ref_batch_stride=H * W,
                             cur_batch_stride=H * W)
    for t in range(2):
        want, _ = oracle.me_full(frames[t], frames[t + 1], 16, rng_px, even=True)
        check(out[t], want)


@pytest.mark.parametrize("kind", ["flat", "saturated", "checker"])
def test_full16_clipped_adversarial(handle, kind):
    H, W = 58, 192
    if kind == "flat":
        f0 = np.full((H, W), 1234, np.uint16)
        f1 = f0.copy()
    elif kind == "saturated":
        f0 = np.full((H, W), 4095, np.uint16)
        f1 = np.zeros((H, W), np.uint16)
    else:
        y, x = np.mgrid[0:H, 0:W]
        f0 = np.where(((y // 2) + (x // 2)) % 2 == 0, 4095, 0).astype(np.uint16)
        f1 = np.roll(f0, 2, axis=1)
    out = handle.estimate(dev(f0), dev(f1), 16, 16)
    want, _ = oracle.me_full(f0, f1, 16, 16, even=True)
    check(out, want)


def test_full16_1920x1080_pairs(handle):
    """A real 1080-row frame (68 block rows, the last 8 rows high), block 16,
    +-32, 7 pairs in one launch as the benchmark's 1088-row workload runs."""
    H, W = 1080, 1920
    frames = synth.pan_clip(1001, H, W, n_frames=8)
    d = dev(frames)
    out = handle.estimate_ex(d, d[1:], search_range=32, batch=7, ref_batch_stride=H * W, cur_batch_stride=H * W)
    torch.cuda.synchronize()
    for t in range(7):
        want, _ = oracle.me_full(frames[t], frames[t + 1], 16, 32, even=True)
        check(out[t], want)


@pytest.mark.parametrize("even", [True, False])
@pytest.mark.parametrize("H,W", [(100, 256), (200, 384), (720, 960)])
@pytest.mark.parametrize("mode", ["standard", "mode4"])
def test_c2f_clipped_rows(handle, even, H, W, mode):
    """The paper's pyramids where the frame height clips the last block row of
    the 64- and 32-pixel levels (and of the 16- and 8-pixel ones at 100 rows);
    two pairs in one call."""
    s = bm.C2F_PRESETS[mode]
    frames = synth.pan_clip(400 + H, H, W, n_frames=3, rect_size=(8, 48))
    d = dev(frames)
    out = handle.estimate_ex(d, d[1:], mode=bm.MODE_C2F, phase=bm.PHASE_EVEN if even else bm.PHASE_RAW, c2f=s,
                             batch=2, ref_batch_stride=H * W, cur_batch_stride=H * W)
    for t in range(2):
        want, _ = oracle.me_c2f(frames[t], frames[t + 1], s.levels, s.stages, even=even)
        check(out[t], want)


@pytest.mark.parametrize("levels", [(64, 32, 32), (32, 16), (16, 16)])
def test_c2f_clipped_rows_unshared_centres(handle, levels):
    """Levels whose children do not share a start centre (one block per CTA,
    or the generic kernel) on a clipped height."""
    H, W = 150, 256
    f0, f1 = synth.pan_clip(410, H, W, n_frames=2, rect_size=(8, 48))
    s = bm.C2FSetting(levels, ((4, 4), (2, 2), (1, 2)))
    out = handle.estimate_ex(dev(f0), dev(f1), mode=bm.MODE_C2F, c2f=s)
    want, _ = oracle.me_c2f(f0, f1, levels, s.stages, even=True)
    check(out[0], want)


def test_c2f_standard_1920x1080(handle):
    H, W = 1080, 1920
    frames = synth.pan_clip(420, H, W, n_frames=3)
    d = dev(frames)
    out = handle.estimate_ex(d, d[1:], mode=bm.MODE_C2F, batch=2, ref_batch_stride=H * W, cur_batch_stride=H * W)
    for t in range(2):
        want, _ = oracle.me_c2f(frames[t], frames[t + 1], even=True)
        check(out[t], want)


def test_c2f_standard_4k(handle):
    """3840 x 2160: the 64-pixel level's last row keeps 48 rows, the 32-pixel
    level's 16."""
    H, W = 2160, 3840
    f0, f1 = synth.pan_clip(1002, H, W, n_frames=2)
    out = handle.estimate_ex(dev(f0), dev(f1), mode=bm.MODE_C2F)
    want, _ = oracle.me_c2f(f0, f1, even=True)
    check(out[0], want)


@pytest.mark.parametrize("block,rng_px,even", [(32, 32, True), (64, 24, True), (8, 12, False), (32, 10, False)])
def test_full_search_one_level_clipped(handle, block, rng_px, even):
    """Exhaustive searches off the strip kernel (one-stage pyramid level) on a
    clipped height."""
    H, W = 1080, 640
    f0, f1 = synth.pan_clip(430, H, W, n_frames=2)
    out = handle.estimate_ex(dev(f0), dev(f1), mode=bm.MODE_FULL, phase=bm.PHASE_EVEN if even else bm.PHASE_RAW,
                             block=block, search_range=rng_px)
    want, _ = oracle.me_full(f0, f1, block, rng_px, even=even)
    check(out[0], want)
