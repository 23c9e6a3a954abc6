"""Pins of the CPU oracle's motion estimation to facts outside the oracle.

Each test ties one part of the oracle to something it does not compute
itself: numbers the paper prints (FME-settings table, Table 8), closed forms
(SAD of a linear ramp), an independent brute force on tiny frames, planted
shifts, identical frames, and tie-break cases built to have equal costs.
"""
import json
import os

import numpy as np
import pytest

from paper_2508_05990_b300 import synth

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")


# --------------------------------------------------------------------------
# independent brute force (numpy + python, written from the definitions)
# --------------------------------------------------------------------------

def brute_force(ref, cur, B, rng_px, step, center=None):
    """All candidates center + (u*step, v*step) with |u|,|v| <= rng_px//step and
    |dx|,|dy| <= rng_px; invalid (out-of-frame) ones skipped; min of
    (sad, |dx|+|dy|, dy, dx).  Returns int64 array [h, w, 3] (dx, dy, sad)."""
    H, W = ref.shape
    h, w = -(-H // B), -(-W // B)
    R = rng_px // step
    out = np.zeros((h, w, 3), np.int64)
    r64 = ref.astype(np.int64)
    c64 = cur.astype(np.int64)
    for i in range(h):
        for j in range(w):
            y0, x0 = i * B, j * B
            bh, bw = min(B, H - y0), min(B, W - x0)
            cb = c64[y0:y0 + bh, x0:x0 + bw]
            cx, cy = (0, 0) if center is None else center[i][j]
            cands = []
            for v in range(-R, R + 1):
                for u in range(-R, R + 1):
                    dx, dy = cx + u * step, cy + v * step
                    if abs(dx) > rng_px or abs(dy) > rng_px:
                        continue
                    if x0 + dx < 0 or x0 + dx + bw > W or y0 + dy < 0 or y0 + dy + bh > H:
                        continue
                    sad = int(np.abs(cb - r64[y0 + dy:y0 + dy + bh, x0 + dx:x0 + dx + bw]).sum())
                    cands.append((sad, abs(dx) + abs(dy), dy, dx))
            best = min(cands)
            out[i, j] = (best[3], best[2], best[0])
    return out


def as_int(field):
    return np.stack([field["dx"].astype(np.int64), field["dy"].astype(np.int64),
                     field["sad"].astype(np.int64)], axis=-1)


def tiny_frames(kind, H, W, seed):
    rng = np.random.default_rng(seed)
    if kind == "random":
        return (rng.integers(0, 4096, (H, W)).astype(np.uint16),
                rng.integers(0, 4096, (H, W)).astype(np.uint16))
    if kind == "flat":
        return np.full((H, W), 1234, np.uint16), np.full((H, W), 1234, np.uint16)
    if kind == "saturated":
        a = np.full((H, W), 4095, np.uint16)
        b = a.copy()
        b[rng.random((H, W)) < 0.3] = 0
        return a, b
    if kind == "checker":
        yy, xx = np.mgrid[0:H, 0:W]
        a = np.where((xx + yy) % 2 == 0, 4095, 0).astype(np.uint16)
        b = np.where((xx // 3 + yy // 2) % 2 == 0, 4095, 0).astype(np.uint16)
        return a, b
    if kind == "scene":
        f0, f1, _ = synth.planted_pair(seed, H, W, block=8, max_shift=4)
        return f0, f1
    raise ValueError(kind)


@pytest.mark.parametrize("kind", ["random", "flat", "saturated", "checker", "scene"])
@pytest.mark.parametrize("shape,B", [((32, 32), 8), ((24, 40), 8), ((36, 28), 8), ((40, 48), 16)])
@pytest.mark.parametrize("even", [True, False])
def test_full_search_equals_brute_force(oracle_mod, kind, shape, B, even):
    ref, cur = tiny_frames(kind, *shape, seed=hash((kind, shape, B)) % 1000)
    rng_px = 6
    field, count = oracle_mod.me_full(ref, cur, B, rng_px, even=even)
    step = 2 if even else 1
    expect = brute_force(ref, cur, B, rng_px, step)
    np.testing.assert_array_equal(as_int(field), expect)
    # scheduled pixel-candidates: every enumerated candidate x block pixels
    H, W = shape
    R = rng_px // step
    assert count == (2 * R + 1) ** 2 * H * W


def test_stage_with_centre_equals_brute_force(oracle_mod):
    ref, cur = tiny_frames("scene", 48, 64, seed=7)
    B, H, W = 16, 48, 64
    h, w = 3, 4
    rng = np.random.default_rng(3)
    centre = np.zeros((h, w), oracle_mod.MV_DTYPE)
    c = [[None] * w for _ in range(h)]
    for i in range(h):
        for j in range(w):
            # a valid even centre: the displaced block stays in the frame
            dx = 2 * int(rng.integers(max(-4, -(j * B) // 2), min(4, (W - B - j * B) // 2) + 1))
            dy = 2 * int(rng.integers(max(-4, -(i * B) // 2), min(4, (H - B - i * B) // 2) + 1))
            centre[i, j] = (dx, dy, 0)
            c[i][j] = (dx, dy)
    field, _ = oracle_mod.me_stage(ref, cur, B, R=2, step=2, lim=10, center=centre)
    np.testing.assert_array_equal(as_int(field), brute_force_lim(ref, cur, B, 2, 2, 10, c))


def brute_force_lim(ref, cur, B, R, step, lim, centre):
    H, W = ref.shape
    h, w = -(-H // B), -(-W // B)
    out = np.zeros((h, w, 3), np.int64)
    for i in range(h):
        for j in range(w):
            y0, x0 = i * B, j * B
            bh, bw = min(B, H - y0), min(B, W - x0)
            cb = cur[y0:y0 + bh, x0:x0 + bw].astype(np.int64)
            best = None
            for v in range(-R, R + 1):
                for u in range(-R, R + 1):
                    dx, dy = centre[i][j][0] + u * step, centre[i][j][1] + v * step
                    if abs(dx) > lim or abs(dy) > lim:
                        continue
                    if x0 + dx < 0 or x0 + dx + bw > W or y0 + dy < 0 or y0 + dy + bh > H:
                        continue
                    sad = int(np.abs(cb - ref[y0 + dy:y0 + dy + bh, x0 + dx:x0 + dx + bw].astype(np.int64)).sum())
                    key = (sad, abs(dx) + abs(dy), dy, dx)
                    best = key if best is None or key < best else best
            out[i, j] = (best[3], best[2], best[0])
    return out


# --------------------------------------------------------------------------
# closed form: SAD of a linear ramp
# --------------------------------------------------------------------------

def ramp(H, W, a, b, c, tx=0, ty=0):
    yy, xx = np.mgrid[0:H, 0:W]
    return (a * (xx + tx) + b * (yy + ty) + c).astype(np.uint16)


@pytest.mark.parametrize("B", [8, 16])
def test_ramp_sad_closed_form(oracle_mod, B):
    """ref = a*x + b*y + c, cur(x, y) = ref(x + tx, y + ty) analytically, so
    SAD(dx, dy) = B^2 * |a (tx - dx) + b (ty - dy)| for every valid candidate."""
    H, W, a, b, c = 64, 64, 1, 37, 400
    tx, ty = 6, -4
    ref = ramp(H, W, a, b, c)
    cur = ramp(H, W, a, b, c, tx, ty)
    h, w = H // B, W // B
    rng = np.random.default_rng(11)
    for _ in range(5):
        centre = np.zeros((h, w), oracle_mod.MV_DTYPE)
        for i in range(h):
            for j in range(w):
                dx = int(rng.integers(-j * B, (w - 1 - j) * B + 1))
                dy = int(rng.integers(-i * B, (h - 1 - i) * B + 1))
                centre[i, j] = (dx, dy, 0)
        field, _ = oracle_mod.me_stage(ref, cur, B, R=0, step=1, center=centre)
        expect = B * B * np.abs(a * (tx - centre["dx"].astype(np.int64)) + b * (ty - centre["dy"].astype(np.int64)))
        np.testing.assert_array_equal(field["sad"].astype(np.int64), expect)
        np.testing.assert_array_equal(field["dx"], centre["dx"])
    # full search finds the shift with zero cost wherever it is a valid candidate
    field, _ = oracle_mod.me_full(ref, cur, B, 8, even=True)
    for i in range(h):
        for j in range(w):
            if 0 <= j * B + tx <= W - B and 0 <= i * B + ty <= H - B:
                assert (field["dx"][i, j], field["dy"][i, j], field["sad"][i, j]) == (tx, ty, 0)


# --------------------------------------------------------------------------
# planted shifts, identical frames, tie-break
# --------------------------------------------------------------------------

@pytest.mark.parametrize("noise", [0.0, 2.0])
def test_planted_shifts_recovered(oracle_mod, noise):
    """Planted per-block shifts are recovered exactly wherever the true source
    block lies inside the frame and is not flat (blob sums clipped at 4095 make
    flat blocks whose candidates tie at zero cost; there the cost is still 0)."""
    f0, f1, mv = synth.planted_pair(1000, 256, 256, block=16, max_shift=8, noise_sigma=noise)
    field, _ = oracle_mod.me_full(f0, f1, 16, 16, even=True)
    ok = total = 0
    for i in range(16):
        for j in range(16):
            dx, dy = int(mv[i, j, 0]), int(mv[i, j, 1])
            if 0 <= j * 16 + dx <= 240 and 0 <= i * 16 + dy <= 240:
                src = f0[i * 16 + dy:i * 16 + dy + 16, j * 16 + dx:j * 16 + dx + 16]
                if noise == 0.0:
                    assert field["sad"][i, j] == 0
                if np.ptp(src) == 0:
                    continue
                total += 1
                ok += (field["dx"][i, j] == dx) and (field["dy"][i, j] == dy)
    assert total > 150
    if noise == 0.0:
        assert ok == total
    else:
        assert ok >= 0.999 * total


@pytest.mark.parametrize("even", [True, False])
def test_identical_frames_zero_motion(oracle_mod, even):
    f = synth.round_clip(synth.blob_texture_scene(np.random.default_rng(5), 96, 80))
    field, _ = oracle_mod.me_full(f, f, 16, 16, even=even)
    assert (field["dx"] == 0).all() and (field["dy"] == 0).all() and (field["sad"] == 0).all()


def test_tie_break_flat(oracle_mod):
    f = np.full((64, 64), 777, np.uint16)
    field, _ = oracle_mod.me_full(f, f.copy(), 16, 16, even=False)
    assert (field["dx"] == 0).all() and (field["dy"] == 0).all()


def test_tie_break_periodic(oracle_mod):
    """A texture of period 8 in x and y, shifted by (4, 4): the zero-cost
    candidates within +-6 are (+-4, +-4), all with |dx|+|dy| = 8, so the
    smaller dy and then the smaller dx win: (-4, -4).  With period 8 in x only
    (rows random) the zero-cost candidates are (+-4, 0): (-4, 0) wins on dx."""
    rng = np.random.default_rng(2)
    tile = rng.integers(0, 4096, (8, 8)).astype(np.uint16)
    ref = np.tile(tile, (8, 8))
    cur = np.roll(np.roll(ref, -4, axis=0), -4, axis=1)
    field, _ = oracle_mod.me_full(ref, cur, 8, 6, even=True)
    inner = (slice(1, -1), slice(1, -1))
    assert (field["dx"][inner] == -4).all() and (field["dy"][inner] == -4).all()
    assert (field["sad"][inner] == 0).all()
    row = rng.integers(0, 4096, (64, 1)).astype(np.uint16)
    ref2 = (np.tile(tile[0:1, :], (64, 8)).astype(np.int64) + row).clip(0, 4095).astype(np.uint16)
    cur2 = np.roll(ref2, -4, axis=1)
    field2, _ = oracle_mod.me_full(ref2, cur2, 8, 6, even=False)
    assert (field2["dx"][inner] == -4).all() and (field2["dy"][inner] == 0).all()


def test_min_cost_invariant_sampled(oracle_mod):
    """The chosen SAD is no greater than the SAD of any valid candidate."""
    frames = synth.pan_clip(21, 96, 128, n_frames=2, rect_size=(16, 48))
    ref, cur = frames[0], frames[1]
    B, rng_px = 16, 16
    field, _ = oracle_mod.me_full(ref, cur, B, rng_px, even=True)
    r64, c64 = ref.astype(np.int64), cur.astype(np.int64)
    for i in range(6):
        for j in range(8):
            y0, x0 = i * B, j * B
            cb = c64[y0:y0 + B, x0:x0 + B]
            s = int(field["sad"][i, j])
            for dy in range(-rng_px, rng_px + 1, 2):
                for dx in range(-rng_px, rng_px + 1, 2):
                    if 0 <= x0 + dx <= 128 - B and 0 <= y0 + dy <= 96 - B:
                        assert s <= int(np.abs(cb - r64[y0 + dy:y0 + dy + B, x0 + dx:x0 + dx + B]).sum())


# --------------------------------------------------------------------------
# coarse-to-fine: paper's printed cost figures (FME-settings table, Table 8)
# --------------------------------------------------------------------------

@pytest.fixture(scope="module")
def cityscapes_pair():
    rng = np.random.default_rng(4242)
    H, W = 1024, 2048
    a = rng.integers(0, 4096, (H, W)).astype(np.uint16)
    b = rng.integers(0, 4096, (H, W)).astype(np.uint16)
    return a, b


def test_fme_settings_gflops_pin(oracle_mod, cityscapes_pair):
    """The scheduled pixel-candidate count of the paper's pyramid reproduces
    the GFLOPs column of the FME-settings table at 1024x2048 (1 op per
    pixel-candidate, R counted in steps, every level runs all three stages)."""
    table = json.load(open(os.path.join(GOLDEN, "fme_settings_gflops.json")))
    ref, cur = cityscapes_pair
    for name, m in table["modes"].items():
        _, count = oracle_mod.me_c2f(ref, cur, levels=m["levels"], stages=[tuple(s) for s in m["stages"]],
                                     even=False)
        tol = 0.011 if name == "mode4" else 0.005
        assert abs(count / 1e9 - m["gflops"]) <= tol, (name, count)


def test_gop12_ablation_pin(oracle_mod, cityscapes_pair):
    """Table 8: MV-only GOP-12 cost = (key frame + 11 propagated frames) / 12
    = (557.02 + 11 * FME) / 12 = 47.94 GFLOPs with the standard FME cost."""
    g = json.load(open(os.path.join(GOLDEN, "ablation_gop12.json")))
    ref, cur = cityscapes_pair
    _, count = oracle_mod.me_c2f(ref[:256, :512], cur[:256, :512])
    per_frame = count / (256 * 512) * (1024 * 2048) / 1e9
    gop = (g["frame_by_frame_gflops"] + (g["gop"] - 1) * per_frame) / g["gop"]
    assert abs(gop - g["mv_only_gflops"]) < 0.005


def test_c2f_single_stage_is_full_search(oracle_mod):
    ref, cur = tiny_frames("scene", 64, 96, seed=9)
    for even in (True, False):
        step = 2 if even else 1
        c2f, _ = oracle_mod.me_c2f(ref, cur, levels=(16,), stages=((8 // step, step),), even=even)
        full, _ = oracle_mod.me_full(ref, cur, 16, 8, even=even)
        np.testing.assert_array_equal(as_int(c2f), as_int(full))


def test_c2f_recovers_global_shift(oracle_mod):
    """A global shift (20, -12) is reachable on the coarse-to-fine path (coarse
    step 8, then step 4, then step 1 or 2): every block whose own and parent
    displaced blocks stay in the frame matches it at zero cost."""
    rng = np.random.default_rng(31)
    big = synth.round_clip(synth.blob_texture_scene(rng, 320, 448, n_blobs=24))
    tx, ty = 20, -12
    ref = big[32:32 + 256, 32:32 + 384]
    cur = big[32 + ty:32 + ty + 256, 32 + tx:32 + tx + 384]
    for even in (False, True):
        field, _ = oracle_mod.me_c2f(ref, cur, even=even)
        B = 32
        for i in range(field.shape[0]):
            for j in range(field.shape[1]):
                flat = np.ptp(cur[i * B:(i + 1) * B, j * B:(j + 1) * B]) == 0
                pi, pj = i // 2, j // 2  # the 64-pixel parent must see the shift too
                parent_ok = 0 <= pj * 64 + tx <= 384 - 64 and 0 <= pi * 64 + ty <= 256 - 64
                if 0 <= j * B + tx <= 384 - B and 0 <= i * B + ty <= 256 - B and parent_ok and not flat:
                    assert (field["dx"][i, j], field["dy"][i, j], field["sad"][i, j]) == (tx, ty, 0)


def test_c2f_even_mapping_count(oracle_mod):
    """EVEN mode maps the fine stage (2, 1) to (1, 2): 17^2 + 9^2 + 3^2
    candidates per level."""
    ref, cur = tiny_frames("scene", 128, 128, seed=3)
    _, count = oracle_mod.me_c2f(ref, cur, even=True)
    assert count == 2 * 128 * 128 * (17 ** 2 + 9 ** 2 + 3 ** 2)
    _, count_raw = oracle_mod.me_c2f(ref, cur, even=False)
    assert count_raw == 2 * 128 * 128 * (17 ** 2 + 9 ** 2 + 5 ** 2)


# --------------------------------------------------------------------------
# learned-seeded refine
# --------------------------------------------------------------------------

def test_seeded_all_fallback_is_full_search(oracle_mod):
    f0, f1, _ = synth.planted_pair(77, 128, 128)
    h = w = 8
    z = np.zeros((h, w), np.float32)
    field, fb, _ = oracle_mod.me_seeded(f0, f1, 16, 16, z, z, z)
    full, _ = oracle_mod.me_full(f0, f1, 16, 16)
    np.testing.assert_array_equal(as_int(field), as_int(full))
    assert fb.all()


def test_seeded_at_optimum_equals_full_and_regret_nonnegative(oracle_mod):
    f0, f1, mv = synth.planted_pair(78, 128, 128, noise_sigma=2.0)
    full, _ = oracle_mod.me_full(f0, f1, 16, 16)
    one = np.ones((8, 8), np.float32)
    field, fb, _ = oracle_mod.me_seeded(f0, f1, 16, 16, full["dx"].astype(np.float32),
                                        full["dy"].astype(np.float32), one)
    np.testing.assert_array_equal(as_int(field), as_int(full))
    assert not fb.any()
    pdx, pdy, conf = synth.proposals(5, 8, 8, 16)
    field, fb, _ = oracle_mod.me_seeded(f0, f1, 16, 16, pdx, pdy, conf)
    assert (field["sad"].astype(np.int64) >= full["sad"].astype(np.int64)).all()
    assert (np.abs(field["dx"]) <= 16).all() and (np.abs(field["dy"]) <= 16).all()
    assert ((field["dx"] % 2) == 0).all() and ((field["dy"] % 2) == 0).all()
    np.testing.assert_array_equal(fb, (conf < 0.5).astype(np.uint8))


@pytest.mark.parametrize("p,centre", [(3.0, 4), (1.0, 2), (0.9, 0), (-3.0, -4), (-1.0, -2), (5.2, 6)])
def test_seeded_rounding_to_even(oracle_mod, p, centre):
    """Proposal p is rounded to the nearest even integer (half away from zero).
    On a ramp whose true shift lies far beyond the +-4 window, the chosen MV is
    the window corner facing the shift, centre + 4."""
    H = W = 128
    ref = ramp(H, W, 1, 17, 400)
    cur = ramp(H, W, 1, 17, 400, 30, 30)
    h = w = 8
    pd = np.full((h, w), p, np.float32)
    field, _, _ = oracle_mod.me_seeded(ref, cur, 16, 32, pd, pd, np.ones((h, w), np.float32))
    i = j = 2
    assert field["dx"][i, j] == centre + 4 and field["dy"][i, j] == centre + 4
