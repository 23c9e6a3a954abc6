"""Seeded synthetic inputs: RGGB Bayer frames (12-bit values in uint16), feature
maps and MV proposals.

This module is the one piece shared by the CUDA path's tests/benchmark and by
the CPU oracle's tests: it draws inputs only and holds none of the method's
arithmetic (no SAD, no search, no warp).

The paper evaluates on CamVid, Cityscapes and ImageNet VID Bayer frames
synthesised through Invertible-ISP (Sec. 4.1), none of which is available here;
these generators stand in for them with scenes of the same kind of structure:
smooth blobs plus fine texture, a global camera pan, independently moving
rectangles, and Poisson-Gaussian sensor noise.  The scene is monochrome (no
per-channel CFA gains) unless ``cfa_gains`` is given.

Recipe (all draws from numpy's PCG64 via ``np.random.default_rng(seed)``):

* blobs: ``n_blobs`` Gaussians A*exp(-r^2 / (2 sigma^2)), A ~ U[200, 3000] DN,
  sigma ~ U[4, 24] px, centre ~ U over the canvas, evaluated within 5 sigma of
  the centre; default ``n_blobs = round(64 * H*W / 256^2)``;
* texture: integer U{-50..50} DN per pixel;
* rounding: half away from zero, then clip to [0, 4095].
"""
from __future__ import annotations

import numpy as np

MAX_DN = 4095


def round_clip(x: np.ndarray) -> np.ndarray:
    """Round half away from zero and clip to the 12-bit range; returns uint16."""
    r = np.sign(x) * np.floor(np.abs(x) + 0.5)
    return np.clip(r, 0, MAX_DN).astype(np.uint16)


def blob_texture_scene(rng: np.random.Generator, H: int, W: int, n_blobs: int | None = None) -> np.ndarray:
    """Clean (unrounded) scene: sum of Gaussian blobs plus integer texture, float64."""
    if n_blobs is None:
        n_blobs = max(1, int(round(64 * H * W / (256 * 256))))
    img = np.zeros((H, W), np.float64)
    amp = rng.uniform(200.0, 3000.0, n_blobs)
    sig = rng.uniform(4.0, 24.0, n_blobs)
    cy = rng.uniform(0.0, H, n_blobs)
    cx = rng.uniform(0.0, W, n_blobs)
    for a, s, y, x in zip(amp, sig, cy, cx):
        rad = 5.0 * s
        y0, y1 = max(0, int(np.floor(y - rad))), min(H, int(np.ceil(y + rad)) + 1)
        x0, x1 = max(0, int(np.floor(x - rad))), min(W, int(np.ceil(x + rad)) + 1)
        if y0 >= y1 or x0 >= x1:
            continue
        yy = (np.arange(y0, y1, dtype=np.float64) - y)[:, None]
        xx = (np.arange(x0, x1, dtype=np.float64) - x)[None, :]
        img[y0:y1, x0:x1] += a * np.exp(-(yy * yy + xx * xx) / (2.0 * s * s))
    img += rng.integers(-50, 51, size=(H, W)).astype(np.float64)
    return img


def planted_pair(seed: int, H: int = 256, W: int = 256, block: int = 16, max_shift: int = 8,
                 noise_sigma: float = 2.0, even: bool = True):
    """Parity pair with planted per-block integer MVs (the 256x256 workload).

    frame0 = blobs + texture; for each block (i, j) an MV (dx, dy) is drawn from
    {-max_shift, ..., max_shift} (even values only when ``even``) and
    frame1[y, x] = frame0[clamp(y + dy), clamp(x + dx)] + N(0, noise_sigma^2),
    rounded and clipped.  So the current block at (x, y) matches the reference
    at (x + dx, y + dy).  Returns (frame0, frame1, mv_true[h, w, 2] as (dx, dy)).
    """
    rng = np.random.default_rng(seed)
    f0 = round_clip(blob_texture_scene(rng, H, W))
    h, w = (H + block - 1) // block, (W + block - 1) // block
    vals = np.arange(-max_shift, max_shift + 1, 2 if even else 1)
    mv = rng.choice(vals, size=(h, w, 2))
    f1 = np.empty((H, W), np.float64)
    for i in range(h):
        for j in range(w):
            dx, dy = int(mv[i, j, 0]), int(mv[i, j, 1])
            ys = np.clip(np.arange(i * block, min(H, (i + 1) * block)) + dy, 0, H - 1)
            xs = np.clip(np.arange(j * block, min(W, (j + 1) * block)) + dx, 0, W - 1)
            f1[i * block:(i + 1) * block, j * block:(j + 1) * block] = f0[np.ix_(ys, xs)]
    if noise_sigma > 0:
        f1 = f1 + rng.normal(0.0, noise_sigma, size=(H, W))
    return f0, round_clip(f1), mv.astype(np.int32)


def pan_clip(seed: int, H: int, W: int, n_frames: int = 8, n_rects: int = 12, gain: float = 0.5,
             read_sigma: float = 3.0, pan_speed=(2.0, 6.0), rect_size=(32, 256), rect_speed: float = 20.0,
             cfa_gains=None) -> np.ndarray:
    """Moving-scene clip [n_frames, H, W] uint16 (the 1080p / 4K / multi-stream workloads).

    * static background: blobs + texture on a canvas with a margin for the pan;
      global pan direction ~ U[0, 2 pi), speed ~ U[pan_speed] px/frame, the
      offset rounded to integers per frame;
    * ``n_rects`` rectangles, side lengths ~ U{rect_size}, own level
      U[200, 3000] + own texture U{-50..50}, start ~ U over the frame, velocity
      ~ U[-rect_speed, rect_speed]^2 px/frame, positions rounded per frame,
      composited in index order;
    * clean frame clipped to [0, 4095]; Poisson-Gaussian noise
      gain * Poisson(x / gain) + N(0, read_sigma^2); rounded, clipped.
    * ``cfa_gains``: optional (gR, gG, gB) multiplied into the RGGB sites of the
      clean frame (R at (0, 0)).
    """
    rng = np.random.default_rng(seed)
    margin = int(np.ceil(pan_speed[1] * (n_frames - 1))) + 2
    canvas = blob_texture_scene(rng, H + 2 * margin, W + 2 * margin)
    theta = rng.uniform(0.0, 2.0 * np.pi)
    speed = rng.uniform(pan_speed[0], pan_speed[1])
    rw = rng.integers(rect_size[0], rect_size[1] + 1, n_rects)
    rh = rng.integers(rect_size[0], rect_size[1] + 1, n_rects)
    rx = rng.uniform(0.0, W, n_rects)
    ry = rng.uniform(0.0, H, n_rects)
    vx = rng.uniform(-rect_speed, rect_speed, n_rects)
    vy = rng.uniform(-rect_speed, rect_speed, n_rects)
    level = rng.uniform(200.0, 3000.0, n_rects)
    tex = [rng.integers(-50, 51, size=(int(rh[k]), int(rw[k]))).astype(np.float64) + level[k]
           for k in range(n_rects)]
    frames = np.empty((n_frames, H, W), np.uint16)
    for t in range(n_frames):
        ox = int(np.round(t * speed * np.cos(theta)))
        oy = int(np.round(t * speed * np.sin(theta)))
        img = canvas[margin + oy:margin + oy + H, margin + ox:margin + ox + W].copy()
        for k in range(n_rects):
            px = int(np.round(rx[k] + t * vx[k]))
            py = int(np.round(ry[k] + t * vy[k]))
            y0, y1 = max(0, py), min(H, py + int(rh[k]))
            x0, x1 = max(0, px), min(W, px + int(rw[k]))
            if y0 < y1 and x0 < x1:
                img[y0:y1, x0:x1] = tex[k][y0 - py:y1 - py, x0 - px:x1 - px]
        if cfa_gains is not None:
            gR, gG, gB = cfa_gains
            img[0::2, 0::2] *= gR
            img[0::2, 1::2] *= gG
            img[1::2, 0::2] *= gG
            img[1::2, 1::2] *= gB
        clean = np.clip(img, 0.0, MAX_DN)
        noisy = gain * rng.poisson(clean / gain) + rng.normal(0.0, read_sigma, size=(H, W))
        frames[t] = round_clip(noisy)
    return frames


def features(seed: int, C: int, Hf: int, Wf: int, n: int = 1, layout: str = "NCHW") -> np.ndarray:
    """N(0, 1) float32 feature maps standing in for base-model features z_R.

    Shape (n, C, Hf, Wf) for NCHW or (n, Hf, Wf, C) for NHWC."""
    rng = np.random.default_rng(seed)
    shape = (n, C, Hf, Wf) if layout == "NCHW" else (n, Hf, Wf, C)
    return rng.standard_normal(shape, dtype=np.float32)


def proposals(seed: int, h: int, w: int, search_range: int, true_mv=None, jitter: float = 3.0):
    """Synthetic MV proposals (dx, dy float32) and confidences in [0, 1).

    With ``true_mv`` [h, w, 2] the proposal is true_mv + N(0, jitter^2);
    otherwise U[-range, range].  Confidence ~ U[0, 1)."""
    rng = np.random.default_rng(seed)
    if true_mv is not None:
        base = np.asarray(true_mv, np.float64)
        p = base + rng.normal(0.0, jitter, size=base.shape)
    else:
        p = rng.uniform(-search_range, search_range, size=(h, w, 2))
    conf = rng.uniform(0.0, 1.0, size=(h, w)).astype(np.float32)
    return p[..., 0].astype(np.float32), p[..., 1].astype(np.float32), conf


def he_normal_params(seed: int, shapes) -> np.ndarray:
    """Initial network parameters, flat float32: for each (kind, shape) in order,
    kind "w" draws N(0, 2 / fan_in) with fan_in = prod(shape[1:]) (He-normal) and
    kind "b" gives zeros.  Random draws only; the layout is the caller's."""
    rng = np.random.default_rng(seed)
    parts = []
    for kind, shape in shapes:
        n = int(np.prod(shape))
        if kind == "b":
            parts.append(np.zeros(n))
        else:
            parts.append(rng.normal(0.0, np.sqrt(2.0 / int(np.prod(shape[1:]))), n))
    return np.concatenate(parts).astype(np.float32)


# Workloads (all synthetic).  Seeds: workload k uses 1000 + k; clips and
# streams add their index.
WORKLOADS = {
    "parity_256": dict(W=256, H=256, block=16, range=16, C=64, stride=4, seed=1000),
    "1080p": dict(W=1920, H=1088, frames=8, block=16, range=32, C=256, stride=8, seed=1001),
    "4k": dict(W=3840, H=2160, frames=8, block=16, range=32, C=128, stride=4, seed=1002),
}
