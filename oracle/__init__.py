"""CPU oracle for Bayer-domain block motion estimation and MV feature propagation.

TEST INFRASTRUCTURE ONLY.  Only ``tests/``, ``__graft_entry__.smoke()`` and the
CPU-baseline leg of ``bench.py`` may import this package.  The product path
(``paper_2508_05990_b300``) shares no code with it and never calls it.

The arithmetic lives in ``oracle.c`` (plain C, compiled here with gcc,
``-ffp-contract=off``); this module only marshals numpy arrays.  Each function
cites the passage of arXiv 2508.05990 it restates:

* ``me_stage``   -- one coarse-to-fine matching stage (Sec. 3.2 "Parallel
  Coarse-to-fine Block Matching"; Sec. 4.1 "CUDA Settings": (2R+1)^2
  candidates, R counted in steps) with the SAD criterion (Sec. 3.2 "Matching
  Criterion").
* ``me_full``    -- exhaustive block matching, the plain definition of ME
  (Sec. 2.2 "Definition", "Block Matching-based ME").
* ``me_c2f``     -- the block pyramid x three stages (Sec. 3.2 "Pyramid Block
  Structure"; FME-settings table).
* ``me_seeded``  -- one R=2/step-2 stage around a proposal, full search below a
  confidence threshold (the learned-proposal form; not in the paper).
* ``propagate``  -- z_pred = Warp(z_R, MV) (Sec. 3.3), NEAREST and BILINEAR in
  float with a fixed evaluation order; ``propagate_bilinear_f64`` in double.

Readings of points the paper leaves open (MV sign, out-of-frame candidates,
partial blocks, tie-break, CFA phase, interpolation) are stated in the header
of ``oracle.c``.
"""
from __future__ import annotations

import ctypes
import os
import subprocess
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "oracle.c")
_LIB = os.path.join(_HERE, "liboracle.so")
_lock = threading.Lock()
_lib = None

MV_DTYPE = np.dtype([("dx", "<i2"), ("dy", "<i2"), ("sad", "<u4")])

# Paper standard FME setting (FME-settings table): blocks [64, 32],
# stages (R, step) = (8, 8), (4, 4), (2, 1).
STANDARD_LEVELS = (64, 32)
STANDARD_STAGES = ((8, 8), (4, 4), (2, 1))


def build(force: bool = False) -> str:
    """Compile ``oracle.c`` into ``liboracle.so`` (gcc, OpenMP, no FP contraction)."""
    with _lock:
        if force or not os.path.exists(_LIB) or os.path.getmtime(_LIB) < os.path.getmtime(_SRC):
            cmd = ["gcc", "-O2", "-fopenmp", "-ffp-contract=off", "-fno-fast-math", "-fPIC",
                   "-shared", "-std=c11", "-Wall", "-o", _LIB + ".tmp", _SRC, "-lm"]
            subprocess.run(cmd, check=True)
            os.replace(_LIB + ".tmp", _LIB)
    return _LIB


def _load():
    global _lib
    if _lib is None:
        build()
        lib = ctypes.CDLL(_LIB)
        P = ctypes.c_void_p
        I = ctypes.c_int
        F = ctypes.c_float
        LL = ctypes.c_longlong
        lib.oracle_set_threads.argtypes = [I]
        lib.oracle_get_threads.restype = I
        lib.oracle_me_stage.argtypes = [P, P, I, I, I, I, I, I, I, P, P]
        lib.oracle_me_stage.restype = LL
        lib.oracle_me_full.argtypes = [P, P, I, I, I, I, I, I, P]
        lib.oracle_me_full.restype = LL
        lib.oracle_me_c2f.argtypes = [P, P, I, I, I, P, I, P, P, I, I, P]
        lib.oracle_me_c2f.restype = LL
        lib.oracle_me_seeded.argtypes = [P, P, I, I, I, I, I, P, P, P, F, P, P]
        lib.oracle_me_seeded.restype = LL
        lib.oracle_propagate_f32.argtypes = [P, I, I, I, I, I, P, I, I, I, I, P]
        lib.oracle_propagate_bilinear_f64.argtypes = [P, I, I, I, I, P, I, I, I, I, P]
        _lib = lib
    return _lib


def _ptr(a: np.ndarray):
    return ctypes.c_void_p(a.ctypes.data)


def _frames(ref, cur):
    ref = np.ascontiguousarray(ref, dtype=np.uint16)
    cur = np.ascontiguousarray(cur, dtype=np.uint16)
    if ref.shape != cur.shape or ref.ndim != 2:
        raise ValueError("ref and cur must be 2-D frames of one shape")
    return ref, cur


def set_threads(n: int) -> None:
    _load().oracle_set_threads(int(n))


def get_threads() -> int:
    return int(_load().oracle_get_threads())


def grid_shape(H: int, W: int, B: int):
    """MV field shape h x w = ceil(H/B) x ceil(W/B) (Sec. 4.1 "CUDA Settings")."""
    return (H + B - 1) // B, (W + B - 1) // B


def me_stage(ref, cur, B, R, step, lim=1 << 30, center=None):
    """One stage: candidates center + (u*step, v*step), |u|,|v| <= R, |dx|,|dy| <= lim.

    Returns (field[h, w] of MV_DTYPE, scheduled pixel-candidate count)."""
    ref, cur = _frames(ref, cur)
    H, W = ref.shape
    h, w = grid_shape(H, W, B)
    out = np.zeros((h, w), MV_DTYPE)
    cptr = None
    if center is not None:
        center = np.ascontiguousarray(center, dtype=MV_DTYPE).reshape(h, w)
        cptr = _ptr(center)
    n = _load().oracle_me_stage(_ptr(ref), _ptr(cur), W, H, W, B, R, step, lim, cptr, _ptr(out))
    if n < 0:
        raise RuntimeError("a block had no valid candidate")
    return out, int(n)


def me_full(ref, cur, B, search_range, even=True):
    """Exhaustive search over |dx|,|dy| <= range (EVEN: even offsets only)."""
    ref, cur = _frames(ref, cur)
    H, W = ref.shape
    h, w = grid_shape(H, W, B)
    out = np.zeros((h, w), MV_DTYPE)
    n = _load().oracle_me_full(_ptr(ref), _ptr(cur), W, H, W, B, search_range, 1 if even else 0, _ptr(out))
    if n < 0:
        raise RuntimeError("a block had no valid candidate")
    return out, int(n)


def me_c2f(ref, cur, levels=STANDARD_LEVELS, stages=STANDARD_STAGES, even=False):
    """Block pyramid x coarse-to-fine stages; returns (finest field, pixel-candidate count)."""
    ref, cur = _frames(ref, cur)
    H, W = ref.shape
    lv = np.ascontiguousarray(levels, dtype=np.int32)
    sr = np.ascontiguousarray([s[0] for s in stages], dtype=np.int32)
    ss = np.ascontiguousarray([s[1] for s in stages], dtype=np.int32)
    h, w = grid_shape(H, W, int(lv[-1]))
    out = np.zeros((h, w), MV_DTYPE)
    n = _load().oracle_me_c2f(_ptr(ref), _ptr(cur), W, H, W, _ptr(lv), len(lv), _ptr(sr), _ptr(ss),
                              len(sr), 1 if even else 0, _ptr(out))
    return out, int(n)


def me_seeded(ref, cur, B, search_range, prop_dx, prop_dy, conf, thresh=0.5):
    """Refine +-4 (R=2, step 2) around each proposal; full search where conf < thresh.

    Returns (field, fallback flags[h, w] uint8, pixel-candidate count)."""
    ref, cur = _frames(ref, cur)
    H, W = ref.shape
    h, w = grid_shape(H, W, B)
    pdx = np.ascontiguousarray(prop_dx, dtype=np.float32).reshape(h, w)
    pdy = np.ascontiguousarray(prop_dy, dtype=np.float32).reshape(h, w)
    cf = np.ascontiguousarray(conf, dtype=np.float32).reshape(h, w)
    out = np.zeros((h, w), MV_DTYPE)
    fb = np.zeros((h, w), np.uint8)
    n = _load().oracle_me_seeded(_ptr(ref), _ptr(cur), W, H, W, B, search_range, _ptr(pdx), _ptr(pdy),
                                 _ptr(cf), float(thresh), _ptr(out), _ptr(fb))
    return out, fb, int(n)


NEAREST, BILINEAR = 0, 1
NCHW, NHWC = 0, 1


def _feat(feat, layout):
    feat = np.ascontiguousarray(feat, dtype=np.float32)
    if feat.ndim != 3:
        raise ValueError("feature map must be 3-D (C,H,W) or (H,W,C)")
    if layout == NCHW:
        C, Hf, Wf = feat.shape
    else:
        Hf, Wf, C = feat.shape
    return feat, C, Hf, Wf


def propagate(feat, mv, B, stride, interp=BILINEAR, layout=NCHW):
    """z_pred = Warp(z_R, MV) in float (Sec. 3.3); returns an array shaped like feat."""
    feat, C, Hf, Wf = _feat(feat, layout)
    mv = np.ascontiguousarray(mv, dtype=MV_DTYPE)
    out = np.empty_like(feat)
    _load().oracle_propagate_f32(_ptr(feat), C, Hf, Wf, layout, interp, _ptr(mv), mv.shape[0], mv.shape[1],
                                 B, stride, _ptr(out))
    return out


def propagate_bilinear_f64(feat, mv, B, stride, layout=NCHW):
    """Bilinear Warp evaluated in double (precision reference)."""
    feat, C, Hf, Wf = _feat(feat, layout)
    mv = np.ascontiguousarray(mv, dtype=MV_DTYPE)
    out = np.empty(feat.shape, np.float64)
    _load().oracle_propagate_bilinear_f64(_ptr(feat), C, Hf, Wf, layout, _ptr(mv), mv.shape[0], mv.shape[1],
                                          B, stride, _ptr(out))
    return out
