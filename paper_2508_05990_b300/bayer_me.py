"""Thin ctypes binding of libbayer_me.so (C ABI in include/bayer_me.h).

Argument marshalling only: every step of the path runs in the library's CUDA
kernels.  Device buffers are torch CUDA tensors (PyTorch provides device memory
and streams); calls are asynchronous on the current torch stream unless a
stream is given.  If the library is missing this module raises on use -- there
is no fallback.

Names follow the C ABI: ``init``/``destroy`` create and release a handle;
``estimate``, ``estimate_ex``, ``feat_propagate``, ``clip_process_host``,
``sync_status`` and ``probe_alu`` wrap the entry points of the same name.
"""
from __future__ import annotations

import ctypes
import os
from dataclasses import dataclass, field

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_HERE, "libbayer_me.so")

MV_DTYPE = np.dtype([("dx", "<i2"), ("dy", "<i2"), ("sad", "<u4")])

OK, ERR_INVALID_ARG, ERR_UNSUPPORTED, ERR_CUDA, ERR_OOM, ERR_TIMEOUT = range(6)
MODE_FULL, MODE_C2F, MODE_SEEDED = 0, 1, 2
PHASE_EVEN, PHASE_RAW = 0, 1
INTERP_NEAREST, INTERP_BILINEAR = 0, 1
LAYOUT_NCHW, LAYOUT_NHWC = 0, 1
MAX_LEVELS = MAX_STAGES = 4

# Every function the header declares (checked against include/bayer_me.h by the tests).
EXPORTS = ("bayer_me_init", "bayer_me_destroy", "bayer_status_string", "bayer_me_estimate",
           "bayer_me_estimate_ex", "bayer_feat_propagate", "bayer_clip_process_host", "bayer_me_sync_status",
           "bayer_probe_alu", "bayer_me_estimate_c2f_noalloc", "bayer_cnn_forward", "bayer_cnn_loss_grad",
           "bayer_cnn_adamw", "bayer_me_estimate_learned", "bayer_refine_conv", "bayer_me_multi_stream",
           "bayer_me_selftest_wait", "bayer_me_debug_fail_allocs")
PREC_BF16, PREC_FP32 = 0, 1

# Flat parameter layout of the proposal network (BAYER_CNN_* in the header).
CNN_OFFSETS = dict(w1=0, b1=2304, w2=2336, b2=11552, w3=11584, b3=20800, w4=20832, b4=30048, wh=30080, bh=30464)
CNN_NPARAMS = 30476
CNN_SHAPES = [("w", (32, 8, 3, 3)), ("b", (32,)), ("w", (32, 32, 3, 3)), ("b", (32,)), ("w", (32, 32, 3, 3)),
              ("b", (32,)), ("w", (32, 32, 3, 3)), ("b", (32,)), ("w", (12, 32)), ("b", (12,))]


class BayerError(RuntimeError):
    def __init__(self, status: int, what: str):
        super().__init__(f"{what}: {status_string(status)} (status {status})")
        self.status = status


class PairDesc(ctypes.Structure):
    """bayer_pair_t: one frame pair (device buffers) of a multi-stream call."""
    _fields_ = [("ref", ctypes.c_void_p), ("cur", ctypes.c_void_p), ("W", ctypes.c_int), ("H", ctypes.c_int),
                ("pitch", ctypes.c_int), ("mv_out", ctypes.c_void_p), ("feat", ctypes.c_void_p),
                ("feat_out", ctypes.c_void_p), ("C", ctypes.c_int), ("Hf", ctypes.c_int), ("Wf", ctypes.c_int),
                ("stride", ctypes.c_int)]


class Params(ctypes.Structure):
    _fields_ = [("mode", ctypes.c_int), ("phase", ctypes.c_int), ("block", ctypes.c_int), ("range", ctypes.c_int),
                ("n_levels", ctypes.c_int), ("levels", ctypes.c_int * MAX_LEVELS),
                ("n_stages", ctypes.c_int), ("stage_radius", ctypes.c_int * MAX_STAGES),
                ("stage_step", ctypes.c_int * MAX_STAGES), ("conf_thresh", ctypes.c_float),
                ("batch", ctypes.c_int), ("ref_batch_stride", ctypes.c_longlong),
                ("cur_batch_stride", ctypes.c_longlong)]


_lib = None


def load(path: str = LIB_PATH):
    """Load the CUDA library (raises if it has not been built)."""
    global _lib
    if _lib is not None:
        return _lib
    if not os.path.exists(path):
        raise RuntimeError(f"libbayer_me.so not built at {path}; run `python -m paper_2508_05990_b300.build`")
    lib = ctypes.CDLL(path)
    P, I, F, LL = ctypes.c_void_p, ctypes.c_int, ctypes.c_float, ctypes.c_longlong
    lib.bayer_me_init.argtypes = [ctypes.POINTER(P), I]
    lib.bayer_me_destroy.argtypes = [P]
    lib.bayer_status_string.argtypes = [I]
    lib.bayer_status_string.restype = ctypes.c_char_p
    lib.bayer_me_estimate.argtypes = [P, P, P, I, I, I, I, P, P]
    lib.bayer_me_estimate_ex.argtypes = [P, P, P, I, I, I, ctypes.POINTER(Params), P, P, P, P, P]
    lib.bayer_feat_propagate.argtypes = [P, P, I, I, I, I, I, I, P, I, I, I, I, P, P]
    lib.bayer_clip_process_host.argtypes = [P, P, I, I, I, I, I, P, I, I, I, I, I, P, P]
    lib.bayer_me_sync_status.argtypes = [P, P]
    lib.bayer_probe_alu.argtypes = [P, I, ctypes.POINTER(ctypes.c_double), ctypes.POINTER(ctypes.c_double),
                                    ctypes.POINTER(ctypes.c_int)]
    lib.bayer_me_estimate_c2f_noalloc.argtypes = [P, P, I, I, I, ctypes.POINTER(Params), P, P]
    lib.bayer_cnn_forward.argtypes = [P, P, P, I, I, I, I, LL, LL, P, I, P, P, P]
    lib.bayer_cnn_loss_grad.argtypes = [P, P, P, I, I, I, I, LL, LL, P, P, I, F, P, P, P]
    lib.bayer_cnn_adamw.argtypes = [P, P, P, P, P, P, I, F, F, F, F, F, P]
    lib.bayer_me_estimate_learned.argtypes = [P, P, P, I, I, I, I, LL, LL, P, I, F, P, P, P, P]
    lib.bayer_refine_conv.argtypes = [P, P, I, I, I, I, I, P, P, P, P, P, P, I, P, P]
    lib.bayer_me_multi_stream.argtypes = [P, ctypes.POINTER(PairDesc), I, I, I, P, ctypes.POINTER(ctypes.c_int), P]
    lib.bayer_me_selftest_wait.argtypes = [P, I, ctypes.c_uint, P]
    lib.bayer_me_debug_fail_allocs.argtypes = [P, I]
    for name in EXPORTS:
        if name != "bayer_status_string":
            getattr(lib, name).restype = I
    _lib = lib
    return lib


def status_string(status: int) -> str:
    return load().bayer_status_string(int(status)).decode()


def _check(status: int, what: str) -> None:
    if status != OK:
        raise BayerError(status, what)


def _stream(stream):
    if stream is None:
        import torch
        return ctypes.c_void_p(torch.cuda.current_stream().cuda_stream)
    if isinstance(stream, int):
        return ctypes.c_void_p(stream)
    return ctypes.c_void_p(stream.cuda_stream)


def _ptr(t) -> ctypes.c_void_p:
    if t is None:
        return ctypes.c_void_p(None)
    return ctypes.c_void_p(t.data_ptr())


def _check_out(out, numel: int, dtype, device, what: str) -> None:
    """A caller-supplied output must be a contiguous tensor of the record (or
    value) dtype on the inputs' device, with room for every element the kernel
    writes: the kernels write numel elements from its first address."""
    if out.dtype != dtype or not out.is_contiguous() or out.device != device or out.numel() < numel:
        raise ValueError(f"{what}: out must be a contiguous {dtype} tensor on {device} with at least {numel} "
                         f"elements (got {out.dtype}, {tuple(out.shape)}, contiguous={out.is_contiguous()}, "
                         f"{out.device})")


def grid_shape(H: int, W: int, block: int):
    return (H + block - 1) // block, (W + block - 1) // block


@dataclass
class C2FSetting:
    """Pyramid levels (block sizes, large to small) x stages (radius in steps, step)."""
    levels: tuple = (64, 32)
    stages: tuple = ((8, 8), (4, 4), (2, 1))


# The paper's FME settings (Sec. 4.2, FME-settings table; Sec. 3.2 for the
# standard pyramid): block sizes per level, (radius in steps, step) per stage.
C2F_PRESETS = {
    "standard": C2FSetting((64, 32), ((8, 8), (4, 4), (2, 1))),
    "mode1": C2FSetting((64, 32), ((4, 8), (2, 4), (2, 1))),
    "mode2": C2FSetting((64, 32), ((10, 8), (6, 4), (4, 1))),
    "mode3": C2FSetting((32,), ((8, 8), (4, 4), (2, 1))),
    "mode4": C2FSetting((64, 32, 16, 8), ((8, 8), (4, 4), (2, 1))),
}


def c2f_pixel_candidates(setting: C2FSetting, H: int, W: int, even: bool = True) -> int:
    """Pixel-candidates one pair's C2F search schedules (candidates leaving the
    frame included): sum over levels and stages of blocks x block pixels x
    (2R+1)^2, with EVEN mapping an odd step s to s+1 and R*s/(s+1) steps."""
    total = 0
    for B in setting.levels:
        blocks = -(-H // B) * -(-W // B)
        for R, st in setting.stages:
            if even and st % 2:
                R, st = R * st // (st + 1), st + 1
            total += blocks * B * B * (2 * R + 1) ** 2
    return total


class Handle:
    """A library handle bound to one CUDA device (``bayer_me_init``)."""

    def __init__(self, device: int = 0):
        self._lib = load()
        self._h = ctypes.c_void_p()
        _check(self._lib.bayer_me_init(ctypes.byref(self._h), int(device)), "bayer_me_init")
        self.device = device

    def close(self):
        if self._h:
            _check(self._lib.bayer_me_destroy(self._h), "bayer_me_destroy")
            self._h = ctypes.c_void_p()

    destroy = close

    def __enter__(self):
        return self

    def __exit__(self, *exc):
        self.close()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    # -- motion estimation ---------------------------------------------------
    def estimate(self, ref, cur, block: int = 16, search_range: int = 32, out=None, stream=None):
        """Exhaustive EVEN search of one pair; returns an int32 tensor [h, w, 2] view of the records."""
        import torch
        H, W = ref.shape[-2:]
        h, w = grid_shape(H, W, block)
        if out is None:
            out = torch.empty((h, w, 2), dtype=torch.int32, device=ref.device)
        _check_out(out, h * w * 2, torch.int32, ref.device, "estimate")
        _check(self._lib.bayer_me_estimate(self._h, _ptr(ref), _ptr(cur), W, H, block, search_range, _ptr(out),
                                           _stream(stream)), "bayer_me_estimate")
        return out

    def estimate_ex(self, ref, cur, mode=MODE_FULL, phase=PHASE_EVEN, block=16, search_range=32, c2f=None,
                    prop_dxdy=None, conf=None, conf_thresh=0.5, batch=1, ref_batch_stride=0, cur_batch_stride=0,
                    out=None, fallback=None, stream=None, W=None, H=None, pitch=None):
        """General search (FULL / C2F / SEEDED; EVEN / RAW; batched).  ``ref``/``cur`` are uint16
        tensors whose first frame is the first pair's; returns the [batch, h, w, 2] int32 record tensor."""
        import torch
        if H is None or W is None:
            H, W = ref.shape[-2:]
        if pitch is None:
            pitch = W
        p = Params()
        p.mode, p.phase, p.block, p.range = mode, phase, block, search_range
        out_block = block
        if mode == MODE_C2F:
            c2f = c2f or C2FSetting()
            p.n_levels = len(c2f.levels)
            for i, b in enumerate(c2f.levels):
                p.levels[i] = b
            p.n_stages = len(c2f.stages)
            for i, (r, s) in enumerate(c2f.stages):
                p.stage_radius[i] = r
                p.stage_step[i] = s
            out_block = c2f.levels[-1]
        p.conf_thresh = conf_thresh
        p.batch = batch
        p.ref_batch_stride = ref_batch_stride
        p.cur_batch_stride = cur_batch_stride
        h, w = grid_shape(H, W, out_block)
        if out is None:
            out = torch.empty((batch, h, w, 2), dtype=torch.int32, device=ref.device)
        _check_out(out, batch * h * w * 2, torch.int32, ref.device, "estimate_ex")
        _check(self._lib.bayer_me_estimate_ex(self._h, _ptr(ref), _ptr(cur), W, H, pitch, ctypes.byref(p),
                                              _ptr(prop_dxdy), _ptr(conf), _ptr(out), _ptr(fallback),
                                              _stream(stream)), "bayer_me_estimate_ex")
        return out

    # -- propagation ---------------------------------------------------------
    def feat_propagate(self, feat, mv, block: int, stride: int, interp=INTERP_BILINEAR, layout=LAYOUT_NCHW,
                       out=None, stream=None):
        """z_pred = Warp(z_R, MV).  feat: float32 [n, C, Hf, Wf] (NCHW) or [n, Hf, Wf, C] (NHWC);
        mv: int32 records [n, mv_h, mv_w, 2]."""
        import torch
        if feat.dim() == 3:
            feat = feat.unsqueeze(0)
        if mv.dim() == 3:
            mv = mv.unsqueeze(0)
        n = feat.shape[0]
        if layout == LAYOUT_NCHW:
            C, Hf, Wf = feat.shape[1:]
        else:
            Hf, Wf, C = feat.shape[1:]
        if out is None:
            out = torch.empty_like(feat)
        _check(self._lib.bayer_feat_propagate(self._h, _ptr(feat), n, C, Hf, Wf, layout, interp, _ptr(mv),
                                              mv.shape[1], mv.shape[2], block, stride, _ptr(out),
                                              _stream(stream)), "bayer_feat_propagate")
        return out

    # -- host-buffer end-to-end path -----------------------------------------
    def clip_process_host(self, frames: np.ndarray, feats: np.ndarray, block=16, search_range=32, stride=8,
                          interp=INTERP_BILINEAR, mv_out=None, feat_out=None):
        """frames: host uint16 [T, H, W]; feats: host float32 [T-1, C, Hf, Wf].  Returns
        (mv records [T-1, h, w] MV_DTYPE, propagated features [T-1, C, Hf, Wf])."""
        T, H, W = frames.shape
        _, C, Hf, Wf = feats.shape
        h, w = grid_shape(H, W, block)
        if mv_out is None:
            mv_out = np.empty((T - 1, h, w), MV_DTYPE)
        if feat_out is None:
            feat_out = np.empty_like(feats)
        for a in (frames, feats, mv_out, feat_out):
            if not a.flags["C_CONTIGUOUS"]:
                raise ValueError("host buffers must be C-contiguous")
        _check(self._lib.bayer_clip_process_host(self._h, frames.ctypes.data, T, W, H, block, search_range,
                                                 feats.ctypes.data, C, Hf, Wf, stride, interp,
                                                 mv_out.ctypes.data, feat_out.ctypes.data),
               "bayer_clip_process_host")
        return mv_out, feat_out

    # -- learned proposal network and learned-seeded search -----------------
    def cnn_forward(self, ref, cur, w_bf16, search_range=32, batch=1, ref_batch_stride=0, cur_batch_stride=0,
                    prop=None, conf=None, stream=None):
        """Proposals [batch, h, w, 2] and confidences [batch, h, w] (float32 tensors);
        h = ceil(H / 16), w = W / 16."""
        import torch
        H, W = ref.shape[-2:]
        h, w = grid_shape(H, W, 16)
        if prop is None:
            prop = torch.empty((batch, h, w, 2), dtype=torch.float32, device=ref.device)
        if conf is None:
            conf = torch.empty((batch, h, w), dtype=torch.float32, device=ref.device)
        _check(self._lib.bayer_cnn_forward(self._h, _ptr(ref), _ptr(cur), W, H, W, batch, ref_batch_stride,
                                           cur_batch_stride, _ptr(w_bf16), search_range, _ptr(prop), _ptr(conf),
                                           _stream(stream)), "bayer_cnn_forward")
        return prop, conf

    def cnn_loss_grad(self, ref, cur, w_bf16, labels, search_range=32, batch=1, ref_batch_stride=0,
                      cur_batch_stride=0, grad=None, loss=None, neg_weight=1.0, stream=None):
        """(grad [CNN_NPARAMS], loss [1]) float32 tensors; labels: int32 records [batch, h, w, 2]."""
        import torch
        H, W = ref.shape[-2:]
        if grad is None:
            grad = torch.empty(CNN_NPARAMS, dtype=torch.float32, device=ref.device)
        if loss is None:
            loss = torch.empty(1, dtype=torch.float32, device=ref.device)
        _check(self._lib.bayer_cnn_loss_grad(self._h, _ptr(ref), _ptr(cur), W, H, W, batch, ref_batch_stride,
                                             cur_batch_stride, _ptr(w_bf16), _ptr(labels), search_range,
                                             float(neg_weight), _ptr(grad),
                                             _ptr(loss), _stream(stream)), "bayer_cnn_loss_grad")
        return grad, loss

    def cnn_adamw(self, w, w_bf16, grad, m, v, step, lr, beta1=0.9, beta2=0.999, eps=1e-8, weight_decay=0.01,
                  stream=None):
        _check(self._lib.bayer_cnn_adamw(self._h, _ptr(w), _ptr(w_bf16), _ptr(grad), _ptr(m), _ptr(v), int(step),
                                         float(lr), float(beta1), float(beta2), float(eps), float(weight_decay),
                                         _stream(stream)), "bayer_cnn_adamw")

    def estimate_learned(self, ref, cur, w_bf16, search_range=32, conf_thresh=0.5, batch=1, ref_batch_stride=0,
                         cur_batch_stride=0, out=None, fallback=None, n_fallback=None, stream=None):
        """Learned-seeded search; returns the [batch, h, w, 2] int32 record tensor
        (h = ceil(H / 16): a last block row clipped by the frame counts)."""
        import torch
        H, W = ref.shape[-2:]
        h, w = grid_shape(H, W, 16)
        if out is None:
            out = torch.empty((batch, h, w, 2), dtype=torch.int32, device=ref.device)
        _check_out(out, batch * h * w * 2, torch.int32, ref.device, "estimate_learned")
        _check(self._lib.bayer_me_estimate_learned(self._h, _ptr(ref), _ptr(cur), W, H, W, batch, ref_batch_stride,
                                                   cur_batch_stride, _ptr(w_bf16), search_range, float(conf_thresh),
                                                   _ptr(out), _ptr(fallback), _ptr(n_fallback), _stream(stream)),
               "bayer_me_estimate_learned")
        return out

    def refine_conv(self, feat, weights, precision=PREC_BF16, out=None, stream=None):
        """Three 3x3 convs C -> hidden -> hidden -> C on NHWC float32 feat [n, Hf, Wf, C];
        weights = (w1, b1, w2, b2, w3, b3) float32 CUDA tensors."""
        import torch
        if feat.dim() == 3:
            feat = feat.unsqueeze(0)
        n, Hf, Wf, C = feat.shape
        hidden = weights[0].shape[0]
        if out is None:
            out = torch.empty_like(feat)
        _check(self._lib.bayer_refine_conv(self._h, _ptr(feat), n, Hf, Wf, C, hidden, *[_ptr(t) for t in weights],
                                           int(precision), _ptr(out), _stream(stream)), "bayer_refine_conv")
        return out

    def multi_stream(self, pairs, search_range=32, interp=INTERP_BILINEAR, end_ns=None, stream=None, schedule=0):
        """pairs: list of dicts with ref, cur (uint16/int16 [H, W] tensors; W a multiple of 16, H even), mv
        (int32 [ceil(H/16), W/16, 2]) and optionally feat, feat_out (float32 [C, Hf, Wf], Wf = W / stride,
        Hf = ceil(H / stride)) and stride.  Returns the schedule the autotuner chose
        (1000 * (plain-load search windows + 2 * global-memory propagation items) + 100 * per-size launches
        + 10 * blocks per strip + order; order 0 as given, 1 largest first, 2 smallest first; staging by
        TMA tiles where a pair allows it unless the thousands say otherwise).  ``schedule``: 0 lets the
        autotuner choose; a code runs that schedule."""
        import torch
        arr = (PairDesc * len(pairs))()
        for i, q in enumerate(pairs):
            H, W = q["ref"].shape[-2:]
            d = arr[i]
            d.ref, d.cur, d.W, d.H, d.pitch = q["ref"].data_ptr(), q["cur"].data_ptr(), W, H, W
            h, w = grid_shape(H, W, 16)
            _check_out(q["mv"], h * w * 2, torch.int32, q["ref"].device, "multi_stream")
            d.mv_out = q["mv"].data_ptr()
            if q.get("feat") is not None:
                C, Hf, Wf = q["feat"].shape[-3:]
                d.feat, d.feat_out = q["feat"].data_ptr(), q["feat_out"].data_ptr()
                d.C, d.Hf, d.Wf, d.stride = C, Hf, Wf, q.get("stride", 8)
        sched = ctypes.c_int(int(schedule))
        _check(self._lib.bayer_me_multi_stream(self._h, arr, len(pairs), search_range, interp, _ptr(end_ns),
                                               ctypes.byref(sched), _stream(stream)), "bayer_me_multi_stream")
        return sched.value

    def selftest_wait(self, arrive: bool, limit: int = 1000, stream=None):
        """Run the device's bounded-wait path (see the header); read the outcome with sync_status()."""
        _check(self._lib.bayer_me_selftest_wait(self._h, int(arrive), int(limit), _stream(stream)),
               "bayer_me_selftest_wait")

    def debug_fail_allocs(self, n: int):
        """Test hook: the next n workspace growths report ERR_OOM."""
        _check(self._lib.bayer_me_debug_fail_allocs(self._h, int(n)), "bayer_me_debug_fail_allocs")

    def sync_status(self, stream=None) -> int:
        return int(self._lib.bayer_me_sync_status(self._h, _stream(stream)))

    def probe_alu(self, variant: int = 0):
        """(pixel-candidates per clock per SM, SM MHz during the probe, SM count)."""
        a, b, c = ctypes.c_double(), ctypes.c_double(), ctypes.c_int()
        _check(self._lib.bayer_probe_alu(self._h, variant, ctypes.byref(a), ctypes.byref(b), ctypes.byref(c)),
               "bayer_probe_alu")
        return a.value, b.value, c.value


def estimate_c2f_noalloc(ref, cur, c2f=None, phase=PHASE_EVEN, batch=1, ref_batch_stride=0, cur_batch_stride=0,
                         out=None, stream=None, W=None, H=None, pitch=None):
    """Coarse-to-fine search without any device allocation (no handle): the
    intermediate pyramid fields use the library's static 1 MiB device scratch.
    For callers that must not allocate after start-up.  ``out`` must be given
    by such callers (allocating it here would defeat the purpose); it is only
    created when omitted, for convenience in tests.  Calls that overlap on the
    GPU share the scratch and must be serialised.  The C entry point launches
    on the current device, so this wrapper makes ``ref``'s device current for
    the call; ``cur`` and ``out`` must be on that device too."""
    import torch
    lib = load()
    if cur.device != ref.device:
        raise ValueError("estimate_c2f_noalloc: ref and cur must be on the same device")
    if H is None or W is None:
        H, W = ref.shape[-2:]
    if pitch is None:
        pitch = W
    c2f = c2f or C2FSetting()
    p = Params()
    p.mode, p.phase = MODE_C2F, phase
    p.n_levels = len(c2f.levels)
    for i, b in enumerate(c2f.levels):
        p.levels[i] = b
    p.n_stages = len(c2f.stages)
    for i, (r, s) in enumerate(c2f.stages):
        p.stage_radius[i] = r
        p.stage_step[i] = s
    p.batch, p.ref_batch_stride, p.cur_batch_stride = batch, ref_batch_stride, cur_batch_stride
    h, w = grid_shape(H, W, c2f.levels[-1])
    if out is None:
        out = torch.empty((batch, h, w, 2), dtype=torch.int32, device=ref.device)
    _check_out(out, batch * h * w * 2, torch.int32, ref.device, "estimate_c2f_noalloc")
    with torch.cuda.device(ref.device):
        _check(lib.bayer_me_estimate_c2f_noalloc(_ptr(ref), _ptr(cur), W, H, pitch, ctypes.byref(p), _ptr(out),
                                                 _stream(stream)), "bayer_me_estimate_c2f_noalloc")
    return out


def to_bf16_bits(w32):
    """float32 tensor -> bfloat16 tensor viewed as int16 (the layout the C ABI takes as uint16_t)."""
    import torch
    return w32.to(torch.bfloat16).view(torch.int16)


def init(device: int = 0) -> Handle:
    return Handle(device)


def records_to_numpy(t) -> np.ndarray:
    """int32 [..., 2] record tensor -> numpy structured MV_DTYPE array [...]."""
    a = t.detach().cpu().contiguous().numpy()
    return a.view(MV_DTYPE).reshape(a.shape[:-1])
