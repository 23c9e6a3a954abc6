"""Benchmark: 1080p Bayer block ME + MV feature propagation, frames/s.

One step = the whole hot path over one 8-frame 1920x1088 RGGB clip (12-bit
values in uint16): exhaustive block matching (block 16, +-32, EVEN phase) of
the 7 consecutive pairs in one launch, then bilinear propagation of each
pair's 256 x 136 x 240 float32 reference feature map (stride 8) by its MV
field in one launch.  A "frame" is one processed pair, so a step is 7 frames.

Inputs are synthetic (seeded scene generator + N(0,1) feature maps) and
resident in HBM when the timed region starts; one step reads 267 MB of inputs
(8 frames, 7 feature maps) and writes 234 MB, larger than the 126 MB L2, so no
flush is needed between steps.

  python bench.py [--gpus N] [--steps K] [--warmup W] [--impl ours|reference]

Beside the headline, the same JSON line carries (single-GPU runs; ``--no-legs``
skips them):
  * learned_seeded: the same clip through the proposal network, the +-4
    refine and the exhaustive fallback, with fallback rate and SAD regret;
  * multi_stream: 32 streams of mixed sizes (8x 640x480, 8x 1280x720,
    12x 1920x1088, 4x 3840x2160), one pair of each per step in one search
    launch and one propagation launch replayed from a CUDA graph, with p50/p99
    per-frame latency;
  * precision_4k: a 3840x2160 clip, 128-channel stride-4 propagation and the
    three 3x3 refine convs in BF16 on the tensor cores (FP32 run beside it);
  * c2f: the paper's coarse-to-fine pyramid presets (standard, modes 1-4) on
    the same clip, EVEN phase, search alone and search + propagation.

Under torchrun (N > 1) every rank runs an independent replica on its own GPU
(the path shards into independent clips; no collective on the data path) and
rank 0 prints the aggregate.  ``--impl reference`` times the CPU oracle on
this host's cores on a bounded sample of the same workload.
"""
from __future__ import annotations

import argparse
import json
import os
import statistics
import subprocess
import sys
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

METRIC = "1080p Bayer ME+propagation frames/s, plain vs learned-seeded at <=1% SAD regret"
UNIT = "frames/s"
W, H, T = 1920, 1088, 8
BLOCK, RANGE = 16, 32
C, HF, WF, STRIDE = 256, 136, 240, 8
SEED = 1001
PAIRS = T - 1
WORKLOAD = ("1080p clip: 8 frames 1920x1088 RGGB uint16 12-bit; block 16, +-32 EVEN exhaustive search "
            "(1089 candidates); bilinear propagation of 256x136x240 float32 features at stride 8")


def pc_per_pair() -> int:
    """Pixel-candidates of one pair: blocks x pixels per block x candidates."""
    return (H // BLOCK) * (W // BLOCK) * BLOCK * BLOCK * (RANGE + 1) ** 2


def prop_bytes_per_pair() -> int:
    """Algorithmic propagation bytes of one pair: map read once + written once + MV field."""
    return 2 * C * HF * WF * 4 + (H // BLOCK) * (W // BLOCK) * 8


def bench_config(world: int) -> dict:
    """The workload both arms name (the reference arm times a bounded sample of it)."""
    return {"workload": WORKLOAD, "pairs_per_step": PAIRS, "search": "plain exhaustive",
            "l2": "inputs larger than L2 (267 MB read + 234 MB written per step); no flush",
            "parallelism": f"replicas x{world} (independent clips, no collective)"}


ME_SOURCES = ("paper_2508_05990_b300/csrc/me_full16.cu", "paper_2508_05990_b300/csrc/full16.cuh",
              "paper_2508_05990_b300/csrc/common.cuh", "paper_2508_05990_b300/csrc/tma.cuh",
              "paper_2508_05990_b300/csrc/tc_common.cuh")
PROP_SOURCES = ("paper_2508_05990_b300/csrc/propagate.cu", "paper_2508_05990_b300/csrc/prop_tma.cuh",
                "paper_2508_05990_b300/csrc/prop_common.cuh",
                "paper_2508_05990_b300/csrc/common.cuh", "paper_2508_05990_b300/csrc/tma.cuh",
                "paper_2508_05990_b300/csrc/tc_common.cuh")


def profiled_traffic(summary: str, sources) -> int | None:
    """DRAM bytes per launch (dram__bytes_read.sum + dram__bytes_write.sum) from an ncu
    summary under profiles/, or None once the kernel's source differs from the one the
    counters were taken on (the summary records a hash of it)."""
    import hashlib
    import re
    try:
        text = open(os.path.join(ROOT, "profiles", summary)).read()
        blob = b"".join(open(os.path.join(ROOT, f), "rb").read() for f in sources)
    except OSError:
        return None
    m_sha = re.search(r"source_sha256_16:\s*([0-9a-f]{16})", text)
    m_bytes = re.search(r"traffic_bytes_per_launch:\s*(\d+)", text)
    if not m_sha or not m_bytes or m_sha.group(1) != hashlib.sha256(blob).hexdigest()[:16]:
        return None
    return int(m_bytes.group(1))


WEIGHTS = os.path.join(ROOT, "paper_2508_05990_b300", "weights", "proposal_1080p_r32.npz")
# the same network trained on exactly the 2,000 pairs of the learned-proposal workload
WEIGHTS_2000 = os.path.join(ROOT, "paper_2508_05990_b300", "weights", "proposal_1080p_r32_2000pairs.npz")

# batched multi-stream workload: 32 streams of mixed sizes, 16 frames each
MS_SIZES = [(480, 640)] * 8 + [(720, 1280)] * 8 + [(1088, 1920)] * 12 + [(2160, 3840)] * 4
MS_FRAMES, MS_C, MS_STRIDE = 16, 256, 8
MS_SEED = 1004
# precision form at 4K: 8-frame clip, propagation of 128-channel stride-4 maps, refine convs
K4_H, K4_W, K4_T = 2160, 3840, 8
K4_C, K4_HIDDEN, K4_STRIDE = 128, 64, 4
K4_SEED = 1002


def _gen_clip(task):
    """Pool worker: one synthetic clip (seed, H, W, n_frames)."""
    from paper_2508_05990_b300 import synth
    seed, h, w, n = task
    return synth.pan_clip(seed, h, w, n_frames=n)


def gen_clips(tasks, workers=None):
    """Clips generated in parallel by a spawn-started pool (safe beside an open CUDA context)."""
    import multiprocessing as mp
    from concurrent.futures import ProcessPoolExecutor
    workers = workers or min(len(tasks), os.cpu_count() or 1)
    # a worker that dies raises BrokenProcessPool here instead of blocking
    with ProcessPoolExecutor(workers, mp_context=mp.get_context("spawn")) as ex:
        return list(ex.map(_gen_clip, tasks))


def ms_pc_per_step() -> int:
    """Pixel-candidates of one multi-stream step (one pair of every stream)."""
    return sum((hh // BLOCK) * (ww // BLOCK) for hh, ww in MS_SIZES) * BLOCK * BLOCK * (RANGE + 1) ** 2


def ms_prop_bytes_per_step() -> int:
    return sum(2 * MS_C * (hh // MS_STRIDE) * (ww // MS_STRIDE) * 4 + (hh // BLOCK) * (ww // BLOCK) * 8
               for hh, ww in MS_SIZES)


def ms_launches_per_step(sched: int) -> int:
    """Kernel launches of one multi-stream call under schedule code `sched`: a
    search and a propagation launch per class of frame size (the library's rule:
    runs of equal sizes, smallest first, merged until a class holds an eighth of
    the search strips; at most 8), or one of each; then the end-time kernel and
    the scatter of the end times."""
    base = sched % 1000
    if base < 100:
        return 2 + 2
    nw = base % 100 // 10
    sizes = sorted(MS_SIZES, key=lambda hw: hw[0] * hw[1])
    strips = [(hh // BLOCK) * (-(-(ww // BLOCK) // nw)) for hh, ww in sizes]
    min_items = -(-sum(strips) // 8)
    classes, acc = 0, 0
    for k, st in enumerate(strips):
        acc += st
        last = k + 1 == len(strips)
        if last or (sizes[k + 1] != sizes[k] and (acc >= min_items and classes < 7)):
            classes += 1
            acc = 0
    return 2 * classes + 2


def refine_flops_per_frame() -> int:
    """Multiply-adds x 2 of the three 3x3 refine convs (C -> hidden -> hidden -> C) on one map."""
    hf, wf = K4_H // K4_STRIDE, K4_W // K4_STRIDE
    return 2 * hf * wf * 9 * (K4_C * K4_HIDDEN + K4_HIDDEN * K4_HIDDEN + K4_HIDDEN * K4_C)


def dist_env():
    return int(os.environ.get("RANK", 0)), int(os.environ.get("WORLD_SIZE", 1)), int(os.environ.get("LOCAL_RANK", 0))


def init_dist(backend: str):
    rank, world, local = dist_env()
    if world > 1:
        import torch.distributed as dist
        os.environ.setdefault("MASTER_ADDR", "127.0.0.1")
        dist.init_process_group(backend=backend)
    return rank, world, local


def max_over_ranks(x: float, world: int, device=None) -> float:
    if world == 1:
        return x
    import torch
    import torch.distributed as dist
    t = torch.tensor([x], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def barrier(world: int):
    if world > 1:
        import torch.distributed as dist
        dist.barrier()


def make_inputs(rank: int):
    from paper_2508_05990_b300 import synth
    frames = synth.pan_clip(SEED + 1000 * rank, H, W, n_frames=T)
    feats = synth.features(SEED + 1000 * rank + 1, C, HF, WF, n=PAIRS)
    return frames, feats


class ClockSampler:
    """nvidia-smi samples of SM clock and throttle reasons while running."""
    Q = ("timestamp,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,clocks_event_reasons.hw_slowdown,"
         "clocks_event_reasons.hw_thermal_slowdown,clocks_event_reasons.sw_thermal_slowdown,"
         "clocks_event_reasons.sw_power_cap")

    def __init__(self, index: int):
        self.index = index
        self.proc = None

    def __enter__(self):
        try:
            self.proc = subprocess.Popen(["nvidia-smi", f"--query-gpu={self.Q}", "--format=csv,noheader,nounits",
                                          "-lms", "20", "-i", str(self.index)], stdout=subprocess.PIPE,
                                         stderr=subprocess.DEVNULL, text=True)
        except OSError:
            self.proc = None
        return self

    def __exit__(self, *exc):
        self.lines = []
        if self.proc is not None:
            self.proc.terminate()
            try:
                out, _ = self.proc.communicate(timeout=5)
            except subprocess.TimeoutExpired:
                self.proc.kill()
                out, _ = self.proc.communicate()
            self.lines = [l for l in out.splitlines() if l.strip()]

    def summary(self, t0=None, t1=None):
        """Median SM clock and active throttle reasons over the samples taken
        between host times t0 and t1 (all samples if none fall inside)."""
        import datetime
        parsed = []
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for l in self.lines:
            f = [x.strip() for x in l.split(",")]
            if len(f) < 9:
                continue
            try:
                ts = datetime.datetime.strptime(f[0], "%Y/%m/%d %H:%M:%S.%f").timestamp()
                sm, mx = float(f[1]), float(f[2])
            except ValueError:
                continue
            reasons = {n for n, v in zip(names, f[5:9]) if v.lower().startswith("active")}
            parsed.append((ts, sm, mx, reasons))
        inside = [p for p in parsed if t0 is not None and t0 - 0.05 <= p[0] <= t1 + 0.05]
        use = inside or parsed
        if not use:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["unsampled"], "samples": 0}
        return {"sm_mhz": statistics.median(p[1] for p in use), "sm_max_mhz": max(p[2] for p in use),
                "reasons": sorted(set().union(*(p[3] for p in use))), "samples": len(use),
                "window": "timed region" if inside else "whole run"}


class NvmlClockSampler:
    """SM clock and clock-event (throttle) reasons read through NVML every
    ~0.5 ms from a host thread, so that even a timed region of ~10 ms gets tens
    of samples (nvidia-smi's loop samples every 20 ms at best).  NVML is the
    driver's libnvidia-ml.so.1, called through ctypes.  Each sample is (host
    time, SM MHz, max SM MHz, set of active reasons)."""
    # nvmlClocksEventReason* bits (nvml.h)
    REASONS = (("sw_power_cap", 0x4), ("hw_slowdown", 0x8), ("sw_thermal_slowdown", 0x20),
               ("hw_thermal_slowdown", 0x40))
    NVML_CLOCK_SM = 1

    def __init__(self, index: int, period_s: float = 5e-4):
        self.index, self.period = index, period_s
        self.samples, self.ok, self.error = [], False, None

    def __enter__(self):
        import ctypes
        import threading
        try:
            lib = ctypes.CDLL("libnvidia-ml.so.1")
            if lib.nvmlInit_v2() != 0:
                raise OSError("nvmlInit_v2 failed")
            self._lib = lib
            self._h = ctypes.c_void_p()
            if lib.nvmlDeviceGetHandleByIndex_v2(ctypes.c_uint(self.index), ctypes.byref(self._h)) != 0:
                raise OSError("nvmlDeviceGetHandleByIndex_v2 failed")
            mx = ctypes.c_uint()
            if lib.nvmlDeviceGetMaxClockInfo(self._h, self.NVML_CLOCK_SM, ctypes.byref(mx)) != 0:
                raise OSError("nvmlDeviceGetMaxClockInfo failed")
            self._max = float(mx.value)
            self._reasons = getattr(lib, "nvmlDeviceGetCurrentClocksEventReasons", None) or \
                lib.nvmlDeviceGetCurrentClocksThrottleReasons
            self.ok = True
        except (OSError, AttributeError) as e:  # no NVML: the nvidia-smi sampler stands alone
            self.error = str(e)
            return self
        self._stop = threading.Event()
        self._thr = threading.Thread(target=self._run, daemon=True)
        self._thr.start()
        return self

    def _run(self):
        import ctypes
        clk, r = ctypes.c_uint(), ctypes.c_ulonglong()
        while not self._stop.is_set():
            if (self._lib.nvmlDeviceGetClockInfo(self._h, self.NVML_CLOCK_SM, ctypes.byref(clk)) != 0
                    or self._reasons(self._h, ctypes.byref(r)) != 0):
                self.error = "NVML query failed"
                break
            self.samples.append((time.time(), float(clk.value), self._max,
                                 {n for n, b in self.REASONS if r.value & b}))
            time.sleep(self.period)

    def __exit__(self, *exc):
        if self.ok:
            self._stop.set()
            self._thr.join(timeout=2)
            self._lib.nvmlShutdown()

    def summary(self, t0, t1):
        use = [p for p in self.samples if t0 <= p[0] <= t1]
        if not use:
            return None
        return {"sm_mhz": statistics.median(p[1] for p in use), "sm_max_mhz": max(p[2] for p in use),
                "reasons": sorted(set().union(*(p[3] for p in use))), "samples": len(use),
                "window": "timed region", "source": "NVML, ~0.5 ms apart"}


def pcie_link(nbytes=256 << 20, reps=5):
    """Host <-> device copy bandwidth of this machine with pinned buffers: each
    direction alone and both at once (two streams), GB/s."""
    import torch
    h_a = torch.empty(nbytes, dtype=torch.uint8).pin_memory()
    h_b = torch.empty(nbytes, dtype=torch.uint8).pin_memory()
    d_a = torch.empty(nbytes, dtype=torch.uint8, device="cuda")
    d_b = torch.empty(nbytes, dtype=torch.uint8, device="cuda")
    s_up, s_down = torch.cuda.Stream(), torch.cuda.Stream()

    def timed(fn):
        fn()
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        for _ in range(reps):
            fn()
        torch.cuda.synchronize()
        return (time.perf_counter() - t0) / reps

    def both():
        with torch.cuda.stream(s_up):
            d_a.copy_(h_a, non_blocking=True)
        with torch.cuda.stream(s_down):
            h_b.copy_(d_b, non_blocking=True)

    up = timed(lambda: d_a.copy_(h_a, non_blocking=True))
    down = timed(lambda: h_a.copy_(d_a, non_blocking=True))
    bi = timed(both)
    return {"h2d_gbs": round(nbytes / up / 1e9, 1), "d2h_gbs": round(nbytes / down / 1e9, 1),
            "bidirectional_gbs": round(2 * nbytes / bi / 1e9, 1)}


def cpu_model() -> str:
    try:
        with open("/proc/cpuinfo") as f:
            for line in f:
                if line.startswith("model name"):
                    return line.split(":", 1)[1].strip()
    except OSError:
        pass
    return "unknown"


def cpu_baseline_sample(frames, feats, repeats=3):
    """The oracle as it stands on this host's cores: exhaustive search + bilinear
    warp of one pair per step, a warm-up pair then ``repeats`` timed pairs, once
    with every host thread and once with one thread."""
    import oracle
    oracle.build()
    all_threads = oracle.get_threads()

    def rate(threads):
        oracle.set_threads(threads)
        for k in range(repeats + 1):
            if k == 1:
                t0 = time.perf_counter()
            field, _ = oracle.me_full(frames[k % PAIRS], frames[k % PAIRS + 1], BLOCK, RANGE, even=True)
            oracle.propagate(feats[k % PAIRS], field, BLOCK, STRIDE, interp=oracle.BILINEAR)
        return repeats / (time.perf_counter() - t0)

    v_all = rate(all_threads)
    v_one = rate(1)
    oracle.set_threads(all_threads)
    return {"value": round(v_all, 4), "unit": UNIT, "cores": all_threads, "kind": "oracle",
            "value_1_thread": round(v_one, 4), "nproc": os.cpu_count(), "cpu_model": cpu_model(),
            "sample": f"1080p clip, one pair (full +-32 ME + bilinear propagation) per step: a warm-up pair, then "
                      f"{repeats} timed pairs, at all {all_threads} oracle threads (value) and at 1 thread"}


def leg_multi_stream(h, clips, steps, warmup, peaks, pc_clk_sm, nsm, sm_mhz):
    """32 streams of mixed sizes: each step searches one (t, t+1) pair of every
    stream and propagates its stride-8 256-channel map, all in one search
    launch + one propagation launch replayed from a CUDA graph.  Per-pair
    completion times (device global timer, from the step's first CTA) give the
    latency percentiles.  The same pairs issued as separate per-stream calls
    (one search + one propagation launch each) are timed beside it."""
    import torch
    from paper_2508_05990_b300 import bayer_me as bm
    stream = torch.cuda.current_stream()
    gen = torch.Generator(device="cuda")
    gen.manual_seed(MS_SEED)
    d_clips = [torch.from_numpy(c).cuda() for c in clips]
    feats, outs, mvs = [], [], []
    for hh, ww in MS_SIZES:
        feats.append(torch.randn((MS_C, hh // MS_STRIDE, ww // MS_STRIDE), generator=gen, device="cuda"))
        outs.append(torch.empty_like(feats[-1]))
        mvs.append(torch.empty((hh // BLOCK, ww // BLOCK, 2), dtype=torch.int32, device="cuda"))
    n = len(MS_SIZES)

    def pairs(t):
        return [{"ref": d_clips[i][t], "cur": d_clips[i][t + 1], "mv": mvs[i], "feat": feats[i],
                 "feat_out": outs[i], "stride": MS_STRIDE} for i in range(n)]

    tables = [pairs(t) for t in range(MS_FRAMES - 1)]
    end = torch.zeros((steps, n), dtype=torch.int64, device="cuda")
    sched = 0
    for k in range(warmup):
        sched = h.multi_stream(tables[k % len(tables)], RANGE, end_ns=end[0])
    torch.cuda.synchronize()
    if h.sync_status() != bm.OK:
        raise RuntimeError("device status after multi-stream warm-up")
    start, stop = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    start.record(stream)
    for k in range(steps):
        h.multi_stream(tables[k % len(tables)], RANGE, end_ns=end[k])
    stop.record(stream)
    torch.cuda.synchronize()
    ms = start.elapsed_time(stop)
    lat_ms = end.cpu().numpy().astype(np.float64).ravel() / 1e6

    # the same work as separate calls per stream
    sep_steps = max(3, steps // 4)

    def separate(t):
        for i in range(n):
            q = tables[t][i]
            h.estimate(q["ref"], q["cur"], BLOCK, RANGE, out=mvs[i], stream=stream)
            h.feat_propagate(feats[i], mvs[i], BLOCK, MS_STRIDE, interp=bm.INTERP_BILINEAR, out=outs[i],
                             stream=stream)

    separate(0)
    torch.cuda.synchronize()
    start.record(stream)
    for k in range(sep_steps):
        separate(k % len(tables))
    stop.record(stream)
    torch.cuda.synchronize()
    ms_sep = start.elapsed_time(stop) / sep_steps
    if h.sync_status() != bm.OK:
        raise RuntimeError("device status after multi-stream leg")

    step_ms = ms / steps
    t_alu = ms_pc_per_step() / (pc_clk_sm * nsm * sm_mhz * 1e6) * 1e3
    t_hbm = ms_prop_bytes_per_step() / (peaks.get("hbm_gbs", 6400.0) * 1e9) * 1e3
    return {
        "workload": "32 streams (8x 640x480, 8x 1280x720, 12x 1920x1088, 4x 3840x2160), 16 frames each; "
                    "block 16 +-32 EVEN exhaustive; bilinear propagation of 256-channel stride-8 maps",
        "value": round(n * steps / (ms / 1e3), 2), "unit": UNIT, "steps": steps, "warmup": warmup,
        "ms_per_step": round(step_ms, 4), "frames_per_step": n,
        "latency_ms": {"p50": round(float(np.percentile(lat_ms, 50)), 4),
                       "p99": round(float(np.percentile(lat_ms, 99)), 4),
                       "max": round(float(lat_ms.max()), 4),
                       "definition": "first CTA of the step's search launch -> pair's propagated map written"},
        "schedule": {"code": sched, "blocks_per_strip": sched % 100 // 10,
                     "order": {0: "stream order", 1: "largest first", 2: "smallest first"}[sched % 10],
                     "launches": "per frame size, smallest first: search then propagation" if sched % 1000 >= 100
                     else "one search + one propagation launch",
                     "search_windows": "plain loads" if (sched // 1000) & 1 else "TMA tiles",
                     "propagation": "global-memory items" if (sched // 1000) & 2 else "TMA-staged tiles",
                     "picked_by": "autotuner (timed graph replays of each candidate)"},
        "separate_launches": {"ms_per_step": round(ms_sep, 4), "launches_per_step": 2 * n,
                              "speedup_of_batched": round(ms_sep / step_ms, 3)},
        "roofline": {"bound": "alu+hbm", "ideal_ms": round(t_alu + t_hbm, 4), "frac": round((t_alu + t_hbm) / step_ms, 4),
                     "alu_ms": round(t_alu, 4), "hbm_ms": round(t_hbm, 4),
                     "algorithmic_per_step": f"{ms_pc_per_step()} pixel-candidates + {ms_prop_bytes_per_step()} "
                                             "propagation bytes",
                     "peak_source": "measured packed min.u16x2 + dp2a rate x SMs x median SM clock; " + (
                         "MEASURED_PEAKS.json hbm_gbs (of measured)" if "hbm_gbs" in peaks
                         else "fallback 6400 GB/s (MEASURED_PEAKS.json absent)")},
        "gpu_launches": ms_launches_per_step(sched) * steps,
        "l2": "inputs larger than L2 (2.2 GB of feature maps per step); no flush",
    }


def leg_c2f(h, d_frames, d_feats, d_out, stream, steps, warmup, pc_clk_sm, nsm, sm_mhz, full_me_ms, full_step_ms):
    """The paper's FME presets (coarse-to-fine pyramid) on the 1080p clip, EVEN
    phase, 7 pairs per launch, and the standard pyramid in the RAW phase (the
    paper's step-1 fine stage taken literally): the search alone and the search
    plus bilinear propagation of the same feature maps at the last level's block
    size, beside the exhaustive +-32 search of the plain step."""
    import torch
    from paper_2508_05990_b300 import bayer_me as bm
    peak = pc_clk_sm * nsm * sm_mhz * 1e6
    kw = dict(batch=PAIRS, ref_batch_stride=H * W, cur_batch_stride=H * W)
    rows = {}
    launches = 0
    runs = [(name, setting, bm.PHASE_EVEN) for name, setting in bm.C2F_PRESETS.items()]
    runs.append(("raw_standard", bm.C2F_PRESETS["standard"], bm.PHASE_RAW))
    for name, setting, phase in runs:
        B = setting.levels[-1]
        mv = torch.empty((PAIRS, -(-H // B), -(-W // B), 2), dtype=torch.int32, device="cuda")

        def me():
            h.estimate_ex(d_frames, d_frames[1:], mode=bm.MODE_C2F, phase=phase, c2f=setting, out=mv,
                          stream=stream, **kw)

        def step():
            me()
            h.feat_propagate(d_feats, mv, B, STRIDE, interp=bm.INTERP_BILINEAR, out=d_out, stream=stream)

        res = {}
        for label, fn in (("me", me), ("step", step)):
            for _ in range(warmup):
                fn()
            torch.cuda.synchronize()
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            e0.record(stream)
            for _ in range(steps):
                fn()
            e1.record(stream)
            torch.cuda.synchronize()
            res[label] = e0.elapsed_time(e1) / steps
        if h.sync_status() != bm.OK:
            raise RuntimeError("device status after the C2F leg")
        pc = PAIRS * bm.c2f_pixel_candidates(setting, H, W, even=phase == bm.PHASE_EVEN)
        launches += steps * (2 * len(setting.levels) + 1)  # the search's levels, then levels + propagation
        rows[name] = {"phase": "EVEN" if phase == bm.PHASE_EVEN else "RAW",
                      "levels": list(setting.levels), "stages": [list(x) for x in setting.stages],
                      "me_ms": round(res["me"], 4), "ms_per_step": round(res["step"], 4),
                      "value": round(PAIRS / (res["step"] / 1e3), 2), "unit": UNIT,
                      "pixel_candidates_per_launch": pc,
                      "achieved_gpc_per_s": round(pc / (res["me"] / 1e3) / 1e9, 1),
                      "frac_of_alu_peak": round(pc / (res["me"] / 1e3) / peak, 4),
                      "me_vs_full_search": round(full_me_ms / res["me"], 3),
                      "step_vs_plain_step": round(full_step_ms / res["step"], 3)}
    return {"workload": "1080p clip (7 pairs per launch), EVEN phase, and the standard pyramid in the RAW phase; "
                        "levels are block sizes, stages (radius in steps, step); propagation of the plain step's "
                        "feature maps at the last level's block size",
            "presets": rows, "steps": steps, "warmup": warmup,
            "peak_source": "measured packed min.u16x2 + dp2a rate x SMs x median SM clock",
            "gpu_launches": launches}


RAGGED_SEED = 1005


def c2f_pc_in_frame(setting, Hh: int, Ww: int) -> int:
    """Pixel-candidates of one pair's EVEN pyramid counting only pixels inside
    the frame (a clipped block row has fewer): every pixel lies in one block
    per level, so each level costs H * W * sum over stages of (2R+1)^2."""
    per = 0
    for R, st in setting.stages:
        if st % 2:
            R, st = R * st // (st + 1), st + 1
        per += (2 * R + 1) ** 2
    return len(setting.levels) * Hh * Ww * per


def leg_ragged(h, steps, warmup, peak_gpcs):
    """Frames whose height is not a multiple of the block: the real 1920x1080
    frame (exhaustive block 16 +-32, its last block row 8 rows high) beside the
    1920x1088 workload, and the paper's 720x960 runtime resolution (standard
    pyramid, EVEN; 720 is no multiple of 64 or 32) beside 768x960.  Seven pairs
    per launch, search alone; G pixel-candidates/s count in-frame pixels.  With
    the shipped proposal weights, also the learned-seeded search (network, +-4
    refine, fallback) on 1920x1080 beside 1920x1088."""
    import torch
    from paper_2508_05990_b300 import bayer_me as bm
    from paper_2508_05990_b300 import synth
    std = bm.C2F_PRESETS["standard"]
    out = {}
    wbf = None
    if os.path.exists(WEIGHTS):
        wbf = bm.to_bf16_bits(torch.from_numpy(np.load(WEIGHTS)["theta"].astype(np.float32)).cuda()).contiguous()
    for name, Hh, Ww, mode in (("full_1920x1080", 1080, 1920, bm.MODE_FULL), ("full_1920x1088", 1088, 1920, bm.MODE_FULL),
                               ("c2f_standard_720x960", 720, 960, bm.MODE_C2F),
                               ("c2f_standard_768x960", 768, 960, bm.MODE_C2F)):
        frames = torch.from_numpy(synth.pan_clip(RAGGED_SEED, Hh, Ww, n_frames=T)).cuda()
        B = std.levels[-1] if mode == bm.MODE_C2F else BLOCK
        mv = torch.empty((PAIRS, -(-Hh // B), -(-Ww // B), 2), dtype=torch.int32, device="cuda")
        kw = dict(batch=PAIRS, ref_batch_stride=Hh * Ww, cur_batch_stride=Hh * Ww, out=mv)
        run = (lambda: h.estimate_ex(frames, frames[1:], search_range=RANGE, **kw)) if mode == bm.MODE_FULL else \
            (lambda: h.estimate_ex(frames, frames[1:], mode=bm.MODE_C2F, c2f=std, **kw))
        for _ in range(warmup):
            run()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        torch.cuda.synchronize()
        e0.record()
        for _ in range(steps):
            run()
        e1.record()
        torch.cuda.synchronize()
        ms = e0.elapsed_time(e1) / steps
        pc = PAIRS * (Hh * Ww * (2 * (RANGE // 2) + 1) ** 2 if mode == bm.MODE_FULL else c2f_pc_in_frame(std, Hh, Ww))
        out[name] = {"me_ms": round(ms, 4), "frames_per_s": round(PAIRS / (ms / 1e3), 1),
                     "gpc_per_s": round(pc / (ms / 1e3) / 1e9, 1), "frac_of_alu_peak": round(pc / (ms / 1e3) / peak_gpcs, 4)}
    for Hh in ((1080, 1088) if wbf is not None else ()):
        frames = torch.from_numpy(synth.pan_clip(RAGGED_SEED, Hh, 1920, n_frames=T)).cuda()
        mv = torch.empty((PAIRS, -(-Hh // BLOCK), 1920 // BLOCK, 2), dtype=torch.int32, device="cuda")
        nfb = torch.zeros(1, dtype=torch.int32, device="cuda")

        def run():
            h.estimate_learned(frames, frames[1:], wbf, RANGE, 0.5, batch=PAIRS, ref_batch_stride=Hh * 1920,
                               cur_batch_stride=Hh * 1920, out=mv, n_fallback=nfb)
        for _ in range(warmup):
            run()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        torch.cuda.synchronize()
        e0.record()
        for _ in range(steps):
            run()
        e1.record()
        torch.cuda.synchronize()
        ms = e0.elapsed_time(e1) / steps
        out[f"learned_1920x{Hh}"] = {"search_ms": round(ms, 4), "frames_per_s": round(PAIRS / (ms / 1e3), 1),
                                     "fallback_frac": round(int(nfb.item()) / mv[..., 0].numel(), 4)}
    if h.sync_status() != bm.OK:
        raise RuntimeError("device status after the ragged-frame leg")
    out["ratio_1080_vs_1088"] = round(out["full_1920x1080"]["gpc_per_s"] / out["full_1920x1088"]["gpc_per_s"], 4)
    out["ratio_720_vs_768"] = round(out["c2f_standard_720x960"]["gpc_per_s"] / out["c2f_standard_768x960"]["gpc_per_s"],
                                    4)
    out["note"] = ("7 pairs per launch; the paper's standard FME takes 3.36 ms per 720x960 frame on an A100 "
                   "(context, another machine)")
    return out


def leg_refine_4k(h, clip, steps, warmup, peaks):
    """Precision form at 4K: exhaustive search of the 7 pairs, bilinear
    propagation of the 128-channel stride-4 NHWC maps, then the three 3x3 refine
    convs in BF16 on the tensor cores (FP32 accumulation).  The FP32 SIMT run of
    the convs is timed beside it; error against FP64 is a test's job."""
    import torch
    from paper_2508_05990_b300 import bayer_me as bm
    from paper_2508_05990_b300 import synth
    stream = torch.cuda.current_stream()
    pairs = K4_T - 1
    hf, wf = K4_H // K4_STRIDE, K4_W // K4_STRIDE
    d_frames = torch.from_numpy(clip).cuda()
    gen = torch.Generator(device="cuda")
    gen.manual_seed(K4_SEED)
    feats = torch.randn((pairs, hf, wf, K4_C), generator=gen, device="cuda")
    warped = torch.empty_like(feats)
    refined = torch.empty_like(feats)
    theta = synth.he_normal_params(K4_SEED, [("w", (K4_HIDDEN, K4_C, 3, 3)), ("b", (K4_HIDDEN,)),
                                             ("w", (K4_HIDDEN, K4_HIDDEN, 3, 3)), ("b", (K4_HIDDEN,)),
                                             ("w", (K4_C, K4_HIDDEN, 3, 3)), ("b", (K4_C,))])
    shapes = [(K4_HIDDEN, K4_C, 3, 3), (K4_HIDDEN,), (K4_HIDDEN, K4_HIDDEN, 3, 3), (K4_HIDDEN,),
              (K4_C, K4_HIDDEN, 3, 3), (K4_C,)]
    wts, o = [], 0
    for shp in shapes:
        nsz = int(np.prod(shp))
        wts.append(torch.from_numpy(theta[o:o + nsz].astype(np.float32).reshape(shp)).cuda())
        o += nsz
    mv = torch.empty((pairs, K4_H // BLOCK, K4_W // BLOCK, 2), dtype=torch.int32, device="cuda")

    def step(ev=None, prec=bm.PREC_BF16):
        if ev is not None:
            ev[0].record(stream)
        h.estimate_ex(d_frames, d_frames[1:], search_range=RANGE, batch=pairs, ref_batch_stride=K4_H * K4_W,
                      cur_batch_stride=K4_H * K4_W, out=mv, stream=stream)
        if ev is not None:
            ev[1].record(stream)
        h.feat_propagate(feats, mv, BLOCK, K4_STRIDE, interp=bm.INTERP_BILINEAR, layout=bm.LAYOUT_NHWC,
                         out=warped, stream=stream)
        if ev is not None:
            ev[2].record(stream)
        h.refine_conv(warped, wts, precision=prec, out=refined, stream=stream)
        if ev is not None:
            ev[3].record(stream)

    for _ in range(warmup):
        step()
    torch.cuda.synchronize()
    if h.sync_status() != bm.OK:
        raise RuntimeError("device status after 4K warm-up")
    evs = [[torch.cuda.Event(enable_timing=True) for _ in range(4)] for _ in range(steps)]
    for k in range(steps):
        step(evs[k])
    torch.cuda.synchronize()
    me = statistics.mean(e[0].elapsed_time(e[1]) for e in evs)
    pr = statistics.mean(e[1].elapsed_time(e[2]) for e in evs)
    rf = statistics.mean(e[2].elapsed_time(e[3]) for e in evs)
    total = statistics.mean(e[0].elapsed_time(e[3]) for e in evs)
    out_bf16 = refined.clone()
    # FP32 SIMT run of the convs on the same warped maps
    fev = [torch.cuda.Event(enable_timing=True) for _ in range(2)]
    h.refine_conv(warped, wts, precision=bm.PREC_FP32, out=refined, stream=stream)
    fev[0].record(stream)
    h.refine_conv(warped, wts, precision=bm.PREC_FP32, out=refined, stream=stream)
    fev[1].record(stream)
    torch.cuda.synchronize()
    rf32 = fev[0].elapsed_time(fev[1])
    diff = float((out_bf16 - refined).norm() / refined.norm())
    if h.sync_status() != bm.OK:
        raise RuntimeError("device status after 4K leg")
    flops = pairs * refine_flops_per_frame()
    peak = peaks.get("bf16_tflops_sustained", 1400.0)
    t_alu_me = pairs * (K4_H // BLOCK) * (K4_W // BLOCK) * BLOCK * BLOCK * (RANGE + 1) ** 2
    prop_bytes = pairs * (2 * K4_C * hf * wf * 4 + (K4_H // BLOCK) * (K4_W // BLOCK) * 8)
    return {
        "workload": "4K clip: 8 frames 3840x2160 RGGB uint16 12-bit; block 16 +-32 EVEN exhaustive; bilinear "
                    "propagation of 128x540x960 NHWC float32 maps at stride 4; refine convs 128->64->64->128 "
                    "(3x3, ReLU after the first two, He-normal weights)",
        "value": round(pairs / (total / 1e3), 2), "unit": UNIT, "steps": steps, "warmup": warmup,
        "ms_per_step": round(total, 4), "frames_per_step": pairs,
        "me_ms": round(me, 4), "prop_ms": round(pr, 4), "refine_bf16_ms": round(rf, 4),
        "refine_fp32_ms": round(rf32, 4),
        "me_gpc_per_s": round(t_alu_me / (me / 1e3) / 1e9, 1),
        "prop_gbs": round(prop_bytes / (pr / 1e3) / 1e9, 1),
        "roofline": {"bound": "tensor", "kernel": "conv3x3_rows_tc_kernel (3 launches, BF16 operands, FP32 accumulate in TMEM)",
                     "achieved": round(flops / (rf / 1e3) / 1e12, 1), "peak": peak, "unit": "TFLOP/s",
                     "frac": round(flops / (rf / 1e3) / 1e12 / peak, 4),
                     "algorithmic_per_launch_set": f"{flops} FLOP ({pairs} maps x {refine_flops_per_frame()})",
                     "peak_source": ("MEASURED_PEAKS.json bf16_tflops_sustained (of measured)"
                                     if "bf16_tflops_sustained" in peaks
                                     else "fallback 1400 TFLOP/s sustained (MEASURED_PEAKS.json absent)"),
                     "fp32_simt_tflops": round(flops / (rf32 / 1e3) / 1e12, 1)},
        "bf16_vs_fp32_normwise": round(diff, 6),
        # search, propagation, then per refine call three weight packs and three convs
        "gpu_launches": 8 * steps,
    }


def run_ours(args):
    import torch
    rank, world, local = init_dist("nccl")
    torch.cuda.set_device(local)
    from paper_2508_05990_b300 import bayer_me as bm
    from paper_2508_05990_b300 import build
    build.build()

    frames, feats = make_inputs(rank)
    legs = world == 1 and not args.no_legs
    leg_clips = None
    if legs:  # batched multi-stream + 4K clips, generated on the host cores
        tasks = [(MS_SEED + 10 * i, hh, ww, MS_FRAMES) for i, (hh, ww) in enumerate(MS_SIZES)]
        tasks.append((K4_SEED, K4_H, K4_W, K4_T))
        tasks.sort(key=lambda t: -t[1] * t[2])
        got = dict(zip([t[0] for t in tasks], gen_clips(tasks)))
        leg_clips = ([got[MS_SEED + 10 * i] for i in range(len(MS_SIZES))], got[K4_SEED])
    h = bm.Handle(local)
    stream = torch.cuda.current_stream()
    d_frames = torch.from_numpy(frames).cuda()
    d_feats = torch.from_numpy(feats).cuda()
    d_out = torch.empty_like(d_feats)
    hb, wb = H // BLOCK, W // BLOCK
    d_mv = torch.empty((PAIRS, hb, wb, 2), dtype=torch.int32, device="cuda")

    def step(ev=None):
        if ev is not None:
            ev[0].record(stream)
        h.estimate_ex(d_frames, d_frames[1:], search_range=RANGE, batch=PAIRS, ref_batch_stride=H * W,
                      cur_batch_stride=H * W, out=d_mv, stream=stream)
        if ev is not None:
            ev[1].record(stream)
        h.feat_propagate(d_feats, d_mv, BLOCK, STRIDE, interp=bm.INTERP_BILINEAR, out=d_out, stream=stream)
        if ev is not None:
            ev[2].record(stream)

    for _ in range(args.warmup):
        step()
    torch.cuda.synchronize()
    status = h.sync_status()
    if status != bm.OK:
        raise RuntimeError(f"device status {status} after warm-up")

    evs = [[torch.cuda.Event(enable_timing=True) for _ in range(3)] for _ in range(args.steps)]
    start, end = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    barrier(world)
    torch.cuda.synchronize()
    with ClockSampler(local) as clk, NvmlClockSampler(local) as nclk:
        time.sleep(0.5)  # let the samplers start
        t_host0 = time.time()
        start.record(stream)
        for k in range(args.steps):
            step(evs[k])
        end.record(stream)
        torch.cuda.synchronize()
        t_host1 = time.time()
    barrier(world)
    ms_total = start.elapsed_time(end)
    ms_total = max_over_ranks(ms_total, world, device="cuda")
    me_ms = [e[0].elapsed_time(e[1]) for e in evs]
    prop_ms = [e[1].elapsed_time(e[2]) for e in evs]
    gpu_launches = 2 * args.steps

    # learned-seeded form on the same clip: proposal network (tensor cores), +-4
    # refine, exhaustive search of the low-confidence blocks, then propagation
    learned = None
    if os.path.exists(WEIGHTS):
        theta = torch.from_numpy(np.load(WEIGHTS)["theta"].astype(np.float32)).cuda()
        wbf = bm.to_bf16_bits(theta).contiguous()
        d_mv_l = torch.empty_like(d_mv)
        d_fb = torch.empty((PAIRS, hb, wb), dtype=torch.uint8, device="cuda")

        def lstep(ev=None):
            if ev is not None:
                ev[0].record(stream)
            h.estimate_learned(d_frames, d_frames[1:], wbf, RANGE, 0.5, batch=PAIRS, ref_batch_stride=H * W,
                               cur_batch_stride=H * W, out=d_mv_l, fallback=d_fb, stream=stream)
            if ev is not None:
                ev[1].record(stream)
            h.feat_propagate(d_feats, d_mv_l, BLOCK, STRIDE, interp=bm.INTERP_BILINEAR, out=d_out, stream=stream)

        for _ in range(args.warmup):
            lstep()
        torch.cuda.synchronize()
        if h.sync_status() != bm.OK:
            raise RuntimeError("device status after learned warm-up")
        lev = [[torch.cuda.Event(enable_timing=True) for _ in range(2)] for _ in range(args.steps)]
        barrier(world)
        torch.cuda.synchronize()
        start.record(stream)
        for k in range(args.steps):
            lstep(lev[k])
        end.record(stream)
        torch.cuda.synchronize()
        barrier(world)
        ms_l = max_over_ranks(start.elapsed_time(end), world, device="cuda")
        sad_plain = bm.records_to_numpy(d_mv)["sad"].astype(np.int64)
        sad_l = bm.records_to_numpy(d_mv_l)["sad"].astype(np.int64)
        learned = {
            "value": round(world * PAIRS * args.steps / (ms_l / 1e3), 2), "unit": UNIT,
            "ms_per_step": round(ms_l / args.steps, 4),
            "me_avg_ms": round(statistics.mean(e[0].elapsed_time(e[1]) for e in lev), 4),
            "speedup_vs_plain": round(ms_total / ms_l, 3),
            "fallback_rate": round(float(d_fb.float().mean().item()), 4),
            "sad_regret": round(float((sad_l.sum() - sad_plain.sum()) / sad_plain.sum()), 5),
            "mean_block_rel_regret": round(float(((sad_l - sad_plain) / np.maximum(sad_plain, 1)).mean()), 5),
            "search": "proposal CNN (BF16, tcgen05) + +-4 refine; exhaustive +-32 where conf < 0.5",
            "weights": os.path.relpath(WEIGHTS, ROOT) + " (4,000 training pairs)",
            # weight pack, layers 1 and 2, layers 3-4 + head, refine, fallback search, propagation
            "gpu_launches": args.steps * 7,
        }
        if os.path.exists(WEIGHTS_2000):
            # the configured training scale: same clip, same timing
            wbf = bm.to_bf16_bits(torch.from_numpy(np.load(WEIGHTS_2000)["theta"].astype(np.float32)).cuda()).contiguous()
            for _ in range(args.warmup):
                lstep()
            torch.cuda.synchronize()
            start.record(stream)
            for k in range(args.steps):
                lstep()
            end.record(stream)
            torch.cuda.synchronize()
            ms_c = start.elapsed_time(end)
            sad_c = bm.records_to_numpy(d_mv_l)["sad"].astype(np.int64)
            learned["configured_scale"] = {
                "weights": os.path.relpath(WEIGHTS_2000, ROOT) + " (2,000 training pairs)",
                "value": round(PAIRS * args.steps / (ms_c / 1e3), 2), "ms_per_step": round(ms_c / args.steps, 4),
                "fallback_rate": round(float(d_fb.float().mean().item()), 4),
                "sad_regret": round(float((sad_c.sum() - sad_plain.sum()) / sad_plain.sum()), 5)}
        if legs:
            # the network's training step (recipe: batch 16), kernels only
            learned["train_step"] = train_step_timing(h, d_frames, d_mv, steps=10)

    # ALU roofline: measured throughput of the search's primitive (packed min.u16x2 + dp2a, two
    # pixel-candidates per pair) per clock per SM x SMs x SM clock under load; sad.u32 beside it
    pc_clk_sm, probe_mhz, nsm = h.probe_alu(3)
    sad_clk_sm = h.probe_alu(0)[0]
    clocks = nclk.summary(t_host0, t_host1)
    smi = clk.summary(t_host0, t_host1)
    if clocks is None:
        clocks = dict(smi, nvml=nclk.error or "no samples in the timed region")
    else:  # nvidia-smi's reasons too, for the timed region's few 20 ms samples
        clocks["reasons"] = sorted(set(clocks["reasons"]) | set(r for r in smi["reasons"] if r != "unsampled"))
        clocks["nvidia_smi_samples"] = smi["samples"]
    sm_mhz = clocks["sm_mhz"] or probe_mhz
    peaks = {}
    try:
        peaks = json.load(open(os.path.join(ROOT, "MEASURED_PEAKS.json")))
    except (OSError, ValueError):
        pass

    multi_stream = refine_4k = c2f = ragged = None
    if legs:
        c2f = leg_c2f(h, d_frames, d_feats, d_out, stream, steps=10, warmup=3, pc_clk_sm=pc_clk_sm, nsm=nsm,
                      sm_mhz=sm_mhz, full_me_ms=statistics.mean(me_ms), full_step_ms=ms_total / args.steps)
        multi_stream = leg_multi_stream(h, leg_clips[0], steps=30, warmup=3, peaks=peaks, pc_clk_sm=pc_clk_sm,
                                        nsm=nsm, sm_mhz=sm_mhz)
        refine_4k = leg_refine_4k(h, leg_clips[1], steps=10, warmup=3, peaks=peaks)
        ragged = leg_ragged(h, steps=20, warmup=3, peak_gpcs=pc_clk_sm * nsm * sm_mhz * 1e6)
        leg_clips = None
        torch.cuda.empty_cache()

    # end to end through the C ABI with host buffers (pinned), copies inside the timed region
    pin_frames = torch.from_numpy(frames).pin_memory().numpy()
    pin_feats = torch.from_numpy(feats).pin_memory().numpy()
    pin_mv = torch.empty((PAIRS, hb, wb, 2), dtype=torch.int32).pin_memory().numpy().view(bm.MV_DTYPE)
    pin_mv = pin_mv.reshape(PAIRS, hb, wb)
    pin_out = torch.empty(feats.shape, dtype=torch.float32).pin_memory().numpy()
    h.clip_process_host(pin_frames, pin_feats, BLOCK, RANGE, STRIDE, bm.INTERP_BILINEAR, pin_mv, pin_out)
    barrier(world)
    t0 = time.perf_counter()
    for _ in range(args.steps):
        h.clip_process_host(pin_frames, pin_feats, BLOCK, RANGE, STRIDE, bm.INTERP_BILINEAR, pin_mv, pin_out)
    e2e_s = max_over_ranks(time.perf_counter() - t0, world, device="cuda")
    h2d = frames.nbytes + feats.nbytes
    d2h = pin_mv.nbytes + pin_out.nbytes
    link = pcie_link()

    result = None
    if rank == 0:
        me_avg_s = statistics.mean(me_ms) / 1e3
        achieved = PAIRS * pc_per_pair() / me_avg_s / 1e9
        peak = pc_clk_sm * nsm * sm_mhz * 1e6 / 1e9
        prop_avg_s = statistics.mean(prop_ms) / 1e3
        prop_gbs = PAIRS * prop_bytes_per_pair() / prop_avg_s / 1e9
        hbm_peak = peaks.get("hbm_gbs", 6400.0)
        hbm_src = ("MEASURED_PEAKS.json hbm_gbs (of measured)" if "hbm_gbs" in peaks
                   else "fallback 6400 GB/s (MEASURED_PEAKS.json absent)")
        value = world * PAIRS * args.steps / (ms_total / 1e3)
        result = {
            "metric": METRIC, "value": round(value, 2), "unit": UNIT, "n_gpus": world, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": round(ms_total / args.steps, 4), "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "u16 frames (packed 16x2 min), u32 SAD, f32 features",
            "data": "synthetic (seeded pan+rectangles Bayer clip, N(0,1) features)",
            "config": bench_config(world),
            "roofline": {"bound": "alu", "kernel": "me_full16_even_kernel<16>", "achieved": round(achieved, 1),
                         "peak": round(peak, 1), "unit": "G pixel-candidates/s", "frac": round(achieved / peak, 4),
                         "clock_samples": clocks.get("samples"),
                         "peak_source": f"measured packed min.u16x2 + dp2a loop: {pc_clk_sm:.1f} pc/clk/SM x {nsm} "
                                        f"SMs x {sm_mhz:.0f} MHz (median SM clock under load); sad.u32 loop "
                                        f"{sad_clk_sm:.1f} pc/clk/SM",
                         "traffic": profiled_traffic("me_full16_even_1080p_clip.md", ME_SOURCES),
                         "traffic_unit": "DRAM bytes per launch (ncu)",
                         "algorithmic_per_launch": f"{PAIRS * pc_per_pair()} pixel-candidates",
                         "avg_launch_ms": round(me_avg_s * 1e3, 4)},
            "propagation": {"bound": "hbm", "achieved": round(prop_gbs, 1), "peak": hbm_peak, "unit": "GB/s",
                            "frac": round(prop_gbs / hbm_peak, 4), "avg_launch_ms": round(prop_avg_s * 1e3, 4),
                            "traffic": profiled_traffic("prop_nchw_bilinear_1080p_clip.md", PROP_SOURCES),
                            "algorithmic_bytes_per_launch": PAIRS * prop_bytes_per_pair(),
                            "peak_source": hbm_src},
            "mblocks_per_s": round(value * hb * wb / 1e6, 3),
            "e2e": {"value": round(world * PAIRS * args.steps / e2e_s, 2), "unit": UNIT,
                    "h2d_bytes_per_step": int(h2d), "d2h_bytes_per_step": int(d2h),
                    "api": "bayer_clip_process_host (pinned host buffers, 3 streams)",
                    "link": dict(link, frac_of_bidirectional=round((h2d + d2h) * args.steps / e2e_s / 1e9
                                                                   / link["bidirectional_gbs"], 4))},
            "gpu": torch.cuda.get_device_name(local),
            "gpu_launches": gpu_launches,
            "clocks": clocks,
            "multi_stream": multi_stream,
            "precision_4k": refine_4k,
            "c2f": c2f,
            "ragged": ragged,
        }
        if not args.no_cpu_baseline:
            result["cpu_baseline"] = cpu_baseline_sample(frames, feats)
        # the metric's second half last, so that a reader keeping only the end of the line keeps it;
        # within it the headline keys last too
        if learned is not None:
            tail = ("speedup_vs_plain", "fallback_rate", "sad_regret", "value")
            learned = {**{k: v for k, v in learned.items() if k not in tail},
                       **{k: learned[k] for k in tail if k in learned}}
        result["learned_seeded"] = learned
    h.close()
    if world > 1:
        import torch.distributed as dist
        dist.destroy_process_group()
    return result


def run_reference(args):
    rank, world, _ = dist_env()
    if rank != 0:
        return None
    import oracle
    oracle.build()
    frames, feats = make_inputs(0)

    def step(k):
        t = k % PAIRS
        field, _ = oracle.me_full(frames[t], frames[t + 1], BLOCK, RANGE, even=True)
        oracle.propagate(feats[t], field, BLOCK, STRIDE, interp=oracle.BILINEAR)

    for k in range(args.warmup):
        step(k)
    t0 = time.perf_counter()
    for k in range(args.steps):
        step(k)
    dt = time.perf_counter() - t0
    value = args.steps / dt
    cores = oracle.get_threads()
    return {
        "impl": "reference", "metric": METRIC, "value": round(value, 4), "unit": UNIT, "n_gpus": world,
        "steps": args.steps, "warmup": args.warmup, "ms_per_step": round(dt / args.steps * 1e3, 2),
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "u16 frames, u64 SAD, f32 features",
        "data": "synthetic (seeded pan+rectangles Bayer clip, N(0,1) features)",
        "config": bench_config(world),
        "sample": "each step = 1 pair of the 1080p clip (of 7), CPU oracle",
        "cpu_baseline": {"value": round(value, 4), "unit": UNIT, "cores": cores, "kind": "oracle",
                         "sample": "1 pair per step of the 1080p clip, plain C oracle, all host threads"},
        "e2e": {"value": round(value, 4), "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
    }


def run_refine_only(n_maps: int):
    """The 4K form's refine convolutions alone on n_maps 540 x 960 x 128 NHWC maps
    (He-normal weights, N(0,1) input), three untimed and five timed calls: a small
    case for profiling the tensor-core kernels."""
    import torch
    from paper_2508_05990_b300 import bayer_me as bm
    from paper_2508_05990_b300 import build, synth
    build.build()
    shapes = [(K4_HIDDEN, K4_C, 3, 3), (K4_HIDDEN,), (K4_HIDDEN, K4_HIDDEN, 3, 3), (K4_HIDDEN,), (K4_C, K4_HIDDEN, 3, 3),
              (K4_C,)]
    theta = synth.he_normal_params(K4_SEED, [("w" if len(sh) == 4 else "b", sh) for sh in shapes])
    wts, o = [], 0
    for sh in shapes:
        nsz = int(np.prod(sh))
        wts.append(torch.from_numpy(theta[o:o + nsz].astype(np.float32).reshape(sh)).cuda())
        o += nsz
    hf, wf = K4_H // K4_STRIDE, K4_W // K4_STRIDE
    feat = torch.randn((n_maps, hf, wf, K4_C), generator=torch.Generator(device="cuda").manual_seed(K4_SEED),
                       device="cuda")
    h = bm.Handle(0)
    out = torch.empty_like(feat)
    for _ in range(3):
        h.refine_conv(feat, wts, out=out)
    torch.cuda.synchronize()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record()
    for _ in range(5):
        h.refine_conv(feat, wts, out=out)
    e1.record()
    torch.cuda.synchronize()
    ms = e0.elapsed_time(e1) / 5
    flops = n_maps * refine_flops_per_frame()
    h.close()
    return {"refine_maps": n_maps, "ms": round(ms, 4), "tflops": round(flops / (ms / 1e3) / 1e12, 1)}


def train_step_timing(h, d_frames, d_mv, steps: int, batch: int = 16):
    """The proposal network's training step on a batch of `batch` 1080p pairs
    (the clip's 7 pairs repeated, labelled by the exhaustive field): loss +
    gradient (network forward and tensor-core backward) and the AdamW update,
    `steps` timed calls each after three untimed ones."""
    import torch
    from paper_2508_05990_b300 import bayer_me as bm
    from paper_2508_05990_b300 import synth
    idx = torch.arange(batch, device=d_frames.device) % PAIRS
    fr = d_frames.view(torch.int16)  # (CUDA indexing has no uint16 kernels)
    ref, cur = fr[idx].contiguous().view(d_frames.dtype), fr[idx + 1].contiguous().view(d_frames.dtype)
    lab = d_mv[idx].contiguous()
    theta = (np.load(WEIGHTS)["theta"].astype(np.float32) if os.path.exists(WEIGHTS)
             else synth.he_normal_params(5, bm.CNN_SHAPES))
    w = torch.from_numpy(theta).cuda()
    wbf = bm.to_bf16_bits(w).contiguous()
    grad = torch.empty_like(w)
    loss = torch.empty(1, device="cuda")
    m, v = torch.zeros_like(w), torch.zeros_like(w)

    def lg():
        h.cnn_loss_grad(ref, cur, wbf, lab, RANGE, batch=batch, ref_batch_stride=H * W, cur_batch_stride=H * W,
                        grad=grad, loss=loss, neg_weight=5.0)

    def opt():
        h.cnn_adamw(w.clone(), wbf.clone(), grad, m, v, 1, 1e-3)

    out = {"batch": batch, "resolution": f"{W}x{H}"}
    for name, fn in (("loss_grad_ms", lg), ("adamw_ms", opt)):
        for _ in range(3):
            fn()
        torch.cuda.synchronize()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record()
        for _ in range(steps):
            fn()
        e1.record()
        torch.cuda.synchronize()
        out[name] = round(e0.elapsed_time(e1) / steps, 4)
    if h.sync_status() != bm.OK:
        raise RuntimeError("device status after the training step")
    out["pairs_per_s"] = round(batch / (out["loss_grad_ms"] / 1e3), 1)
    return out


def run_train_only(steps: int):
    """The proposal network's training step alone (loss + gradient and AdamW
    on 16 1080p pairs): a small case for profiling the backward kernels."""
    import torch
    from paper_2508_05990_b300 import bayer_me as bm
    from paper_2508_05990_b300 import build, synth
    build.build()
    h = bm.Handle(0)
    d_frames = torch.from_numpy(synth.pan_clip(SEED, H, W, n_frames=T)).cuda()
    d_mv = h.estimate_ex(d_frames, d_frames[1:], block=BLOCK, search_range=RANGE, batch=PAIRS,
                         ref_batch_stride=H * W, cur_batch_stride=H * W)
    res = train_step_timing(h, d_frames, d_mv, steps)
    h.close()
    return res


def run_c2f_only(steps: int):
    """The C2F leg alone on the 1080p clip (its presets, search and search +
    propagation, beside the exhaustive search): a small case for profiling the
    pyramid kernels (frames 33 MB, features 2 x 234 MB on the device)."""
    import torch
    from paper_2508_05990_b300 import bayer_me as bm
    from paper_2508_05990_b300 import build
    build.build()
    frames, feats = make_inputs(0)
    h = bm.Handle(0)
    stream = torch.cuda.current_stream()
    d_frames = torch.from_numpy(frames).cuda()
    d_feats = torch.from_numpy(feats).cuda()
    d_out = torch.empty_like(d_feats)
    full = torch.empty((PAIRS, H // BLOCK, W // BLOCK, 2), dtype=torch.int32, device="cuda")
    kw = dict(batch=PAIRS, ref_batch_stride=H * W, cur_batch_stride=H * W)
    for _ in range(3):
        h.estimate_ex(d_frames, d_frames[1:], search_range=RANGE, out=full, **kw)
    torch.cuda.synchronize()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record()
    for _ in range(steps):
        h.estimate_ex(d_frames, d_frames[1:], search_range=RANGE, out=full, **kw)
    e1.record()
    torch.cuda.synchronize()
    full_ms = e0.elapsed_time(e1) / steps
    pc_clk_sm, mhz, nsm = h.probe_alu(3)
    res = leg_c2f(h, d_frames, d_feats, d_out, stream, steps=steps, warmup=3, pc_clk_sm=pc_clk_sm, nsm=nsm,
                  sm_mhz=mhz, full_me_ms=full_ms, full_step_ms=full_ms)
    h.close()
    return res


def main(argv=None):
    ap = argparse.ArgumentParser(description=__doc__, formatter_class=argparse.RawDescriptionHelpFormatter)
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=300)
    ap.add_argument("--warmup", type=int, default=5)
    ap.add_argument("--impl", choices=["ours", "reference"], default="ours")
    ap.add_argument("--no-cpu-baseline", action="store_true", help="skip the oracle timing leg")
    ap.add_argument("--no-legs", action="store_true",
                    help="skip the batched multi-stream and 4K precision legs (single-GPU runs only)")
    ap.add_argument("--c2f-only", action="store_true",
                    help="run only the coarse-to-fine leg (small case for profiling the pyramid kernels)")
    ap.add_argument("--refine-maps", type=int, default=0,
                    help="profiling aid: time only the BF16 refine convolutions on this many 4K-form maps and exit")
    ap.add_argument("--train-steps", type=int, default=0,
                    help="profiling aid: time only the proposal network's training step (16 1080p pairs) this many "
                         "times and exit")
    args = ap.parse_args(argv)
    if args.train_steps > 0:
        print(json.dumps(run_train_only(args.train_steps)), flush=True)
        return
    if args.c2f_only:
        print(json.dumps(run_c2f_only(10)), flush=True)
        return
    if args.refine_maps > 0:
        print(json.dumps(run_refine_only(args.refine_maps)), flush=True)
        return
    if args.warmup < 3 and args.impl == "ours":
        ap.error("--warmup must be >= 3")
    res = run_reference(args) if args.impl == "reference" else run_ours(args)
    if res is not None:
        print(json.dumps(res), flush=True)


if __name__ == "__main__":
    main()
