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


ME_SOURCES = ("paper_2508_05990_b300/csrc/me_full16.cu", "paper_2508_05990_b300/csrc/common.cuh")
PROP_SOURCES = ("paper_2508_05990_b300/csrc/propagate.cu", "paper_2508_05990_b300/csrc/common.cuh")


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


def cpu_baseline_sample(frames, feats):
    """Oracle (as it stands) on one of the 7 pairs: exhaustive search + bilinear warp."""
    import oracle
    oracle.build()
    t0 = time.perf_counter()
    field, _ = oracle.me_full(frames[0], frames[1], BLOCK, RANGE, even=True)
    oracle.propagate(feats[0], field, BLOCK, STRIDE, interp=oracle.BILINEAR)
    dt = time.perf_counter() - t0
    return {"value": 1.0 / dt, "unit": UNIT, "cores": oracle.get_threads(), "kind": "oracle",
            "sample": "1 of the 7 pairs of the 1080p clip (full ME + bilinear propagation), all host threads"}


def run_ours(args):
    import torch
    rank, world, local = init_dist("nccl")
    torch.cuda.set_device(local)
    from paper_2508_05990_b300 import bayer_me as bm
    from paper_2508_05990_b300 import build
    build.build()

    frames, feats = make_inputs(rank)
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
    with ClockSampler(local) as clk:
        time.sleep(0.5)  # let the sampler start
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
            "weights": os.path.relpath(WEIGHTS, ROOT),
            "gpu_launches": args.steps * 9,
        }

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

    # ALU roofline: measured sad.u32 throughput per clock per SM x SMs x SM clock under load
    pc_clk_sm, probe_mhz, nsm = h.probe_alu(0)
    result = None
    if rank == 0:
        clocks = clk.summary(t_host0, t_host1)
        sm_mhz = clocks["sm_mhz"] or probe_mhz
        me_avg_s = statistics.mean(me_ms) / 1e3
        achieved = PAIRS * pc_per_pair() / me_avg_s / 1e9
        peak = pc_clk_sm * nsm * sm_mhz * 1e6 / 1e9
        prop_avg_s = statistics.mean(prop_ms) / 1e3
        prop_gbs = PAIRS * prop_bytes_per_pair() / prop_avg_s / 1e9
        peaks = {}
        try:
            peaks = json.load(open(os.path.join(ROOT, "MEASURED_PEAKS.json")))
        except (OSError, ValueError):
            pass
        hbm_peak = peaks.get("hbm_gbs", 6400.0)
        value = world * PAIRS * args.steps / (ms_total / 1e3)
        result = {
            "metric": METRIC, "value": round(value, 2), "unit": UNIT, "n_gpus": world, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": round(ms_total / args.steps, 4), "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "u16 frames, u32 SAD, f32 features",
            "data": "synthetic (seeded pan+rectangles Bayer clip, N(0,1) features)",
            "config": {"workload": WORKLOAD, "pairs_per_step": PAIRS, "search": "plain exhaustive",
                       "l2": "inputs larger than L2 (267 MB read + 234 MB written per step); no flush",
                       "parallelism": f"replicas x{world} (independent clips, no collective)"},
            "roofline": {"bound": "alu", "kernel": "me_full16_even_kernel<16>", "achieved": round(achieved, 1),
                         "peak": round(peak, 1), "unit": "G pixel-candidates/s", "frac": round(achieved / peak, 4),
                         "peak_source": f"measured sad.u32 loop: {pc_clk_sm:.1f} pc/clk/SM x {nsm} SMs x "
                                        f"{sm_mhz:.0f} MHz (median SM clock under load)",
                         "traffic": profiled_traffic("me_full16_even_1080p_clip.md", ME_SOURCES),
                         "traffic_unit": "DRAM bytes per launch (ncu)",
                         "algorithmic_per_launch": f"{PAIRS * pc_per_pair()} pixel-candidates",
                         "avg_launch_ms": round(me_avg_s * 1e3, 4)},
            "propagation": {"bound": "hbm", "achieved": round(prop_gbs, 1), "peak": hbm_peak, "unit": "GB/s",
                            "frac": round(prop_gbs / hbm_peak, 4), "avg_launch_ms": round(prop_avg_s * 1e3, 4),
                            "traffic": profiled_traffic("prop_nchw_bilinear_1080p_clip.md", PROP_SOURCES),
                            "algorithmic_bytes_per_launch": PAIRS * prop_bytes_per_pair(),
                            "peak_source": "MEASURED_PEAKS.json hbm_gbs (of measured)"},
            "mblocks_per_s": round(value * hb * wb / 1e6, 3),
            "e2e": {"value": round(world * PAIRS * args.steps / e2e_s, 2), "unit": UNIT,
                    "h2d_bytes_per_step": int(h2d), "d2h_bytes_per_step": int(d2h),
                    "api": "bayer_clip_process_host (pinned host buffers, 3 streams)"},
            "gpu_launches": gpu_launches,
            "clocks": clocks,
            "learned_seeded": learned,
        }
        if not args.no_cpu_baseline:
            result["cpu_baseline"] = cpu_baseline_sample(frames, feats)
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
        "config": {"workload": WORKLOAD, "pairs_per_step": 1,
                   "sample": "each step = 1 pair of the 1080p clip (of 7), CPU oracle"},
        "cpu_baseline": {"value": round(value, 4), "unit": UNIT, "cores": cores, "kind": "oracle",
                         "sample": "1 pair per step of the 1080p clip, plain C oracle, all host threads"},
        "e2e": {"value": round(value, 4), "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
    }


def main(argv=None):
    ap = argparse.ArgumentParser(description=__doc__, formatter_class=argparse.RawDescriptionHelpFormatter)
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=300)
    ap.add_argument("--warmup", type=int, default=5)
    ap.add_argument("--impl", choices=["ours", "reference"], default="ours")
    ap.add_argument("--no-cpu-baseline", action="store_true", help="skip the oracle timing leg")
    args = ap.parse_args(argv)
    if args.warmup < 3 and args.impl == "ours":
        ap.error("--warmup must be >= 3")
    res = run_reference(args) if args.impl == "reference" else run_ours(args)
    if res is not None:
        print(json.dumps(res), flush=True)


if __name__ == "__main__":
    main()
