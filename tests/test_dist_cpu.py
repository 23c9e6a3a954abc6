"""Replica-only multi-process logic of bench.py on CPU (gloo, world size 2):
each rank draws its own clip (different seeds, same shapes), and the timing
reduction takes the maximum over ranks."""
import os
import socket

import pytest
import torch.multiprocessing as mp


def _free_port():
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    port = s.getsockname()[1]
    s.close()
    return port


def _worker(rank, world, port, q):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank), WORLD_SIZE=str(world),
                      LOCAL_RANK=str(rank))
    import sys
    sys.path.insert(0, os.path.dirname(os.path.dirname(os.path.abspath(__file__))))
    import bench
    from paper_2508_05990_b300 import synth
    r, w, local = bench.init_dist("gloo")
    assert (r, w, local) == (rank, world, rank)
    # each replica's clip comes from its own seed
    frames = synth.pan_clip(bench.SEED + 1000 * r, 64, 96, n_frames=2, rect_size=(8, 24))
    t = bench.max_over_ranks(float(10 + r), w)
    bench.barrier(w)
    q.put((r, t, int(frames.sum())))
    import torch.distributed as dist
    dist.destroy_process_group()


def test_two_replicas_gloo():
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_worker, args=(r, 2, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    for p in procs:
        p.join(120)
    assert all(p.exitcode == 0 for p in procs)
    res = sorted(q.get() for _ in range(2))
    assert res[0][1] == res[1][1] == 11.0  # max over ranks
    assert res[0][2] != res[1][2]  # independent clips


def test_reference_arm_other_ranks_do_nothing(monkeypatch):
    import bench
    monkeypatch.setenv("RANK", "1")
    monkeypatch.setenv("WORLD_SIZE", "2")

    class A:
        steps, warmup = 1, 0
    assert bench.run_reference(A()) is None
