"""The benchmark's multi-rank host logic, run as two gloo ranks on CPU: each rank renders its own
pose of the scene (weak scaling over views, no data-path collective), the job's time is the
slowest rank's (max over ranks) and its rate counts the views of all ranks; a non-zero rank of the
reference arm exits without work."""
import argparse
import io
import os
import socket
import sys
from contextlib import redirect_stdout

import numpy as np
import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _worker(rank, world, port, q):
    sys.path.insert(0, ROOT)
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank),
                      WORLD_SIZE=str(world), LOCAL_RANK=str(rank))
    import torch
    import torch.distributed as dist
    import bench
    dist.init_process_group("gloo", rank=rank, world_size=world)
    cam = bench.rank_camera(rank)
    W = torch.tensor(np.asarray(cam["W"], np.float64).reshape(-1))
    Ws = [torch.zeros(9, dtype=torch.float64) for _ in range(world)]
    dist.all_gather(Ws, W)
    t = 0.25 * (rank + 1)  # this rank's timed seconds
    slowest = bench.max_over_ranks(t, dist)
    rate = bench.job_rate(world, 10, slowest)
    out = io.StringIO()
    args = argparse.Namespace(gpus=world, steps=1, warmup=0)
    with redirect_stdout(out):
        ref_rc = bench.run_reference(args) if rank > 0 else 0
    dist.barrier()
    dist.destroy_process_group()
    q.put((rank, [w.tolist() for w in Ws], slowest, rate, ref_rc, out.getvalue()))


def test_two_gloo_ranks_weak_scaling_and_max_over_ranks():
    import multiprocessing as mp
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_worker, args=(r, 2, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    res = sorted(q.get(timeout=240) for _ in procs)
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    (r0, W0, s0, v0, rc0, o0), (r1, W1, s1, v1, rc1, o1) = res
    assert (r0, r1) == (0, 1)
    assert W0 == W1  # both ranks see the same gathered poses
    assert not np.allclose(W0[0], W0[1])  # one distinct pose per rank
    sys.path.insert(0, ROOT)
    import bench
    from paper_2409_04751_gb300 import scenes
    assert s0 == s1 == pytest.approx(0.5)  # the slowest rank's time on every rank
    assert v0 == v1 == pytest.approx(2 * 10 / 0.5)  # views of all ranks over that time
    assert rc1 == 0 and o1 == ""  # the reference arm's rank 1 prints nothing
    # rank 0's view is the benchmark view (config 1's pose, seed 1 * 1000 + 1)
    assert bench.rank_camera(0)["W"].tolist() == scenes.pose_camera(1752, 1168, 180.0, 1001)["W"].tolist()
    assert np.allclose(np.asarray(W0[0]), bench.rank_camera(0)["W"].reshape(-1))
