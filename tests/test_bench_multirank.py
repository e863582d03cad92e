"""The benchmark's multi-rank aggregation on CPU ranks (gloo, world size 2):
time = max over ranks, evaluations = sum over ranks, and per-rank sampler
seeds that differ (independent runs, weak scaling)."""

import os
import socket
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _worker(rank, world, port, q):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank), WORLD_SIZE=str(world))
    sys.path.insert(0, ROOT)
    import torch
    import torch.distributed as dist
    import bench
    import workloads as w
    dist.init_process_group("gloo", rank=rank, world_size=world)
    t, e = bench.job_totals(1.5 + rank, 1000 * (rank + 1), world, torch.device("cpu"))
    seed = bench.replace_seed(w.shear39().sampler, rank).seed
    q.put((rank, t, e, seed))
    dist.barrier()
    dist.destroy_process_group()


def test_job_totals_two_gloo_ranks():
    import torch.multiprocessing as mp
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_worker, args=(r, 2, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    out = sorted(q.get(timeout=120) for _ in procs)
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    for rank, t, e, _ in out:
        assert t == pytest.approx(2.5) and e == pytest.approx(3000.0)
    assert out[0][3] != out[1][3]


def test_job_totals_single_rank():
    import bench
    assert bench.job_totals(2.0, 10, 1, None) == (2.0, 10.0)
