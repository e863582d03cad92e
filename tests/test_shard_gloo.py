"""One nested-sampling run split over ranks (ShardedRun, the multi-device
chain split the paper leaves to future work; the k chains of an iteration are
independent, Sec. 2.2) on CPU gloo ranks, world sizes 2 and 3.

Each rank holds a shard whose chains are evolved by the oracle's slice sampler
(a test stand-in for the device shard, which needs a GPU); ShardedRun's
exchange (one padded all-gather of every shard's final chain states per
iteration, unpadded in shard order) must hand every rank exactly the
single-process sampler's iteration: the same dead sequence, live set and
evidence on every rank."""

import math
import os
import socket
import sys
from types import SimpleNamespace

import numpy as np
import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _sampler():
    import workloads as w
    from oracle.gauss import GaussOracle
    from oracle.ns import NestedSampler
    cfg = w.gauss_test(3, n_live=40, n_delete=7, repeats=4, seed=19)
    orc = GaussOracle(w.make_gauss_inputs(cfg))
    ons = NestedSampler.from_config(orc.loglike, 3, cfg.sampler)
    ons.initialise()
    return ons


class OracleShard:
    """Shard s of G of an oracle nested sampler: the iteration's deletion,
    covariance and starts are computed for all chains (as every device does),
    the slice moves only for this shard's chains."""

    def __init__(self, ons, n_shards, shard):
        from paper_2509_13307_gb300.api import shard_bounds
        self.ons = ons
        self.n_delete, self.d = ons.n_delete, ons.d
        self.n_shards, self.shard = n_shards, shard
        self.chain_range = shard_bounds(ons.n_delete, n_shards)[shard]

    def _status(self):
        return SimpleNamespace(converged=self.ons.converged(), logZ=self.ons.acc.logZ)

    def shard_evolve(self):
        from oracle import philox
        o = self.ons
        if o.converged():
            return self._status()
        n, k, it = o.n_live, o.n_delete, o.it
        order = o.sorted_order()
        self.deleted, survivors = order[:k], order[k:]
        self.lstar = float(o.logL[self.deleted[-1]])
        for j, s in enumerate(self.deleted):
            o.acc.add(float(o.logL[s]), n - j)
            o.dead_x.append(o.x[s].copy())
            o.dead_logL.append(float(o.logL[s]))
            o.dead_nlive.append(n - j)
        Lc = o.live_cholesky()
        b, e = self.chain_range
        self.local = np.zeros((e - b, self.d + 2))
        for c in range(b, e):
            u = philox.uniform_scalar(o.seed, philox.PURPOSE_START, 0, it, c, 0)
            s = survivors[int(math.floor(u * (n - k)))]
            x, lx, ev = o.slice_chain(it, c, o.x[s].copy(), float(o.logL[s]), self.lstar, Lc)
            self.local[c - b, :self.d], self.local[c - b, self.d], self.local[c - b, self.d + 1] = x, lx, ev
        return SimpleNamespace(converged=False, logZ=o.acc.logZ)

    def shard_export(self):
        import torch
        return torch.tensor(self.local, dtype=torch.float64)

    def shard_insert(self, finals):
        o = self.ons
        f = finals.numpy()
        assert f.shape == (self.n_delete, self.d + 2)
        for c in range(self.n_delete):
            o.x[self.deleted[c]] = f[c, :self.d]
            o.logL[self.deleted[c]] = f[c, self.d]
        o.it += 1
        return self._status()


def _worker(rank, world, port, n_iter, q):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank), WORLD_SIZE=str(world))
    sys.path.insert(0, ROOT)
    import torch.distributed as dist
    from paper_2509_13307_gb300.api import ShardedRun
    dist.init_process_group("gloo", rank=rank, world_size=world)
    shard = OracleShard(_sampler(), world, rank)
    run = ShardedRun(shard, group=None)
    for _ in range(n_iter):
        run.step(1)
    o = shard.ons
    q.put((rank, np.array(o.dead_logL), o.x.copy(), o.logL.copy(), o.acc.logZ, o.acc.logX))
    dist.barrier()
    dist.destroy_process_group()


@pytest.mark.parametrize("world", [2, 3])
def test_sharded_run_equals_single_process_run(world):
    import torch.multiprocessing as mp
    n_iter = 5
    ref = _sampler()
    for _ in range(n_iter):
        ref.iterate()
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_worker, args=(r, world, port, n_iter, q)) for r in range(world)]
    for p in procs:
        p.start()
    outs = sorted((q.get(timeout=300) for _ in procs), key=lambda t: t[0])
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    for rank, dead, x, lg, lz, lx in outs:
        assert np.array_equal(dead, np.array(ref.dead_logL)), rank
        assert np.array_equal(x, ref.x) and np.array_equal(lg, ref.logL), rank
        assert lz == ref.acc.logZ and lx == ref.acc.logX


def test_shard_bounds_cover_the_chains():
    from paper_2509_13307_gb300.api import shard_bounds
    for k, G in [(500, 1), (500, 2), (500, 3), (7, 3), (5, 5), (1000, 8)]:
        b = shard_bounds(k, G)
        assert b[0][0] == 0 and b[-1][1] == k
        assert all(b[i][1] == b[i + 1][0] for i in range(G - 1))
        assert max(e - s for s, e in b) - min(e - s for s, e in b) <= 1
