"""One nested-sampling run split into shards of its chains (ns_shard_*), the
multi-device chain split the paper leaves to future work (Sec. 4.1, Sec. 5):
on one GPU the shards run one after another and the host concatenates their
exported chain states in shard order (the all-gather a multi-GPU run does with
NCCL), so no kernel waits on another shard.  Every shard must then hold,
bit for bit, the state of the same run made unsharded (which test_gpu_ns pins
to the oracle), and the Gaussian test run must match the oracle directly."""

import numpy as np
import pytest
import torch

import workloads as w
from gpu_helpers import cuda_problem

pytestmark = pytest.mark.gpu


def _iterate(shards):
    sts = [r.shard_evolve() for r in shards]
    if sts[0].converged:
        return sts
    finals = torch.cat([r.shard_export() for r in shards])
    return [r.shard_insert(finals) for r in shards]


def _shards(prob, sc, G, **kw):
    from paper_2509_13307_gb300 import NestedRun
    return [NestedRun.from_config(prob, sc, n_shards=G, shard=s, **kw) for s in range(G)]


@pytest.mark.parametrize("prec,G", [("fp64", 2), ("fp64", 3), ("bf16", 2)])
def test_shards_reproduce_the_unsharded_run(prec, G):
    from paper_2509_13307_gb300 import NestedRun, shard_bounds
    sc = w.shear_tiny(repeats=5).sampler
    prob = cuda_problem("shear_tiny", prec, max_batch=sc.n_live)
    ref = NestedRun.from_config(prob, sc)
    shards = _shards(prob, sc, G)
    assert [r.chain_range for r in shards] == shard_bounds(sc.n_delete, G)
    for _ in range(3):
        s_ref = ref.step(1)
        sts = _iterate(shards)
        a = ref.last_iteration()
        x_ref, l_ref = ref.live_points()
        for r, st in zip(shards, sts):
            b = r.last_iteration()
            assert a[0] == b[0] and all(np.array_equal(u, v) for u, v in zip(a[1:], b[1:]))
            x, lg = r.live_points()
            assert np.array_equal(x, x_ref) and np.array_equal(lg, l_ref)
            assert st.logZ == s_ref.logZ and st.logX == s_ref.logX and st.evaluations == s_ref.evaluations
    e_ref = ref.evidence(32)
    for r in shards:
        assert r.evidence(32) == e_ref
        xd, ld, nd = r.dead_points()
        xr, lr, nr = ref.dead_points()
        assert np.array_equal(ld, lr) and np.array_equal(nd, nr) and np.array_equal(xd, xr)


def test_sharded_gauss_run_matches_the_oracle_to_convergence():
    from oracle.gauss import GaussOracle
    from oracle.ns import NestedSampler
    from paper_2509_13307_gb300 import Problem
    cfg = w.gauss_test(3, n_live=40, n_delete=6, seed=23)
    inp = w.make_gauss_inputs(cfg)
    ons = NestedSampler.from_config(GaussOracle(inp).loglike, 3, cfg.sampler)
    ons.initialise()
    ons.run()
    prob = Problem(inp, "fp64", max_batch=40)
    shards = _shards(prob, cfg.sampler, 4)
    for _ in range(10000):
        sts = _iterate(shards)
        if sts[0].converged:
            break
    assert all(s.iterations == ons.it for s in sts)
    e_o = ons.evidence(n_replays=40)
    for r in shards:
        e = r.evidence(40)
        assert e["n_dead"] == e_o["n_dead"]
        assert e["logZ"] == pytest.approx(e_o["logZ"], rel=1e-11, abs=1e-11)
        assert e["logZ_err"] == pytest.approx(e_o["logZ_err"], rel=1e-8)


def test_shard_call_order_is_enforced():
    from paper_2509_13307_gb300._lib import GpunsError
    sc = w.shear_tiny(repeats=3).sampler
    prob = cuda_problem("shear_tiny", "fp64", max_batch=sc.n_live)
    r0, r1 = _shards(prob, sc, 2)
    with pytest.raises(GpunsError):
        r0.step(1)                      # a shard advances only through ns_shard_*
    with pytest.raises(GpunsError):
        r0.shard_export()               # nothing evolved yet
    r0.shard_evolve()
    with pytest.raises(GpunsError):
        r0.shard_evolve()               # the iteration waits for its insert
    with pytest.raises(ValueError):
        r0.shard_insert(torch.zeros((3, prob.d + 2), dtype=torch.float64, device="cuda"))
    from paper_2509_13307_gb300 import NestedRun
    with pytest.raises(GpunsError):
        NestedRun.from_config(prob, sc, n_shards=sc.n_delete + 1, shard=0)
    with pytest.raises(GpunsError):
        NestedRun.from_config(prob, sc, n_shards=2, shard=2)
