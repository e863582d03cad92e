"""Row A15 (packed runs) and row A7 (coarse-z emulator interpolation).

Packing: runs of one model with different priors (so different dimensions),
live-point counts and deletion counts share each round's likelihood batch;
every run must reproduce, exactly, the same run made alone (whose bookkeeping
is itself pinned to the oracle by test_gpu_ns).

Interpolation: the emulator on 10 coarse z nodes, Catmull-Rom interpolated to
the 50-node table (App. B of the paper interpolates in z on a 10x coarser
grid; the reading here is Catmull-Rom): FP64 log L and the adjoint against the
oracle."""

from dataclasses import replace

import numpy as np
import pytest
import torch

import workloads as w
from gpu_helpers import cuda_problem, free_theta, oracle_for, random_cube

pytestmark = pytest.mark.gpu


def _t(a):
    return torch.tensor(np.ascontiguousarray(a), dtype=torch.float64, device="cuda")


def _inputs_with_fixed(name, fixed):
    inp, orc = oracle_for(name)
    names = inp["param_names"]
    pri = list(inp["priors"])
    fid = inp["fiducial"]
    for nm in fixed:
        i = names.index(nm)
        pri[i] = ("F", float(fid[i]), 0.0)
    return dict(inp, priors=pri), orc


def _problem_with_fixed(name, fixed, precision="fp64", max_batch=64):
    from paper_2509_13307_gb300 import Problem
    inp2, orc = _inputs_with_fixed(name, fixed)
    return Problem(inp2, precision, max_batch=max_batch, data=orc.data, cov=orc.cov)


def test_packed_runs_reproduce_single_runs():
    from paper_2509_13307_gb300 import NestedRun, MultiRun
    fixed_sets = [[], ["w0", "wa"], ["b_2", "b_3", "A_IA", "eta_IA"]]
    samplers = [w.SamplerConfig(n_live=30, n_delete=6, repeats=4, seed=31),
                w.SamplerConfig(n_live=40, n_delete=8, repeats=5, seed=32),
                w.SamplerConfig(n_live=24, n_delete=4, repeats=3, seed=33)]
    probs = [_problem_with_fixed("shear_tiny", f) for f in fixed_sets]
    assert [p.d for p in probs] == [21, 19, 17]
    multi = MultiRun(probs, samplers)
    singles = [NestedRun.from_config(p, sc) for p, sc in zip(probs, samplers)]
    for it in range(3):
        sts = multi.step(1)
        for i, run in enumerate(singles):
            s1 = run.step(1)
            a = multi.last_iteration(i)
            b = run.last_iteration()
            assert a[0] == b[0]
            for x, y in zip(a[1:], b[1:]):
                assert np.array_equal(x, y)
            assert sts[i].logZ == s1.logZ and sts[i].evaluations == s1.evaluations
    for i, run in enumerate(singles):
        assert multi.evidence(i, 32) == run.evidence(32)
    multi.close()


def test_packed_runs_match_the_oracle():
    """Packed runs against the oracle itself: a d = 19 run (w0, wa fixed) and a
    d = 21 run share every likelihood batch; each reproduces, exactly, the
    oracle's nested sampler on the same Philox streams (deleted slots, start
    slots, evaluations per chain; L*, log Z to FP64 round-off)."""
    from oracle.ns import NestedSampler
    from oracle.shear import ShearOracle
    from paper_2509_13307_gb300 import MultiRun
    fixed_sets = [["w0", "wa"], []]
    samplers = [w.SamplerConfig(n_live=36, n_delete=9, repeats=4, seed=41),
                w.SamplerConfig(n_live=28, n_delete=7, repeats=3, seed=42)]
    probs, onss = [], []
    for f, sc in zip(fixed_sets, samplers):
        inp2, orc = _inputs_with_fixed("shear_tiny", f)
        probs.append(_problem_with_fixed("shear_tiny", f))
        o2 = ShearOracle(inp2, data=orc.data, cov=orc.cov)
        ons = NestedSampler.from_config(o2.loglike_cube, probs[-1].d, sc)
        ons.initialise()
        onss.append(ons)
    assert [p.d for p in probs] == [19, 21]
    multi = MultiRun(probs, samplers)
    for it in range(3):
        sts = multi.step(1)
        for i, ons in enumerate(onss):
            ons.iterate()
            rec = ons.records[-1]
            lstar, dele, starts, evals = multi.last_iteration(i)
            assert lstar == pytest.approx(rec.lstar, rel=1e-12, abs=1e-12)
            assert np.array_equal(dele, rec.deleted)
            assert np.array_equal(starts, rec.starts)
            assert np.array_equal(evals, rec.evals)
            assert sts[i].logZ == pytest.approx(ons.acc.logZ, rel=1e-12, abs=1e-12)
            assert sts[i].evaluations == ons.n_evals
    multi.close()


@pytest.mark.parametrize("name", ["shear39_interp", "shear39_interp_linear"])
def test_interpolated_emulator_fp64_parity(name):
    inp, orc = oracle_for(name)
    p = cuda_problem(name, "fp64", max_batch=8)
    th = free_theta(inp, random_cube(4, p.d, 51))
    got = p.loglike(_t(th)).cpu().numpy()
    ref = np.array([orc.loglike(t) for t in th])
    assert np.all(np.abs(got / ref - 1) < 1e-9)


@pytest.mark.parametrize("name", ["shear39_interp", "shear39_interp_linear"])
def test_interpolated_emulator_adjoint(name):
    inp, orc = oracle_for(name)
    p = cuda_problem(name, "fp64", max_batch=8)
    th = free_theta(inp, random_cube(1, p.d, 52, 0.1, 0.9))
    _, g = p.loglike_grad(_t(th))
    ref = orc.grad_complex_step(th[0])
    assert np.max(np.abs(g.cpu().numpy()[0] - ref)) / np.max(np.abs(ref)) < 1e-9
