"""GPU nested sampler against the CPU oracle on the same Philox streams
(rows A1-A5, A11): the slice bookkeeping (deleted slots, start slots,
evaluations per chain) must match exactly; thresholds, live points and the
evidence accumulators to FP64 round-off."""

import math

import numpy as np
import pytest
import torch

import workloads as w
from gpu_helpers import cuda_problem, oracle_for
from oracle.gauss import GaussOracle
from oracle.ns import NestedSampler

pytestmark = pytest.mark.gpu


def _gauss_pair(d, n, k, repeats, seed):
    from paper_2509_13307_gb300 import Problem, NestedRun
    cfg = w.gauss_test(d, n_live=n, n_delete=k, repeats=repeats, seed=seed)
    inp = w.make_gauss_inputs(cfg)
    orc = GaussOracle(inp)
    ons = NestedSampler.from_config(orc.loglike, d, cfg.sampler)
    ons.initialise()
    prob = Problem(inp, "fp64", max_batch=max(n, k))
    run = NestedRun.from_config(prob, cfg.sampler)
    return ons, prob, run


def _compare_iterations(ons, run, n_iter):
    for _ in range(n_iter):
        ons.iterate()
        st = run.step(1)
        rec = ons.records[-1]
        lstar, dele, starts, evals = run.last_iteration()
        assert lstar == pytest.approx(rec.lstar, rel=1e-12, abs=1e-12)
        assert np.array_equal(dele, rec.deleted)
        assert np.array_equal(starts, rec.starts)
        assert np.array_equal(evals, rec.evals), (evals, rec.evals)
        assert st.logZ == pytest.approx(ons.acc.logZ, rel=1e-12, abs=1e-12)
        assert st.logX == pytest.approx(ons.acc.logX, rel=1e-13)
    x, lg = run.live_points()
    assert np.allclose(x, ons.x, rtol=0, atol=1e-10)
    assert np.allclose(lg, ons.logL, rtol=1e-10, atol=1e-10)
    assert st.evaluations == ons.n_evals


@pytest.mark.parametrize("k", [1, 6])
def test_bookkeeping_gauss(k):
    ons, prob, run = _gauss_pair(5, 60, k, None, 7)
    _compare_iterations(ons, run, 4)


def test_bookkeeping_more_than_64_parameters():
    """70 full parameters: 67 fixed (the last three at full indices 64 - 66)
    and 3 free at full indices 67 - 69.  The Gaussian likelihood sums over
    every full parameter, so a proposal row whose parameters past 64 were not
    written by the prior transform would leave the oracle's bookkeeping."""
    from paper_2509_13307_gb300 import Problem, NestedRun
    from oracle.priors import cube_to_theta
    cfg = w.gauss_test(3, n_live=40, n_delete=4, seed=29)
    inp = dict(w.make_gauss_inputs(cfg))
    priors = [("F", 0.3 + 0.005 * i, 0.0) for i in range(67)] + [("U", 0.0, 1.0)] * 3
    inp["priors"], inp["n_params"] = priors, len(priors)
    orc = GaussOracle(inp)
    ons = NestedSampler.from_config(lambda u: orc.loglike(cube_to_theta(priors, u)), 3, cfg.sampler)
    ons.initialise()
    prob = Problem(inp, "fp64", max_batch=40)
    run = NestedRun.from_config(prob, cfg.sampler)
    _compare_iterations(ons, run, 4)


def test_bookkeeping_shear5_plain_ns():
    """The 5-parameter toy with k = 1 (plain nested sampling)."""
    from paper_2509_13307_gb300 import NestedRun
    inp, orc = oracle_for("shear5")
    sc = w.shear5().sampler
    prob = cuda_problem("shear5", "fp64", max_batch=sc.n_live)
    ons = NestedSampler.from_config(orc.loglike_cube, prob.d, sc)
    ons.initialise()
    run = NestedRun.from_config(prob, sc)
    _compare_iterations(ons, run, 3)


def test_bookkeeping_odd_rounds_per_launch():
    """Rounds per graph launch are rounded up to an even number (the round
    batch counters alternate by parity): an odd request still reproduces the
    oracle's bookkeeping exactly."""
    from paper_2509_13307_gb300 import Problem, NestedRun
    cfg = w.gauss_test(4, n_live=50, n_delete=10, seed=13)
    inp = w.make_gauss_inputs(cfg)
    orc = GaussOracle(inp)
    ons = NestedSampler.from_config(orc.loglike, 4, cfg.sampler)
    ons.initialise()
    prob = Problem(inp, "fp64", max_batch=50)
    run = NestedRun.from_config(prob, cfg.sampler, rounds_per_sync=3)
    _compare_iterations(ons, run, 3)


def test_bookkeeping_shear_tiny_batched():
    from paper_2509_13307_gb300 import NestedRun
    inp, orc = oracle_for("shear_tiny")
    sc = w.shear_tiny(repeats=6).sampler
    prob = cuda_problem("shear_tiny", "fp64", max_batch=sc.n_live)
    ons = NestedSampler.from_config(orc.loglike_cube, prob.d, sc)
    ons.initialise()
    run = NestedRun.from_config(prob, sc)
    _compare_iterations(ons, run, 2)


def test_bookkeeping_two_chain_groups():
    """Chains split into two groups whose rounds run on two streams: the
    bookkeeping is still the oracle's (each chain's proposals and likelihoods
    do not depend on which batch scores them)."""
    from paper_2509_13307_gb300 import NestedRun
    inp, orc = oracle_for("shear_tiny")
    sc = w.shear_tiny(repeats=6).sampler
    prob = cuda_problem("shear_tiny", "fp64", max_batch=sc.n_live)
    ons = NestedSampler.from_config(orc.loglike_cube, prob.d, sc)
    ons.initialise()
    run = NestedRun.from_config(prob, sc, chain_groups=2)
    _compare_iterations(ons, run, 2)


def test_chain_groups_bf16_identical():
    """BF16: one and two chain groups give bit-identical runs."""
    from paper_2509_13307_gb300 import NestedRun
    sc = w.shear_tiny(repeats=4).sampler
    prob = cuda_problem("shear_tiny", "bf16", max_batch=sc.n_live)
    r1 = NestedRun.from_config(prob, sc, chain_groups=1)
    r2 = NestedRun.from_config(prob, sc, chain_groups=2)
    s1, s2 = r1.step(3), r2.step(3)
    x1, l1 = r1.live_points()
    x2, l2 = r2.live_points()
    assert np.array_equal(x1, x2) and np.array_equal(l1, l2)
    assert s1.logZ == s2.logZ and s1.evaluations == s2.evaluations


def test_full_run_matches_oracle():
    """Both samplers to convergence: same number of dead points, log Z, H and
    the simulated-shrinkage error (same Philox replays)."""
    ons, prob, run = _gauss_pair(3, 40, 4, None, 11)
    ons.run()
    st = run.run()
    assert st.converged and st.iterations == ons.it
    e_o = ons.evidence(n_replays=50)
    e_g = run.evidence(n_replays=50)
    assert e_g["n_dead"] == e_o["n_dead"]
    assert e_g["logZ"] == pytest.approx(e_o["logZ"], rel=1e-11, abs=1e-11)
    assert e_g["H"] == pytest.approx(e_o["H"], rel=1e-9, abs=1e-10)
    assert e_g["logX"] == pytest.approx(e_o["logX"], rel=1e-12)
    assert e_g["logZ_err"] == pytest.approx(e_o["logZ_err"], rel=1e-8)
    xd, ld, nd = run.dead_points()
    assert np.allclose(ld, np.array(ons.dead_logL), rtol=1e-11, atol=1e-11)
    assert np.array_equal(nd, np.array(ons.dead_nlive))


def test_gaussian_evidence_closed_form():
    from paper_2509_13307_gb300 import Problem, NestedRun
    d = 5
    cfg = w.gauss_test(d, n_live=200, n_delete=40, seed=21)
    inp = w.make_gauss_inputs(cfg)
    orc = GaussOracle(inp)
    prob = Problem(inp, "fp64", max_batch=200)
    zs = []
    for seed in range(4):
        run = NestedRun(prob, 200, 40, seed=100 + seed)
        st = run.run()
        e = run.evidence()
        assert st.status_bits == 0
        zs.append((e["logZ"] - orc.log_evidence()) / e["logZ_err"])
        assert abs(e["H"] - orc.information()) < 1.0
    assert np.all(np.abs(zs) < 4.0), zs


def test_slice_cap_is_reported():
    from paper_2509_13307_gb300 import Problem, NestedRun
    cfg = w.gauss_test(4, n_live=50, n_delete=5)
    prob = Problem(w.make_gauss_inputs(cfg), "fp64", max_batch=50)
    run = NestedRun(prob, 50, 5, width=1e-3, step_cap=2)
    st = run.step(2)
    assert st.status_bits & 1


def test_invalid_run_settings():
    from paper_2509_13307_gb300 import Problem, NestedRun
    from paper_2509_13307_gb300._lib import GpunsError
    cfg = w.gauss_test(4, n_live=50, n_delete=5)
    prob = Problem(w.make_gauss_inputs(cfg), "fp64", max_batch=50)
    for n, k in [(50, 50), (50, 0), (5000, 10)]:
        with pytest.raises(GpunsError):
            NestedRun(prob, n, k)


@pytest.mark.parametrize("prec", ["bf16", "fp32"])
def test_reduced_precision_evidence_agrees_with_fp64(prec):
    """FP32 / BF16 runs diverge from the FP64 stream chaotically (the design
    notes' P10), so they are judged statistically: log Z within four combined
    standard errors of the FP64 run on the 5-parameter toy."""
    from paper_2509_13307_gb300 import NestedRun
    inp, orc = oracle_for("shear5")
    res = {}
    for pr in ("fp64", prec):
        prob = cuda_problem("shear5", pr, max_batch=100)
        run = NestedRun(prob, 100, 10, seed=5)
        st = run.run()
        assert st.converged
        res[pr] = run.evidence()
        run.close()
        prob.close()
    a, b = res["fp64"], res[prec]
    sig = math.hypot(a["logZ_err"], b["logZ_err"])
    assert abs(a["logZ"] - b["logZ"]) < 4 * sig, (a, b)
