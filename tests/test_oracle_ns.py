"""Pins of the oracle's nested sampler and evidence bookkeeping: closed-form
evidence sums, the analytic evidence of a Gaussian likelihood under a uniform
prior, the shrinkage invariant E[ln X_i] = -sum 1/n_j measured with true prior
volumes, and uniformity of the constrained draws."""

import math

import numpy as np
import pytest
from scipy import stats

import workloads as w
from oracle.evidence import Accumulator, log_evidence, simulated_error
from oracle.gauss import GaussOracle
from oracle.ns import NestedSampler


def test_accumulator_constant_likelihood_closed_form():
    # L = e^c everywhere: Z = e^c (1 - X_N), X_N = exp(-sum 1/n_i), H = -ln(1 - X_N)
    c = 3.7
    n = 40
    nl = [n] * 100 + [n - j for j in range(n)]     # k = 1 run, then the final live points
    acc = log_evidence([c] * len(nl), nl)
    logX = -sum(1.0 / v for v in nl)
    assert acc.logX == pytest.approx(logX, rel=1e-14)
    assert acc.logZ == pytest.approx(c + math.log1p(-math.exp(logX)), rel=1e-13)
    assert acc.H == pytest.approx(-math.log1p(-math.exp(logX)), rel=1e-9, abs=1e-12)


def test_accumulator_two_level_closed_form():
    # L = e^a for the first N1 deaths then e^b: Z = e^a (1 - X1) + e^b (X1 - X2)
    a, b, n = -2.0, 1.5, 25
    seq = [a] * 30 + [b] * 45
    nl = [n] * 75
    acc = log_evidence(seq, nl)
    X1, X2 = math.exp(-30 / n), math.exp(-75 / n)
    Z = math.exp(a) * (1 - X1) + math.exp(b) * (X1 - X2)
    assert acc.logZ == pytest.approx(math.log(Z), rel=1e-13)
    H = (math.exp(a) * (1 - X1) * (a - math.log(Z)) + math.exp(b) * (X1 - X2) * (b - math.log(Z))) / Z
    assert acc.H == pytest.approx(H, rel=1e-10)


def test_simulated_error_matches_skilling_estimate():
    # a likelihood with ln L growing linearly in -ln X: scatter ~ sqrt(H / n)
    n = 100
    N = 3000
    i = np.arange(N)
    logL = 0.5 * (i / n)
    nl = np.full(N, n)
    acc = log_evidence(logL, nl)
    err, reps = simulated_error(logL, nl, seed=11, n_replays=400)
    assert err == pytest.approx(math.sqrt(acc.H / n), rel=0.25)
    assert abs(np.mean(reps) - acc.logZ) < 4 * err / math.sqrt(400) + 0.05


def _gauss_run(d, n, k, seed):
    cfg = w.gauss_test(d, n_live=n, n_delete=k, seed=seed)
    o = GaussOracle(w.make_gauss_inputs(cfg))
    ns = NestedSampler.from_config(o.loglike, d, cfg.sampler)
    ns.initialise()
    ns.run()
    return o, ns


@pytest.mark.parametrize("k", [1, 25])
def test_gaussian_evidence_zscores(k):
    """log Z of N(0.5, 0.05^2 I) on [0,1]^2 is 0 (to 1e-20); over 10 seeds the
    z-scores must look standard normal and the reported error match the scatter."""
    zs, lzs, errs = [], [], []
    for seed in range(10):
        o, ns = _gauss_run(2, 50, k, 100 + seed)
        e = ns.evidence(n_replays=100)
        truth = o.log_evidence()
        zs.append((e["logZ"] - truth) / e["logZ_err"])
        lzs.append(e["logZ"])
        errs.append(e["logZ_err"])
        assert ns.status == 0
        assert abs(e["H"] - o.information()) < 1.0
    zs = np.array(zs)
    assert np.all(np.abs(zs) < 4.0)
    assert abs(zs.mean()) < 3.0 / math.sqrt(len(zs)) + 0.3
    assert 0.5 < np.std(lzs, ddof=1) / np.mean(errs) < 1.8


@pytest.mark.parametrize("k", [1, 25])
def test_true_log_volume_invariant_and_uniform_draws(k):
    """With the true enclosed prior volume X(L*) = pi r^2 (r < 0.5, disc inside
    the square), E[ln X_i] = -sum_{j<=i} 1/n_j (Sec. 2.2 bookkeeping), and the
    replacement points are uniform in the disc: (|x - mu| / r*)^2 ~ U(0, 1)."""
    n, d, S = 50, 2, 10
    idx = [120, 200, 280]
    lnX = {i: [] for i in idx}
    rho = []
    for seed in range(S):
        o, ns = _gauss_run(d, n, k, 500 + seed)
        Lmax = -d * math.log(o.sigma * math.sqrt(2 * math.pi))
        dead = np.array(ns.dead_logL)
        nl = np.array(ns.dead_nlive)
        expected = -np.cumsum(1.0 / nl)
        for i in idx:
            r2 = -2 * o.sigma ** 2 * (dead[i] - Lmax)
            assert r2 < 0.45 ** 2
            lnX[i].append(math.log(math.pi * r2) - expected[i])
        for rec in ns.records:
            r2 = -2 * o.sigma ** 2 * (rec.lstar - Lmax)
            if r2 < 0.45 ** 2:
                rho.extend(np.sum((rec.new_x - o.mu) ** 2, axis=1) / r2)
    for i in idx:
        # Var[ln X_i] = sum 1/n_j^2 (per-deletion shrinkage Beta(n_j, 1))
        sd = math.sqrt(np.sum(1.0 / np.array(ns.dead_nlive[:i + 1], float) ** 2) / S)
        assert abs(np.mean(lnX[i])) < 4 * sd, (i, np.mean(lnX[i]), sd)
    rho = np.array(rho)
    assert rho.max() < 1.0
    assert stats.kstest(rho, "uniform").pvalue > 1e-3


def test_slice_bookkeeping_deterministic():
    o, ns1 = _gauss_run(3, 30, 5, 77)
    _, ns2 = _gauss_run(3, 30, 5, 77)
    assert ns1.it == ns2.it
    assert np.array_equal(np.array(ns1.dead_logL), np.array(ns2.dead_logL))
    assert all(np.array_equal(a.evals, b.evals) for a, b in zip(ns1.records, ns2.records))
