"""CMB-like dense-covariance likelihood (Sec. 3.1 problem; rows A5, A6, A12,
A13 at C1 shapes) on the GPU against the FP64 oracle: the model vector, log L
through the whitening fold and through the literal per-evaluation whitening,
both covariance factorisation paths (host for small D, blocked device kernels
for large D), the FP32 and BF16 forms within derived bounds, and the nested
sampler's bookkeeping."""

import functools
import math

import numpy as np
import pytest
import torch

import workloads as w
from gpu_helpers import free_theta, random_cube
from oracle.cmb import CMBOracle
from oracle.ns import NestedSampler

pytestmark = pytest.mark.gpu

CMB = {"cmb_tiny": w.cmb_tiny, "cmb_d600": lambda: w.cmb6(n_ell=200), "cmb6": w.cmb6}


@functools.lru_cache(maxsize=None)
def cmb_oracle(name):
    inp = w.make_cmb_inputs(CMB[name]())
    return inp, CMBOracle(inp)


def cmb_problem(name, precision, solve="fold", max_batch=64):
    from paper_2509_13307_gb300 import Problem
    inp, orc = cmb_oracle(name)
    return Problem(inp, precision, max_batch=max_batch, data=orc.data, cov=orc.cov, solve=solve)


def _points(inp, n, seed):
    return free_theta(inp, random_cube(n, 6, seed))


@pytest.mark.parametrize("name", ["cmb_tiny", "cmb_d600"])
@pytest.mark.parametrize("solve", ["fold", "literal"])
def test_fp64_loglike_matches_oracle(name, solve):
    inp, orc = cmb_oracle(name)
    th = _points(inp, 12, 21)
    p = cmb_problem(name, "fp64", solve)
    got = p.loglike(torch.tensor(th, device="cuda")).cpu().numpy()
    ref = np.array([orc.loglike(t) for t in th])
    assert np.allclose(got, ref, rtol=1e-9, atol=0), np.max(np.abs(got / ref - 1))


def test_fp64_model_matches_oracle():
    inp, orc = cmb_oracle("cmb_tiny")
    th = _points(inp, 9, 22)
    p = cmb_problem("cmb_tiny", "fp64")
    got = p.model(torch.tensor(th, device="cuda")).cpu().numpy()
    ref = np.array([orc.model(t) for t in th])
    assert np.allclose(got, ref, rtol=1e-12, atol=1e-12 * np.abs(ref).max())


def _fold_terms(orc, theta, bf16=False):
    """Oracle-side pieces of the fold y = c' - W' h: returns y and the sum of
    absolute terms per element, |c'_a| + sum_k |W'_ak h_k| (FP64)."""
    inp = orc.inp
    sig = inp["emu_out_sig"]
    Linv = np.linalg.inv(orc.L)
    Wf = Linv @ (sig[:, None] * inp["emu_W"][-1])
    cf = Linv @ (orc.data - inp["emu_out_mu"] - sig * inp["emu_b"][-1])
    h = orc.hidden(theta, bf16)
    y = cf - Wf @ h
    return y, np.abs(cf) + np.abs(Wf) @ np.abs(h), Wf, h


@pytest.mark.parametrize("name", ["cmb_tiny", "cmb_d600"])
def test_fp32_within_derived_bound(name):
    """FP32 fold: each y_a is a K-term FP32 dot product (K = hidden width) plus
    c', so |dy_a| <= gamma_K eps32 (|c'_a| + sum_k |W'_ak h_k|) with the input
    activations themselves carrying relative error ~ (layers) eps32; chi^2
    then moves by at most 2 sum_a |y_a| |dy_a|.  The bound uses
    eps_m = 4 (K + 8) 2^-24 per element (accumulation, weights stored in FP32,
    and propagated activation error); the FP64 final add adds nothing."""
    inp, orc = cmb_oracle(name)
    th = _points(inp, 8, 23)
    p = cmb_problem(name, "fp32")
    got = p.loglike(torch.tensor(th, device="cuda")).cpu().numpy()
    K = inp["emu_W"][-1].shape[1]
    eps_m = 4 * (K + 8) * 2.0 ** -24
    for t, g in zip(th, got):
        y, absterm, _, _ = _fold_terms(orc, t)
        ref = orc.c0 - 0.5 * float(y @ y)
        bound = eps_m * float(np.abs(y) @ absterm) + 1e-9 * abs(ref)
        assert abs(g - ref) <= bound, (g - ref, bound)


def test_bf16_against_bf16_aware_oracle():
    """BF16: hidden layers on tensor cores, bf16 activations.  Against the
    oracle with the same bf16 roundings the residual error is the FP32 head
    bound plus, per activation whose bf16 rounding flips under a different
    FP32 summation order or the SFU exponential, a first-order change
    |d chi^2| = |2 y . W'_k| 2^-8 |h_k|; allow two such flips per evaluation."""
    inp, orc = cmb_oracle("cmb_tiny")
    th = _points(inp, 16, 24)
    p = cmb_problem("cmb_tiny", "bf16")
    got = p.loglike(torch.tensor(th, device="cuda")).cpu().numpy()
    K = inp["emu_W"][-1].shape[1]
    eps_m = 4 * (K + 8) * 2.0 ** -24
    errs = []
    for t, g in zip(th, got):
        y, absterm, Wf, h = _fold_terms(orc, t, bf16=True)
        ref = orc.c0 - 0.5 * float(y @ y)
        flip = np.abs(2 * (y @ Wf)) * 2.0 ** -8 * np.abs(h)
        bound = eps_m * float(np.abs(y) @ absterm) + 2 * 0.5 * float(flip.max()) + 1e-9 * abs(ref)
        errs.append(abs(g - ref))
        assert abs(g - ref) <= bound, (g - ref, bound)
    # and the bf16 model itself stays close to the FP64 one on these points
    ref64 = np.array([orc.loglike(t) for t in th])
    assert np.median(np.abs(got - ref64)) < 0.05 * np.median(np.abs(ref64 - orc.c0))


def test_bookkeeping_cmb_tiny():
    """Nested slice sampling on the CMB problem: the GPU FP64 path reproduces
    the oracle's bookkeeping exactly for two batched iterations."""
    from paper_2509_13307_gb300 import NestedRun
    inp, orc = cmb_oracle("cmb_tiny")
    sc = w.cmb_tiny(repeats=4).sampler
    prob = cmb_problem("cmb_tiny", "fp64", max_batch=sc.n_live)
    ons = NestedSampler.from_config(orc.loglike_cube, prob.d, sc)
    ons.initialise()
    run = NestedRun.from_config(prob, sc)
    for _ in range(2):
        ons.iterate()
        st = run.step(1)
        rec = ons.records[-1]
        lstar, dele, starts, evals = run.last_iteration()
        assert lstar == pytest.approx(rec.lstar, rel=1e-11)
        assert np.array_equal(dele, rec.deleted)
        assert np.array_equal(starts, rec.starts)
        assert np.array_equal(evals, rec.evals)
        assert st.logZ == pytest.approx(ons.acc.logZ, rel=1e-11)


def test_invalid_settings():
    from paper_2509_13307_gb300 import Problem
    from paper_2509_13307_gb300._lib import GpunsError
    inp, orc = cmb_oracle("cmb_tiny")
    with pytest.raises(GpunsError):
        Problem(inp, "fp32", data=orc.data, cov=orc.cov, solve="literal")
    bad = np.array(orc.cov)
    bad[0, 0] = -1.0
    with pytest.raises(GpunsError):
        Problem(inp, "fp64", data=orc.data, cov=bad)


def test_full_size_c1():
    """The 6-parameter CMB configuration at full size (D = 7521, dense
    covariance factorised by the device kernels): FP64 fold against the
    oracle's literal forward substitution to 1e-9, and the FP32 fold within
    the derived bound of the FP32 test, on a few points."""
    inp, orc = cmb_oracle("cmb6")
    th = _points(inp, 3, 25)
    ref = np.array([orc.loglike(t) for t in th])
    p64 = cmb_problem("cmb6", "fp64", max_batch=8)
    got64 = p64.loglike(torch.tensor(th, device="cuda")).cpu().numpy()
    assert np.allclose(got64, ref, rtol=1e-9, atol=0), np.max(np.abs(got64 / ref - 1))
    p64.close()
    p32 = cmb_problem("cmb6", "fp32", max_batch=8)
    got32 = p32.loglike(torch.tensor(th, device="cuda")).cpu().numpy()
    K = inp["emu_W"][-1].shape[1]
    eps_m = 4 * (K + 8) * 2.0 ** -24
    for t, g in zip(th, got32):
        y, absterm, _, _ = _fold_terms(orc, t)
        bound = eps_m * float(np.abs(y) @ absterm) + 1e-9 * abs(orc.c0)
        assert abs(g - (orc.c0 - 0.5 * float(y @ y))) <= bound


@functools.lru_cache(maxsize=None)
def tt_oracle(name):
    inp = w.make_cmb_inputs(CMB[name]())
    return inp, CMBOracle(inp, form="tt_cv")


def tt_problem(name, precision, max_batch=64):
    from paper_2509_13307_gb300 import Problem
    inp, orc = tt_oracle(name)
    return Problem(inp, precision, max_batch=max_batch, data=orc.data, form="tt_cv")


def _tt_pieces(orc, theta, bf16=False):
    """Reference log L of the TT form from the oracle's (optionally bf16) hidden
    activations, and the first-order bound pieces: r = C/d, the absolute-term
    sum A_ell of each output (|mu| + sigma (|b| + sum_k |W h|)), and
    d log L / d h."""
    inp = orc.inp
    n = orc.n_tt
    W, b = inp["emu_W"][-1][:n], inp["emu_b"][-1][:n]
    mu, sig = inp["emu_out_mu"][:n], inp["emu_out_sig"][:n]
    h = orc.hidden(theta, bf16)
    C = mu + sig * (W @ h + b)
    k, d = orc.k, orc.data
    r = C / d
    g = np.log(r) + 1.0 / r - 1.0
    ref = orc.loglike_tt(theta) if not bf16 else None
    if bf16:
        from oracle.cmb import chi2_logpdf
        ref = float(sum(chi2_logpdf(q * dd / c, q) + math.log(q / c) for q, dd, c in zip(k, d, C)))
    A = np.abs(mu) + sig * (np.abs(b) + np.abs(W) @ np.abs(h))
    gp = 1.0 / r - 1.0 / r ** 2
    dldh = -((0.5 * k * gp * sig / d) @ W)
    return ref, r, g, A, gp, dldh, h


@pytest.mark.parametrize("name", ["cmb_tiny", "cmb_d600"])
def test_tt_fp64_matches_oracle(name):
    inp, orc = tt_oracle(name)
    th = _points(inp, 10, 41)
    p = tt_problem(name, "fp64")
    got = p.loglike(torch.tensor(th, device="cuda")).cpu().numpy()
    ref = np.array([orc.loglike(t) for t in th])
    assert np.allclose(got, ref, rtol=1e-9, atol=0), np.max(np.abs(got / ref - 1))


@pytest.mark.parametrize("precision", ["fp32", "bf16"])
def test_tt_reduced_precision_within_derived_bound(precision):
    """FP32 head: |dC_ell| <= 4 (K + 8) 2^-24 A_ell; log L moves by at most
    sum (k/2) |g'(r)| |dC| / d, plus 2^-22 sum (k/2) g for the FP32 terms and
    their sum.  BF16 additionally: against the oracle with the same bf16
    roundings, plus two first-order activation-rounding flips
    |d log L / d h_k| 2^-8 |h_k|."""
    inp, orc = tt_oracle("cmb_tiny")
    th = _points(inp, 12, 42)
    p = tt_problem("cmb_tiny", precision)
    got = p.loglike(torch.tensor(th, device="cuda")).cpu().numpy()
    K = inp["emu_W"][-1].shape[1]
    eps_m = 4 * (K + 8) * 2.0 ** -24
    bf16 = precision == "bf16"
    for t, gv in zip(th, got):
        ref, r, g, A, gp, dldh, h = _tt_pieces(orc, t, bf16)
        half_k = 0.5 * orc.k
        bound = float(np.sum(half_k * np.abs(gp) * eps_m * A / orc.data)) + 2.0 ** -22 * float(np.sum(half_k * g))
        if bf16:
            bound += 2 * float(np.max(np.abs(dldh) * 2.0 ** -8 * np.abs(h)))
        bound += 1e-9 * abs(ref)
        assert abs(gv - ref) <= bound, (gv - ref, bound)


def test_tt_nested_sampling_bookkeeping():
    from paper_2509_13307_gb300 import NestedRun
    inp, orc = tt_oracle("cmb_tiny")
    sc = w.cmb_tiny(repeats=4).sampler
    prob = tt_problem("cmb_tiny", "fp64", max_batch=sc.n_live)
    ons = NestedSampler.from_config(orc.loglike_cube, prob.d, sc)
    ons.initialise()
    run = NestedRun.from_config(prob, sc)
    for _ in range(2):
        ons.iterate()
        st = run.step(1)
        rec = ons.records[-1]
        lstar, dele, starts, evals = run.last_iteration()
        assert np.array_equal(dele, rec.deleted) and np.array_equal(evals, rec.evals)
        assert st.logZ == pytest.approx(ons.acc.logZ, rel=1e-11)
