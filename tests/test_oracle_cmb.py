"""Pins of the oracle's CMB-like likelihood (Sec. 3.1 test problem, dense
covariance form) against closed forms, library routines and invariants."""

import copy
import math

import numpy as np
import pytest
from scipy import linalg

import workloads as w
from oracle.cmb import CMBOracle, sigmoid_linear


@pytest.fixture(scope="module")
def tiny():
    inp = w.make_cmb_inputs(w.cmb_tiny())
    return inp, CMBOracle(inp)


def test_activation_closed_forms():
    x = np.array([-2.0, -0.5, 0.0, 0.7, 3.0])
    # gamma = 1: identity
    assert np.array_equal(sigmoid_linear(x, 1.0, 0.8), x)
    # gamma = 0, beta = 1: x sigmoid(x), the SiLU / swish
    assert np.allclose(sigmoid_linear(x, 0.0, 1.0), x / (1.0 + np.exp(-x)), rtol=0, atol=1e-15)
    # value at one point written out: g = 0.25, beta = 2, x = 0.7
    s = 1.0 / (1.0 + math.exp(-1.4))
    assert sigmoid_linear(0.7, 0.25, 2.0) == pytest.approx((0.25 + 0.75 * s) * 0.7, rel=1e-15)
    # large beta: gamma x for x < 0 and x for x > 0 (leaky ReLU with slope gamma)
    with np.errstate(over="ignore"):
        y = sigmoid_linear(x, 0.3, 1e6)
    assert np.allclose(y, np.where(x > 0, x, 0.3 * x), atol=1e-12)


def test_linear_network_reduces_to_composed_affine_map(tiny):
    """gamma = 1 makes every hidden layer affine: the emulator must equal the
    product of the weight matrices applied to the standardised input."""
    inp, _ = tiny
    lin = copy.deepcopy(inp)
    lin["act_g"] = [np.ones_like(g) for g in inp["act_g"]]
    o = CMBOracle(lin, data=np.zeros(inp["n_data"]), cov=np.eye(inp["n_data"]))
    th = np.array(inp["fiducial"]) * 1.03
    x = (th - inp["emu_in_center"]) / inp["emu_in_scale"]
    A = np.eye(6)
    c = np.zeros(6)
    for W, b in zip(inp["emu_W"], inp["emu_b"]):
        A = W @ A
        c = W @ c + b
    y = A @ x + c
    assert np.allclose(o.emulator(th), inp["emu_out_mu"] + inp["emu_out_sig"] * y, rtol=1e-12, atol=0)


def test_identity_covariance_chi2_is_sum_of_squares(tiny):
    inp, o = tiny
    D = inp["n_data"]
    rng = np.random.default_rng(5)
    data = rng.standard_normal(D)
    oi = CMBOracle(inp, data=data, cov=np.eye(D))
    th = np.array(inp["fiducial"]) * 0.98
    r = data - oi.model(th)
    assert oi.chi2(th) == pytest.approx(float(r @ r), rel=1e-13)
    assert oi.c0 == pytest.approx(-0.5 * D * math.log(2 * math.pi), rel=1e-15)


def test_forward_substitution_matches_library_solve(tiny):
    inp, o = tiny
    rng = np.random.default_rng(6)
    r = rng.standard_normal(inp["n_data"])
    y = o.forward_subst(r)
    ref = linalg.solve_triangular(o.L, r, lower=True)
    assert np.allclose(y, ref, rtol=1e-12, atol=1e-12)


def test_mock_scale_and_whitened_noise(tiny):
    inp, o = tiny
    mfid = o.model(np.asarray(inp["fiducial"]))
    target = (inp["cov_rel"] * math.sqrt(np.mean(mfid ** 2))) ** 2
    assert np.mean(np.diag(o.cov)) == pytest.approx(target, rel=1e-12)
    # data = m_fid + L eps, so the whitened residual at the fiducial is eps
    y = o.forward_subst(o.data - mfid)
    assert np.allclose(y, inp["noise_eps"], rtol=0, atol=1e-9)
    assert o.loglike_full(np.asarray(inp["fiducial"])) == pytest.approx(
        o.c0 - 0.5 * float(inp["noise_eps"] @ inp["noise_eps"]), rel=1e-12)


def test_wishart_base_spectrum():
    """E[W] = I and a Marchenko-Pastur spectrum for D / nu = 1/2:
    eigenvalues within [(1 - r)^2, (1 + r)^2] up to edge fluctuations."""
    D, nu = 200, 400
    W = w.wishart_base(D, nu, 2)
    assert np.allclose(W, W.T)
    e = np.linalg.eigvalsh(W)
    r = math.sqrt(D / nu)
    assert e.min() > 0.8 * (1 - r) ** 2 and e.max() < 1.15 * (1 + r) ** 2
    assert np.mean(np.diag(W)) == pytest.approx(1.0, abs=0.02)


def test_bf16_rounding_matches_torch():
    torch = pytest.importorskip("torch")
    x = np.random.default_rng(8).standard_normal(4096) * 10.0 ** np.random.default_rng(9).uniform(-3, 3, 4096)
    ref = torch.tensor(x, dtype=torch.float32).to(torch.bfloat16).to(torch.float64).numpy()
    assert np.array_equal(CMBOracle.to_bf16(x), ref)


def test_tt_cosmic_variance_form():
    """The TT form: chi-squared log density against scipy, the closed form
    -(k/2)(d/C + ln C) + const, and its maximum at C = d for every multipole."""
    from scipy import stats
    from oracle.cmb import chi2_logpdf
    for k, x in ((5.0, 3.2), (41.0, 47.5), (2001.0, 1987.0)):
        assert chi2_logpdf(x, k) == pytest.approx(stats.chi2.logpdf(x, k), rel=1e-12)
    inp = w.make_cmb_inputs(w.cmb_tiny())
    o = CMBOracle(inp, form="tt_cv")
    th = np.array(inp["fiducial"]) * 1.01
    C = o.model(th)[: o.n_tt]
    k, d = o.k, o.data
    const = np.sum((0.5 * k - 1) * np.log(k * d) - 0.5 * k * np.log(2.0)
                   - np.array([math.lgamma(0.5 * q) for q in k]) + np.log(k))
    closed = const - np.sum(0.5 * k * (d / C + np.log(C)))
    assert o.loglike_full(th) == pytest.approx(closed, rel=1e-12)
    # each term is maximised at C = d: d/dC [-(k/2)(d/C + ln C)] = (k/2)(d/C^2 - 1/C) = 0
    for j in range(3):
        f = lambda c: -(0.5 * k[j]) * (d[j] / c + math.log(c))
        assert f(d[j]) > f(d[j] * 1.001) and f(d[j]) > f(d[j] * 0.999)
    # mock: d = C_fid X / k with the seeded chi-squared draws
    cfid = o.model(np.asarray(inp["fiducial"]))[: o.n_tt]
    assert np.allclose(d * k / cfid, inp["tt_chi2"], rtol=1e-13)
