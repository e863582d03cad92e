"""NUTS driver (ns_nuts_run) against the oracle NUTS on the same Philox
streams, its sampling of a known posterior, and a short run on the shear
likelihood's adjoint."""

import numpy as np
import pytest
import torch

import workloads as w
from gpu_helpers import cuda_problem
from oracle.gauss import GaussOracle
from oracle.nuts import NUTS, UnconstrainedTarget

pytestmark = pytest.mark.gpu


def _gauss(d, max_batch=32):
    from paper_2509_13307_gb300 import Problem
    cfg = w.gauss_test(d)
    inp = w.make_gauss_inputs(cfg)
    return inp, Problem(inp, "fp64", max_batch=max_batch)


def test_nuts_matches_oracle_on_gaussian_test_problem():
    from paper_2509_13307_gb300 import nuts
    d = 3
    inp, prob = _gauss(d)
    mu, sig = inp["mu"], inp["sigma"]

    def lg(th):
        r = (th - mu) / sig
        return -0.5 * float(r @ r) - d * np.log(sig * np.sqrt(2 * np.pi)), -r / sig

    z0 = np.array([[0.3, -0.2, 0.1], [-0.4, 0.25, 0.05]])
    out = nuts(prob, 2, 20, 12, z0=z0, seed=17, init_step=0.05, adapt_mass=False)
    orc = NUTS(UnconstrainedTarget(inp["priors"], lg), d, seed=17, adapt_mass=False)
    for c in range(2):
        zs, lps, st, eps, _ = orc.run_chain(c, z0[c], 20, 12, eps0=0.05)
        assert np.allclose(out["z"][c], zs, rtol=1e-8, atol=1e-10)
        assert np.allclose(out["logp"][c], lps, rtol=1e-10, atol=1e-10)
        assert out["step_size"][c] == pytest.approx(eps, rel=1e-10)


def test_nuts_samples_gaussian_posterior():
    from paper_2509_13307_gb300 import nuts
    d = 5
    inp, prob = _gauss(d, max_batch=16)
    out = nuts(prob, 16, 300, 250, seed=3, init_step=0.1)
    th = out["theta"].reshape(-1, d)
    assert np.all(np.abs(th.mean(axis=0) - inp["mu"]) < 0.01)
    assert np.all(np.abs(th.std(axis=0) / inp["sigma"] - 1.0) < 0.12)
    assert 0.6 < out["stats"]["mean_accept"] < 0.95
    assert out["stats"]["divergences"] == 0


@pytest.mark.parametrize("precision", ["fp64", "bf16"])
def test_nuts_on_shear_adjoint(precision):
    from paper_2509_13307_gb300 import nuts
    prob = cuda_problem("shear_tiny", precision, max_batch=16)
    out = nuts(prob, 8, 20, 10, seed=9, init_step=0.02, max_depth=6)
    assert np.all(np.isfinite(out["logp"]))
    assert out["stats"]["gradient_evals"] > 8 * 30
    assert np.all(np.isfinite(out["theta"]))


def test_nuts_posterior_agrees_with_nested_sampling():
    """The two samplers of the paper's comparison (nested sampling and NUTS on
    the hand-written adjoint, Sec. 3.2) sample the same posterior of the small
    shear problem (FP64): for each of the 21 parameters
    z = (mean_NUTS - mean_NS) / sqrt(se_NUTS^2 + se_NS^2), se_NUTS from the
    spread of the chain means and se_NS^2 = sd^2 / (Kish ESS of the weights)
    plus the variance of the mean over simulated shrinkage sequences (the
    weights are themselves random, Eq. 1), has mean z^2 below 4 and no |z|
    above 6; the standard deviations agree within 35 %."""
    from paper_2509_13307_gb300 import NestedRun, nuts
    prob = cuda_problem("shear_tiny", "fp64", max_batch=400)
    run = NestedRun(prob, 400, 100, seed=21)
    st = run.run()
    assert st.converged
    x, lg, logw = run.posterior()
    _, _, nd = run.dead_points()
    nl = np.concatenate([nd, run.n_live - np.arange(run.n_live)]).astype(float)
    run.close()
    th = np.concatenate([prob.prior_transform(torch.tensor(x[i:i + 400], device="cuda")).cpu().numpy()
                         for i in range(0, len(x), 400)])
    wgt = np.exp(logw)
    m_ns = wgt @ th
    s_ns = np.sqrt(wgt @ (th - m_ns) ** 2)
    ess = 1.0 / np.sum(wgt ** 2)
    # the weights' own randomness: the posterior mean under 64 simulated
    # shrinkage sequences t_i ~ Beta(n_i, 1) (the evidence error's procedure)
    rng = np.random.default_rng(5)
    reps = []
    for _ in range(64):
        lnX = np.cumsum(np.log(rng.random(len(nl))) / nl)
        lnX_prev = np.concatenate([[0.0], lnX[:-1]])
        lw = lg + lnX_prev + np.log(-np.expm1(lnX - lnX_prev))
        wr = np.exp(lw - lw.max())
        reps.append((wr / wr.sum()) @ th)
    se_ns = np.sqrt(s_ns ** 2 / ess + np.var(reps, axis=0, ddof=1))
    n_ch = 16
    pick = np.random.default_rng(3).choice(len(wgt), size=n_ch, p=wgt)
    xc = np.clip(x[pick], 1e-9, 1 - 1e-9)
    out = nuts(prob, n_ch, 200, 250, z0=np.log(xc) - np.log1p(-xc), seed=13, init_step=0.05, max_depth=8)
    t = out["theta"]
    m_h = t.reshape(-1, t.shape[-1]).mean(axis=0)
    s_h = t.reshape(-1, t.shape[-1]).std(axis=0)
    se_h = t.mean(axis=1).std(axis=0, ddof=1) / np.sqrt(n_ch)
    z = (m_h - m_ns) / np.sqrt(se_h ** 2 + se_ns ** 2)
    print(f"ESS(NS) {ess:.0f}, mean z^2 {np.mean(z ** 2):.2f}, max |z| {np.max(np.abs(z)):.2f}, sd ratio {np.min(s_h / s_ns):.2f} .. "
          f"{np.max(s_h / s_ns):.2f}, accept {out['stats']['mean_accept']:.2f}, depth {out['stats']['mean_depth']:.1f}")
    assert np.mean(z ** 2) < 4.0 and np.all(np.abs(z) < 6.0), z
    assert np.all(np.abs(s_h / s_ns - 1.0) < 0.35), s_h / s_ns
