"""CMB-like Gaussian likelihood (the paper's CMB test problem, Sec. 3.1, in the
dense-covariance form of the 6-parameter LCDM configuration), in plain FP64
NumPy.  Test infrastructure only.

Steps, each following the cited passage:
  emulator    MLP stand-in for the CosmoPower C_ell emulator (Sec. 2.5): hidden
              layers h <- f(W h + b) with CosmoPower's activation
              f(x) = [gamma + (1 - gamma) sigmoid(beta x)] x (one gamma, beta per
              unit), a linear head, outputs de-standardised as mu + sigma * y.
              Inputs are the 6 parameters standardised over the prior box.
  model       m(theta) = the emulator output (TT, TE, EE stacked).
  loglike     Gaussian: -1/2 |L^-1 (d - m)|^2 - sum ln L_aa - D/2 ln 2 pi, the
              whitening by explicit forward substitution (no fast algebra);
              or, for the cosmic-variance-limited TT analysis of Sec. 3.1
              (form "tt_cv"), the density of the observed d_ell given
              C_ell(theta) when k d_ell / C_ell is chi-squared with
              k = 2 ell + 1 degrees of freedom:
              ln L = sum_ell [ln f_k(k d / C) + ln(k / C)],
              ln f_k(x) = (k/2 - 1) ln x - x/2 - (k/2) ln 2 - ln Gamma(k/2).

Mock data and covariance: C = s W with W the seeded Wishart-style base of the
workload inputs and s setting the mean variance to (cov_rel * rms m_fid)^2;
data = m_fid + L eps.  TT mock: d_ell = C_fid,ell X_ell / k_ell with the seeded
chi-squared draws X_ell of the workload inputs.
"""

from __future__ import annotations

import math

import numpy as np

from .priors import cube_to_theta, theta_free_to_full


def sigmoid_linear(x, g, beta):
    """CosmoPower's activation [g + (1 - g) / (1 + exp(-beta x))] x."""
    return (g + (1.0 - g) / (1.0 + np.exp(-beta * x))) * x


def chi2_logpdf(x, k):
    """ln of the chi-squared density with k degrees of freedom at x > 0."""
    return (0.5 * k - 1.0) * math.log(x) - 0.5 * x - 0.5 * k * math.log(2.0) - math.lgamma(0.5 * k)


class CMBOracle:
    def __init__(self, inp: dict, data=None, cov=None, wishart=None, form: str = "gauss"):
        self.inp = inp
        self.priors = inp["priors"]
        self.D = int(inp["n_data"])
        self.form = form
        if form == "tt_cv":
            self.n_tt = len(inp["ell"])
            self.k = 2.0 * np.asarray(inp["ell"], float) + 1.0
            self.data = np.asarray(data, float) if data is not None else self.make_mock_tt()
            return
        if data is None or cov is None:
            data, cov = self.make_mock(wishart)
        self.set_data(data, cov)

    def make_mock_tt(self):
        cfid = self.model(np.asarray(self.inp["fiducial"], float))[: self.n_tt]
        return cfid * self.inp["tt_chi2"] / self.k

    # ----------------------------------------------------------- emulator
    @staticmethod
    def to_bf16(a):
        """Round to the nearest bfloat16 (ties to even) through float32, returned as float64."""
        f = np.asarray(a, dtype=np.float32).copy()
        u = f.view(np.uint32)
        u += np.uint32(0x7FFF) + ((u >> np.uint32(16)) & np.uint32(1))
        u &= np.uint32(0xFFFF0000)
        return u.view(np.float32).astype(np.float64)

    def hidden(self, theta, bf16=False):
        """Last hidden activation h.  With bf16=True the weights of the hidden
        layers >= 1 and every hidden activation are rounded to bfloat16 (the
        arithmetic stays FP64): the model the tensor-core path computes, up to
        its FP32 accumulation order."""
        inp = self.inp
        x = (np.asarray(theta)[inp["emu_inputs"]] - inp["emu_in_center"]) / inp["emu_in_scale"]
        Ws, bs = inp["emu_W"], inp["emu_b"]
        h = x
        for l in range(len(Ws) - 1):
            W = self.to_bf16(Ws[l]) if (bf16 and l >= 1) else Ws[l]
            h = sigmoid_linear(W @ h + bs[l], inp["act_g"][l], inp["act_beta"][l])
            if bf16:
                h = self.to_bf16(h)
        return h

    def emulator(self, theta, bf16=False):
        """De-standardised emulator output mu + sigma * y, shape (D,); the
        linear head in FP64 (FP32 on the tensor-core path)."""
        inp = self.inp
        y = inp["emu_W"][-1] @ self.hidden(theta, bf16) + inp["emu_b"][-1]
        return inp["emu_out_mu"] + inp["emu_out_sig"] * y

    def model(self, theta):
        return self.emulator(theta)

    # ----------------------------------------------------------- data
    def make_mock(self, wishart=None):
        inp = self.inp
        mfid = self.model(np.asarray(inp["fiducial"], float))
        if wishart is None:
            from workloads import wishart_base
            wishart = wishart_base(self.D, int(inp["wishart_nu"]), int(inp["seed_cov"]))
        s = (inp["cov_rel"] * math.sqrt(np.mean(mfid * mfid))) ** 2 / np.mean(np.diag(wishart))
        cov = s * wishart
        data = mfid + np.linalg.cholesky(cov) @ inp["noise_eps"]
        return data, cov

    def set_data(self, data, cov):
        self.data = np.asarray(data, float)
        self.cov = np.asarray(cov, float)
        self.L = np.linalg.cholesky(self.cov)
        self.c0 = -np.sum(np.log(np.diag(self.L))) - 0.5 * self.D * math.log(2.0 * math.pi)

    # ----------------------------------------------------------- likelihood
    def forward_subst(self, r):
        """Solve L y = r by explicit forward substitution."""
        L = self.L
        y = np.zeros(self.D, dtype=np.result_type(r, L))
        for a in range(self.D):
            y[a] = (r[a] - L[a, :a] @ y[:a]) / L[a, a]
        return y

    def whitened(self, theta, bf16=False):
        return self.forward_subst(self.data - self.emulator(theta, bf16))

    def chi2(self, theta):
        y = self.whitened(theta)
        return float(np.sum(y * y))

    def loglike_tt(self, theta):
        C = self.model(theta)[: self.n_tt]
        return float(sum(chi2_logpdf(k * d / c, k) + math.log(k / c) for k, d, c in zip(self.k, self.data, C)))

    def loglike_full(self, theta):
        if self.form == "tt_cv":
            return self.loglike_tt(theta)
        return -0.5 * self.chi2(theta) + self.c0

    def loglike(self, theta_free):
        return self.loglike_full(theta_free_to_full(self.priors, np.asarray(theta_free)))

    def loglike_cube(self, cube):
        return self.loglike_full(cube_to_theta(self.priors, cube))
