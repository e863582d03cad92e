"""No-U-Turn sampler (Hoffman & Gelman 2014) with dual-averaging step-size
adaptation, in plain FP64 NumPy.  Test infrastructure only.

The paper compares its nested-sampling evidences with an HMC/NUTS + learned
harmonic-mean analysis (Sec. 3.2); this is the NUTS half, sampling the same
posteriors.  The algorithm follows the published NUTS with the slice variable
(efficient NUTS with dual averaging, Algorithms 3 and 6 of Hoffman & Gelman):

  * target: the posterior in unconstrained coordinates z in R^d with
    unit-cube coordinate c = 1 / (1 + e^-z) and theta = prior transform(c),
    log p(z) = log L(theta) + sum_i ln(c_i (1 - c_i));
  * momentum r ~ N(0, M), M = diag(1 / minv); kinetic energy 1/2 sum minv r^2;
  * slice: ln u = H(z, r) + ln U;  a leaf is valid if ln u <= H, divergent if
    ln u - H > 1000;
  * the trajectory doubles (direction +-1 with probability 1/2) up to
    max_depth times; the new subtree's leapfrog states are generated in order
    and every completed binary sub-subtree is checked for a U-turn,
    (z_end - z_start) . r_start >= 0 and (z_end - z_start) . r_end >= 0 in the
    direction of travel; the subtree's candidate is a uniformly chosen valid
    leaf (reservoir selection, which has the distribution of the recursive
    merge rule); it replaces the current sample with probability
    min(1, n'/n) if the subtree did not stop; the whole trajectory stops at a
    U-turn between its two ends;
  * warm-up: dual averaging of ln eps towards acceptance statistic delta
    (gamma 0.05, t0 10, kappa 0.75, mu = ln(10 eps0)); with mass adaptation
    the inverse mass becomes the regularised variance of z over warm-up
    iterations [W/4, 3W/4) and dual averaging restarts there; sampling uses
    the averaged step size.

Random numbers come from Philox4x32-10 (counter purpose | j << 8, iteration,
chain, extra): momentum (NUTS_MOM, j = dimension pair), slice (NUTS_SLICE),
direction (NUTS_DIR, j = depth), merge (NUTS_MERGE, j = depth) and reservoir
(NUTS_LEAF, j = depth, extra = leaf index), so that the library's driver, fed
the same gradients, makes the same moves.
"""

from __future__ import annotations

import math

import numpy as np

from . import philox
from .special import inv_normal_cdf

PURPOSE_NUTS_MOM = 7
PURPOSE_NUTS_SLICE = 8
PURPOSE_NUTS_DIR = 9
PURPOSE_NUTS_MERGE = 10
PURPOSE_NUTS_LEAF = 11

DELTA_MAX = 1000.0


def momentum_normals(seed, it, chain, d):
    """d standard normals by Box-Muller on the NUTS_MOM pairs (dims 2j, 2j + 1)."""
    return philox.normals(seed, PURPOSE_NUTS_MOM, it, chain, 0, d)


def u01(seed, purpose, j, it, chain, extra=0):
    return philox.uniform_scalar(seed, purpose, j, it, chain, extra)


class UnconstrainedTarget:
    """log p(z) and its gradient from a physical-parameter log-likelihood with
    gradient, through the logistic map to the unit cube and the prior
    transform (uniform: theta = a + (b - a) c; Gaussian: theta = a + b Phi^-1(c))."""

    def __init__(self, priors, loglike_grad):
        self.free = [p for p in priors if p[0] != "F"]
        self.loglike_grad = loglike_grad

    def theta(self, z):
        c = 1.0 / (1.0 + np.exp(-z))
        th = np.empty_like(z)
        dth = np.empty_like(z)
        for i, (kind, a, b) in enumerate(self.free):
            if kind == "U":
                th[i] = a + (b - a) * c[i]
                dth[i] = b - a
            else:
                x = inv_normal_cdf(c[i])
                th[i] = a + b * x
                dth[i] = b * math.sqrt(2.0 * math.pi) * math.exp(0.5 * x * x)
        return th, c, dth

    def __call__(self, z):
        th, c, dth = self.theta(z)
        logL, g = self.loglike_grad(th)
        logp = logL + float(np.sum(np.log(c) + np.log1p(-c)))
        grad = g * dth * c * (1.0 - c) + (1.0 - 2.0 * c)
        return logp, grad


class NUTS:
    def __init__(self, target, d, seed, delta=0.8, max_depth=10, adapt_mass=True):
        self.f = target
        self.d = d
        self.seed = seed
        self.delta = delta
        self.max_depth = max_depth
        self.adapt_mass = adapt_mass

    def iteration(self, it, chain, z, logp, grad, eps, minv):
        """One NUTS transition; returns (z, logp, grad, accept statistic, depth, divergent, n_grad)."""
        d, seed = self.d, self.seed
        r0 = momentum_normals(seed, it, chain, d) / np.sqrt(minv)
        H0 = logp - 0.5 * float(np.sum(minv * r0 * r0))
        log_u = H0 + math.log(u01(seed, PURPOSE_NUTS_SLICE, 0, it, chain))
        zm = zp = z.copy()
        rm = rp = r0.copy()
        gm = gp = grad.copy()
        z_new, lp_new, g_new = z, logp, grad
        n, s, j = 1, True, 0
        a_sum, n_a, n_grad, divergent = 0.0, 0, 0, False
        while s and j < self.max_depth:
            v = -1.0 if u01(seed, PURPOSE_NUTS_DIR, j, it, chain) < 0.5 else 1.0
            zc, rc, gc = (zm, rm, gm) if v < 0 else (zp, rp, gp)
            left = {}
            n1, s1 = 0, True
            cand = None
            for i in range(2 ** j):
                rc = rc + 0.5 * v * eps * gc
                zc = zc + v * eps * minv * rc
                lpc, gc = self.f(zc)
                rc = rc + 0.5 * v * eps * gc
                n_grad += 1
                H = lpc - 0.5 * float(np.sum(minv * rc * rc))
                if not math.isfinite(H):
                    H = -math.inf
                a_sum += min(1.0, math.exp(min(0.0, H - H0))) if H > -math.inf else 0.0
                n_a += 1
                if log_u - H > DELTA_MAX:
                    s1, divergent = False, True
                    break
                if log_u <= H:
                    n1 += 1
                    if u01(seed, PURPOSE_NUTS_LEAF, j, it, chain, i) * n1 < 1.0:
                        cand = (zc, lpc, gc)
                for lev in range(1, j + 1):
                    if i % (2 ** lev) == 0:
                        left[lev] = (zc, rc)
                stop = False
                for lev in range(1, j + 1):
                    if (i + 1) % (2 ** lev) == 0:
                        zl, rl = left[lev]
                        dz = v * (zc - zl)
                        if float(dz @ rl) < 0.0 or float(dz @ rc) < 0.0:
                            stop = True
                            break
                if stop:
                    s1 = False
                    break
            if v < 0:
                zm, rm, gm = zc, rc, gc
            else:
                zp, rp, gp = zc, rc, gc
            if s1 and n1 > 0 and cand is not None:
                if u01(seed, PURPOSE_NUTS_MERGE, j, it, chain) * n < n1:
                    z_new, lp_new, g_new = cand
            n += n1
            dz = zp - zm
            s = s1 and float(dz @ rm) >= 0.0 and float(dz @ rp) >= 0.0
            j += 1
        return z_new, lp_new, g_new, a_sum / max(n_a, 1), j, divergent, n_grad

    def run_chain(self, chain, z0, n_warmup, n_samples, eps0=0.1, minv=None):
        d = self.d
        minv = np.ones(d) if minv is None else np.asarray(minv, float).copy()
        z = np.asarray(z0, float).copy()
        logp, grad = self.f(z)
        eps = eps0
        mu, hbar, log_eps_bar, m_da = math.log(10.0 * eps0), 0.0, 0.0, 0
        w_lo, w_hi = n_warmup // 4, (3 * n_warmup) // 4
        window = []
        out_z, out_lp, stats = [], [], []
        for it in range(n_warmup + n_samples):
            z, logp, grad, acc, depth, div, ng = self.iteration(it, chain, z, logp, grad, eps, minv)
            stats.append((acc, depth, div, ng, eps))
            if it < n_warmup:
                m_da += 1
                eta = 1.0 / (m_da + 10.0)
                hbar = (1.0 - eta) * hbar + eta * (self.delta - acc)
                log_eps = mu - math.sqrt(m_da) / 0.05 * hbar
                w = m_da ** -0.75
                log_eps_bar = w * log_eps + (1.0 - w) * log_eps_bar
                eps = math.exp(log_eps)
                if self.adapt_mass and w_lo <= it < w_hi:
                    window.append(z.copy())
                if self.adapt_mass and it == w_hi - 1 and len(window) > 1:
                    var = np.var(np.array(window), axis=0, ddof=1)
                    nw = len(window)
                    minv = (nw / (nw + 5.0)) * var + 1e-3 * (5.0 / (nw + 5.0))
                    mu, hbar, log_eps_bar, m_da = math.log(10.0 * eps), 0.0, 0.0, 0
                if it == n_warmup - 1:
                    eps = math.exp(log_eps_bar)
            else:
                out_z.append(z.copy())
                out_lp.append(logp)
        return np.array(out_z), np.array(out_lp), stats, eps, minv
