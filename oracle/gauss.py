"""Isotropic Gaussian test likelihood on the unit cube with a uniform prior.
Test infrastructure only.

    log L(x) = -1/2 sum_i ((x_i - mu)/sigma)^2 - d ln(sigma sqrt(2 pi))

Its evidence (Eq. 1 with pi = 1 on the cube) and information have closed forms:
    log Z = d ln[Phi((1-mu)/sigma) - Phi(-mu/sigma)]
    H     = E_post[ln L] - ln Z, with the truncated-normal second moment
            E[(x-mu)^2/sigma^2] = 1 - (beta phi(beta) - alpha phi(alpha)) / (Phi(beta) - Phi(alpha)),
            alpha = -mu/sigma, beta = (1-mu)/sigma.
"""

from __future__ import annotations

import math

import numpy as np
from scipy.special import ndtr


class GaussOracle:
    def __init__(self, inp: dict):
        self.d = int(inp["n_params"])
        self.mu = float(inp["mu"])
        self.sigma = float(inp["sigma"])
        self.priors = inp["priors"]

    def loglike(self, x):
        x = np.asarray(x)
        r = (x - self.mu) / self.sigma
        return -0.5 * np.sum(r * r, axis=-1) - self.d * math.log(self.sigma * math.sqrt(2 * math.pi))

    loglike_cube = loglike
    loglike_full = loglike

    def log_evidence(self) -> float:
        a, b = -self.mu / self.sigma, (1.0 - self.mu) / self.sigma
        return self.d * math.log(ndtr(b) - ndtr(a))

    def information(self) -> float:
        a, b = -self.mu / self.sigma, (1.0 - self.mu) / self.sigma
        phi = lambda t: math.exp(-0.5 * t * t) / math.sqrt(2 * math.pi)
        mass = ndtr(b) - ndtr(a)
        m2 = 1.0 - (b * phi(b) - a * phi(a)) / mass
        e_lnL = -0.5 * self.d * m2 - self.d * math.log(self.sigma * math.sqrt(2 * math.pi))
        return e_lnL - self.log_evidence()
