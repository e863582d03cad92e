"""Pins of the oracle's NUTS (Hoffman & Gelman 2014): it samples a known
density (moments and a Kolmogorov-Smirnov test against the normal law), the
dual averaging reaches its target acceptance, and the unconstrained-target
gradient matches central differences."""

import math

import numpy as np
import pytest
from scipy import stats

from oracle.nuts import NUTS, UnconstrainedTarget


def gauss_target(scales):
    s = np.asarray(scales, float)

    def f(z):
        return -0.5 * float(np.sum((z / s) ** 2)), -z / s ** 2
    return f


def test_nuts_samples_a_correlated_free_gaussian():
    scales = [1.0, 0.3, 3.0]
    nuts = NUTS(gauss_target(scales), 3, seed=11, delta=0.8, max_depth=8, adapt_mass=True)
    zs = []
    accs = []
    for c in range(4):
        z, lp, st, eps, minv = nuts.run_chain(c, np.full(3, 0.5), 300, 800, eps0=0.2)
        zs.append(z)
        accs += [a for a, *_ in st[300:]]
    z = np.concatenate(zs)
    for i, s in enumerate(scales):
        x = z[:, i] / s
        assert abs(np.mean(x)) < 0.12
        assert abs(np.std(x) - 1.0) < 0.1
        assert stats.kstest(x, "norm").pvalue > 1e-3
    assert 0.6 < np.mean(accs) < 0.95


def test_unconstrained_target_gradient_matches_differences():
    priors = [("U", -1.0, 2.0), ("N", 0.3, 0.05), ("F", 7.0, 0.0), ("U", 0.0, 5.0)]

    def loglike_grad(th):
        w = np.array([0.7, -1.3, 0.2])
        return float(np.sum(np.sin(w * th))), w * np.cos(w * th)

    t = UnconstrainedTarget(priors, loglike_grad)
    z = np.array([0.4, -0.8, 1.1])
    lp, g = t(z)
    h = 1e-6
    for i in range(3):
        e = np.zeros(3)
        e[i] = h
        fd = (t(z + e)[0] - t(z - e)[0]) / (2 * h)
        assert g[i] == pytest.approx(fd, rel=1e-7, abs=1e-9)
