"""Small numerical helpers for the oracle.  Test infrastructure only."""

from __future__ import annotations

import math

import numpy as np
from scipy.special import ndtri


def lse2(a: float, b: float) -> float:
    """log(exp(a) + exp(b)) for scalars, -inf aware."""
    if a == -math.inf:
        return b
    if b == -math.inf:
        return a
    m = max(a, b)
    return m + math.log(math.exp(a - m) + math.exp(b - m))


def lse(x) -> float:
    x = np.asarray(x, dtype=float)
    if x.size == 0:
        return -math.inf
    m = np.max(x)
    if m == -math.inf:
        return -math.inf
    return float(m + np.log(np.sum(np.exp(x - m))))


def log1mexp_neg(x: float) -> float:
    """log(1 - exp(-x)) for x > 0."""
    return math.log(-math.expm1(-x))


def inv_normal_cdf(u):
    """Phi^-1(u), via scipy.special.ndtri (library routine)."""
    return ndtri(u)
