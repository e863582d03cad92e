"""Evidence bookkeeping for nested sampling with batched deletion.
Test infrastructure only.

Skilling (2006) nested sampling estimates Z = int L dX (Eq. 1 of the paper,
with X the enclosed prior mass) as sum_i w_i L_i over dead points.  Deleting
the k lowest of n live points at once (Sec. 2.2) is the same as deleting them
one at a time with n, n-1, ..., n-k+1 live points, so the j-th deletion of a
batch shrinks X by t with E[ln t] = -1/(n-j).  With the expected shrinkage:

    ln X_i = ln X_{i-1} - 1/n_i
    w_i    = X_{i-1} - X_i              (ln w_i = ln X_{i-1} + ln(1 - e^{-1/n_i}))
    ln Z   = LSE(ln Z, ln L_i + ln w_i)
    H      = e^{ln w_i + ln L_i - ln Z'} ln L_i + e^{ln Z - ln Z'} (H + ln Z) - ln Z'

The statistical error is estimated by simulating the shrinkage: S replays draw
ln t_i = ln(U_i) / n_i (t_i ~ Beta(n_i, 1)), recompute ln Z, and report the
standard deviation (ddof = 1) of the replays; U_i comes from Philox with
counter (ERR, replay s, dead index i, 0).
"""

from __future__ import annotations

import math

import numpy as np

from . import philox
from .special import lse, lse2, log1mexp_neg


class Accumulator:
    def __init__(self):
        self.logZ = -math.inf
        self.logX = 0.0
        self.H = 0.0
        self.n_dead = 0

    def add(self, logL: float, n_live: int):
        logw = self.logX + log1mexp_neg(1.0 / n_live)
        logZ_new = lse2(self.logZ, logL + logw)
        if logZ_new == -math.inf:
            H = 0.0
        else:
            H = math.exp(logw + logL - logZ_new) * logL if logL > -math.inf else 0.0
            if self.logZ > -math.inf:
                H += math.exp(self.logZ - logZ_new) * (self.H + self.logZ)
            H -= logZ_new
        self.H = H
        self.logZ = logZ_new
        self.logX -= 1.0 / n_live
        self.n_dead += 1

    def copy(self):
        a = Accumulator()
        a.logZ, a.logX, a.H, a.n_dead = self.logZ, self.logX, self.H, self.n_dead
        return a


def log_evidence(logL_seq, nlive_seq):
    acc = Accumulator()
    for L, n in zip(logL_seq, nlive_seq):
        acc.add(float(L), int(n))
    return acc


def simulated_error(logL_seq, nlive_seq, seed: int, n_replays: int = 200):
    """Std (ddof = 1) of ln Z over replays of the shrinkage sequence."""
    logL = np.asarray(logL_seq, float)
    nl = np.asarray(nlive_seq, float)
    N = logL.size
    idx = np.arange(N, dtype=np.uint64)
    out = np.empty(n_replays)
    for s in range(n_replays):
        u = philox.uniform(seed, philox.PURPOSE_ERR, 0, s, idx, 0)
        lnt = np.log(u) / nl
        logX = np.cumsum(lnt)
        logX_prev = np.concatenate([[0.0], logX[:-1]])
        logw = logX_prev + np.log(-np.expm1(lnt))
        out[s] = lse(logL + logw)
    return float(np.std(out, ddof=1)), out
