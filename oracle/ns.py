"""Nested slice sampling with batched deletion, in plain Python/NumPy FP64.
Test infrastructure only.

Nested sampling (Sec. 2.1; Skilling 2006) keeps n live points drawn from the
prior; each iteration here deletes the k lowest (Sec. 2.2: "selecting k live
points with the lowest likelihoods ... evolving them ... in parallel") and
replaces each by a point drawn from the prior under the hard constraint
log L > L*, obtained by hit-and-run slice sampling (Sec. 2.1; Neal 2003).
The paper does not print the NSS internals; this follows the recorded reading:

  * work in the unit cube (every prior is uniform there after the transform);
  * sort live points by (log L, index); delete the first k; L* = log L of the
    k-th; the j-th deleted point is booked with n - j live points;
  * Sigma = covariance (ddof = 1) of all n live cube points before deletion,
    plus ridge * I; L_Sigma = chol(Sigma);
  * chain c starts from survivor floor(u (n - k)) in sorted order
    (u from Philox START), and makes R = 5 d slice moves;
  * a move draws z ~ N(0, I_d) (Philox DIR, Box-Muller) and slices along
    u = L_Sigma z / |z|, i.e. a direction of unit Mahalanobis length;
    stepping out with width w: l = -w u0, r = l + w (u0 from Philox STEPOUT),
    then l -= w while x + l u is inside, r += w while x + r u is inside
    (at most `step_cap` steps each); shrinkage: t = l + U (r - l)
    (U from Philox SHRINK, step s), accept if inside, else l = t if t < 0
    else r = t (at most `step_cap` steps; if exhausted the chain stays put);
  * "inside" = strictly inside the open unit cube AND log L > L*; a point
    outside the cube is rejected without a likelihood evaluation; a
    non-finite log L counts as outside;
  * chain c's final point replaces the c-th deleted slot;
  * stop when ln(Z + X mean(L_live)) - ln Z < tol; at the end the live points
    are added in ascending order with n, n-1, ..., 1 live points.
"""

from __future__ import annotations

import math
from dataclasses import dataclass, field

import numpy as np

from . import philox
from .evidence import Accumulator, simulated_error
from .special import lse

STATUS_SLICE_CAP = 1
STATUS_NONFINITE = 2


@dataclass
class IterRecord:
    it: int
    lstar: float
    deleted: np.ndarray           # live slots deleted, ascending (logL, idx)
    starts: np.ndarray            # live slot each chain started from
    evals: np.ndarray             # likelihood evaluations per chain
    new_x: np.ndarray
    new_logL: np.ndarray
    logZ: float
    logX: float
    H: float


@dataclass
class NestedSampler:
    loglike_cube: callable
    d: int
    n_live: int
    n_delete: int
    repeats: int
    seed: int
    tol: float = 1e-3
    width: float = 1.0
    step_cap: int = 100
    ridge: float = 1e-12
    it: int = 0
    status: int = 0
    n_evals: int = 0
    records: list = field(default_factory=list)

    @classmethod
    def from_config(cls, loglike_cube, d, sc):
        return cls(loglike_cube=loglike_cube, d=d, n_live=sc.n_live, n_delete=sc.n_delete,
                   repeats=sc.n_repeats(d), seed=sc.seed, tol=sc.tol, width=sc.width,
                   step_cap=sc.step_cap, ridge=sc.ridge)

    # ------------------------------------------------------------ helpers
    def _eval(self, x):
        v = float(self.loglike_cube(x))
        self.n_evals += 1
        if not math.isfinite(v):
            self.status |= STATUS_NONFINITE
            return -math.inf
        return v

    def initialise(self):
        n, d = self.n_live, self.d
        self.x = np.array([philox.init_point(self.seed, i, d) for i in range(n)])
        self.logL = np.array([self._eval(self.x[i]) for i in range(n)])
        self.acc = Accumulator()
        self.dead_x, self.dead_logL, self.dead_nlive = [], [], []
        self.it = 0

    def sorted_order(self):
        return np.lexsort((np.arange(self.n_live), self.logL))

    def live_cholesky(self):
        S = np.cov(self.x, rowvar=False, ddof=1).reshape(self.d, self.d)
        S = S + self.ridge * np.eye(self.d)
        return np.linalg.cholesky(S)

    def _inside(self, x, lstar, evals):
        if np.any(x <= 0.0) or np.any(x >= 1.0):
            return False, None
        v = self._eval(x)
        evals[0] += 1
        return (v > lstar), v

    def slice_chain(self, it, c, x, lx, lstar, Lc):
        """R slice moves of chain c from (x, lx); returns final point, log L, evals."""
        evals = [0]
        w = self.width
        cap = self.step_cap
        for m in range(self.repeats):
            z = philox.normals(self.seed, philox.PURPOSE_DIR, it, c, m, self.d)
            u = Lc @ (z / np.linalg.norm(z))
            u0 = philox.uniform_scalar(self.seed, philox.PURPOSE_STEPOUT, 0, it, c, m)
            l = -w * u0
            r = l + w
            nl = 0
            while nl < cap and self._inside(x + l * u, lstar, evals)[0]:
                l -= w
                nl += 1
            nr = 0
            while nr < cap and self._inside(x + r * u, lstar, evals)[0]:
                r += w
                nr += 1
            if nl == cap or nr == cap:
                self.status |= STATUS_SLICE_CAP
            accepted = False
            for s in range(cap):
                us = philox.uniform_scalar(self.seed, philox.PURPOSE_SHRINK, s, it, c, m)
                t = l + us * (r - l)
                xp = x + t * u
                ok, v = self._inside(xp, lstar, evals)
                if ok:
                    x, lx = xp, v
                    accepted = True
                    break
                if t < 0.0:
                    l = t
                else:
                    r = t
            if not accepted:
                self.status |= STATUS_SLICE_CAP
        return x, lx, evals[0]

    # --------------------------------------------------------- iterations
    def iterate(self):
        n, k, d = self.n_live, self.n_delete, self.d
        it = self.it
        order = self.sorted_order()
        deleted = order[:k]
        survivors = order[k:]
        lstar = float(self.logL[deleted[-1]])
        for j, s in enumerate(deleted):
            self.acc.add(float(self.logL[s]), n - j)
            self.dead_x.append(self.x[s].copy())
            self.dead_logL.append(float(self.logL[s]))
            self.dead_nlive.append(n - j)
        Lc = self.live_cholesky()
        new_x = np.empty((k, d))
        new_L = np.empty(k)
        starts = np.empty(k, dtype=int)
        evals = np.empty(k, dtype=int)
        for c in range(k):
            u = philox.uniform_scalar(self.seed, philox.PURPOSE_START, 0, it, c, 0)
            s = survivors[int(math.floor(u * (n - k)))]
            starts[c] = s
            new_x[c], new_L[c], evals[c] = self.slice_chain(
                it, c, self.x[s].copy(), float(self.logL[s]), lstar, Lc)
        for c in range(k):
            self.x[deleted[c]] = new_x[c]
            self.logL[deleted[c]] = new_L[c]
        self.records.append(IterRecord(it, lstar, deleted.copy(), starts, evals, new_x, new_L,
                                       self.acc.logZ, self.acc.logX, self.acc.H))
        self.it += 1

    def live_logZ(self):
        return self.acc.logX + lse(self.logL) - math.log(self.n_live)

    def converged(self):
        lz = self.acc.logZ
        if lz == -math.inf:
            return False
        tot = lse([lz, self.live_logZ()])
        return (tot - lz) < self.tol

    def run(self, max_iters=10 ** 9):
        for _ in range(max_iters):
            if self.converged():
                break
            self.iterate()
        return self

    # ------------------------------------------------------------ results
    def final_sequence(self):
        """Dead log L and live counts, with the live points appended."""
        order = self.sorted_order()
        n = self.n_live
        logL = list(self.dead_logL) + [float(self.logL[s]) for s in order]
        nl = list(self.dead_nlive) + [n - j for j in range(n)]
        return np.array(logL), np.array(nl)

    def evidence(self, n_replays=200):
        acc = self.acc.copy()
        order = self.sorted_order()
        n = self.n_live
        for j, s in enumerate(order):
            acc.add(float(self.logL[s]), n - j)
        logL, nl = self.final_sequence()
        err, _ = simulated_error(logL, nl, self.seed, n_replays)
        return dict(logZ=acc.logZ, logZ_err=err, logX=acc.logX, H=acc.H,
                    n_dead=acc.n_dead, skilling_err=math.sqrt(max(acc.H, 0.0) / n))
