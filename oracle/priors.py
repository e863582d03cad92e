"""Prior transform from the unit cube to physical parameters (Table 1 of the
paper: uniform U(a, b) and Gaussian N(mu, sigma) priors).  Test infrastructure
only.

Each free parameter takes one cube coordinate c in (0, 1):
    uniform  theta = a + (b - a) c
    Gaussian theta = mu + sigma * Phi^-1(c)
Fixed parameters are inserted at their values; the cube has one coordinate per
non-fixed parameter, in parameter order.
"""

from __future__ import annotations

import numpy as np

from .special import inv_normal_cdf


def free_indices(priors):
    return [i for i, p in enumerate(priors) if p[0] != "F"]


def cube_to_theta(priors, cube):
    """cube: (..., d_free) -> theta_full: (..., n_params)."""
    cube = np.asarray(cube, dtype=float)
    free = free_indices(priors)
    out = np.empty(cube.shape[:-1] + (len(priors),))
    f = 0
    for i, (kind, a, b) in enumerate(priors):
        if kind == "F":
            out[..., i] = a
            continue
        c = cube[..., f]
        f += 1
        if kind == "U":
            out[..., i] = a + (b - a) * c
        elif kind == "N":
            out[..., i] = a + b * inv_normal_cdf(c)
        else:
            raise ValueError(kind)
    assert f == len(free)
    return out


def theta_free_to_full(priors, theta_free):
    """Physical free parameters (..., d_free) -> full vector with fixed values."""
    theta_free = np.asarray(theta_free)
    out = np.empty(theta_free.shape[:-1] + (len(priors),), dtype=theta_free.dtype)
    f = 0
    for i, (kind, a, _b) in enumerate(priors):
        if kind == "F":
            out[..., i] = a
        else:
            out[..., i] = theta_free[..., f]
            f += 1
    return out
