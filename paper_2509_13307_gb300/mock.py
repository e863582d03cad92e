"""Mock data and covariance for the shear problems (App. A: a multivariate
Gaussian likelihood with a simulated LSST-like covariance, n_gal = 30 arcmin^-2
over the bins, sigma_e = 0.3, f_sky = 0.35).  Host-side set-up code run once
per problem, fed by the library's own FP64 model vector (ns_model_batch)."""

from __future__ import annotations

import numpy as np


def pair_list(n_bins: int):
    return [(i, j) for i in range(n_bins) for j in range(i, n_bins)]


def diagonal_covariance(model_fid: np.ndarray, frac: float = 0.1) -> np.ndarray:
    """Diagonal covariance with standard deviation frac * |fiducial|."""
    return np.diag((frac * model_fid) ** 2)


def knox_covariance(model_fid, n_bins, ell, delta_ell, f_sky, shape_noise, V, rank_amp):
    """Gaussian covariance of tomographic spectra,
        Cov[(ij, l), (kl, l)] = (Ct_ik Ct_jl + Ct_il Ct_jk) / ((2 l + 1) dl f_sky),
    Ct_ij = C_ij + delta_ij sigma_e^2 / n_gal, block-diagonal in multipole, plus
    rank_amp * S (V V^T / r) S with S = diag(sqrt(diag Cov)) (dense low rank)."""
    pairs = pair_list(n_bins)
    n_ell = len(ell)
    Cm = model_fid.reshape(len(pairs), n_ell)
    Ct = np.zeros((n_ell, n_bins, n_bins))
    for p, (i, j) in enumerate(pairs):
        Ct[:, i, j] = Cm[p]
        Ct[:, j, i] = Cm[p]
    Ct[:, np.arange(n_bins), np.arange(n_bins)] += shape_noise
    norm = (2.0 * np.asarray(ell) + 1.0) * np.asarray(delta_ell) * f_sky
    D = len(pairs) * n_ell
    cov = np.zeros((D, D))
    I = np.array([p[0] for p in pairs])
    J = np.array([p[1] for p in pairs])
    for e in range(n_ell):
        blk = (Ct[e][I[:, None], I[None, :]] * Ct[e][J[:, None], J[None, :]]
               + Ct[e][I[:, None], J[None, :]] * Ct[e][J[:, None], I[None, :]]) / norm[e]
        idx = np.arange(len(pairs)) * n_ell + e
        cov[np.ix_(idx, idx)] = blk
    s = np.sqrt(np.diag(cov))
    cov = cov + rank_amp * (s[:, None] * (V @ V.T) / V.shape[1] * s[None, :])
    return cov
