"""Seeded synthetic inputs.

Every random quantity the likelihood setup needs is drawn here with numpy's
seeded generators and handed, as plain arrays, to both the CUDA path and the
CPU oracle.  Random numbers the nested sampler itself draws are not here: each
side generates them from the counter-based Philox4x32-10 definition.

The emulator is a stand-in for the trained CosmoPower-JAX networks the paper
uses (Sec. 2.5, App. A): a random-init MLP with weights N(0, 1/fan_in), inputs
standardised over the prior box and outputs de-standardised as
mean_table + sigma * y, where mean_table is a smooth synthetic log10 P(k, z)
shape (below).  That shape is a fixed input table, not part of the method.
"""

from __future__ import annotations

import numpy as np

from .configs import ShearConfig, GaussConfig, CMBConfig

ARCMIN2_PER_SR = (180.0 * 60.0 / np.pi) ** 2


def log_grid(lo: float, hi: float, n: int) -> np.ndarray:
    """n values log-spaced on [lo, hi] (endpoints included)."""
    return lo * (hi / lo) ** (np.arange(n) / (n - 1))


def _synthetic_log10_pk(lnk: np.ndarray, z: np.ndarray) -> np.ndarray:
    """A smooth, positive stand-in for log10 P(k, z) [Mpc^3]: a broken power law
    (slope 0.96 below k ~ 0.015/Mpc, about -1.24 above) times a growth-like
    factor (1+z)^-1.6.  Returned with shape (len(z), len(lnk))."""
    k = np.exp(lnk)
    q = k / 0.015
    p = 5.36e4 * q ** 0.96 / (1.0 + q * q) ** 1.1
    g2 = (1.0 + z) ** -1.6
    return np.log10(p[None, :] * g2[:, None])


def _mlp_weights(rng: np.random.Generator, dims, bias_sd: float):
    Ws, bs = [], []
    for fan_in, fan_out in zip(dims[:-1], dims[1:]):
        Ws.append(rng.standard_normal((fan_out, fan_in)) / np.sqrt(fan_in))
        bs.append(bias_sd * rng.standard_normal(fan_out))
    return Ws, bs


def _chebyshev(s: np.ndarray, n: int) -> np.ndarray:
    """T_0 .. T_{n-1} at s in [-1, 1], shape (len(s), n)."""
    return np.cos(np.arange(n)[None, :] * np.arccos(np.clip(s, -1.0, 1.0))[:, None])


def _smooth_output_layer(rng: np.random.Generator, n_k: int, z_nodes: np.ndarray, z_max: float, fan_in: int,
                         bias_sd: float, n_zb: int = 4, n_kb: int = 16):
    """Output layer whose rows vary smoothly over the (ln k, z) table:
    W[(jz, ik), :] = sum_{m < n_zb, q < n_kb} c_mq T_m(s_z) T_q(s_k) V[m, q, :],
    s_z = 2 z / z_max - 1, s_k = 2 ik / (n_k - 1) - 1, V ~ N(0, 1/fan_in),
    c_mq = 2^-m / (1 + q / 4), rescaled so the rows have variance 1/fan_in on
    average; the bias likewise with scalar coefficients.  A real P(k, z) is
    smooth in both variables (slow, growth-like variation in z); with this
    layer the emulator on a coarser z grid is the same function evaluated at
    fewer z nodes (the draws V do not depend on the z grid)."""
    V = rng.standard_normal((n_zb, n_kb, fan_in)) / np.sqrt(fan_in)
    vb = rng.standard_normal((n_zb, n_kb)) * bias_sd
    c = (0.5 ** np.arange(n_zb))[:, None] / (1.0 + np.arange(n_kb)[None, :] / 4.0)
    Tz = _chebyshev(2.0 * np.asarray(z_nodes) / z_max - 1.0, n_zb)
    Tk = _chebyshev(2.0 * np.arange(n_k) / (n_k - 1) - 1.0, n_kb)
    # normalisation over the fine reference grid (independent of z_nodes)
    zr = np.linspace(0.0, z_max, 50)
    Tzr = _chebyshev(2.0 * zr / z_max - 1.0, n_zb)
    norm = np.sqrt(np.mean((Tzr ** 2) @ (c ** 2) @ (Tk ** 2).T))
    coef = np.einsum("zm,kq,mq->zkmq", Tz, Tk, c / norm)          # (nz, nk, n_zb, n_kb)
    W = np.einsum("zkmq,mqf->zkf", coef, V).reshape(len(z_nodes) * n_k, fan_in)
    b = np.einsum("zkmq,mq->zk", coef, vb).reshape(-1)
    return W, b


def make_shear_inputs(cfg: ShearConfig) -> dict:
    """All inputs of a shear problem.  Emulator output ordering is z-major:
    output o = jz * n_k + ik, i.e. log10 P at (k_ik, z_jz)."""
    priors = cfg.priors()
    dims = cfg.emu_dims
    rng_e = np.random.default_rng(cfg.seed_emulator)
    if cfg.emu_smooth_out:
        Ws, bs = _mlp_weights(rng_e, dims[:-1], cfg.emu_bias_sd)
        Wo, bo = _smooth_output_layer(rng_e, cfg.n_k, np.linspace(0.0, cfg.z_max, cfg.n_z_emu), cfg.z_max,
                                      dims[-2], cfg.emu_bias_sd)
        Ws.append(Wo)
        bs.append(bo)
    else:
        Ws, bs = _mlp_weights(rng_e, dims, cfg.emu_bias_sd)

    # Emulator input standardisation over the prior box of each input parameter.
    centers, scales = [], []
    for idx in cfg.emu_inputs:
        kind, a, b = priors[idx]
        if kind == "U":
            centers.append(0.5 * (a + b))
            scales.append(0.5 * (b - a))
        elif kind == "N":
            centers.append(a)
            scales.append(3.0 * b)
        else:  # fixed input: map its value to 0
            centers.append(a)
            scales.append(1.0)

    lnk_min, lnk_max = np.log(cfg.k_min), np.log(cfg.k_max)
    lnk = np.linspace(lnk_min, lnk_max, cfg.n_k)
    z_emu = np.linspace(0.0, cfg.z_max, cfg.n_z_emu)
    mu = _synthetic_log10_pk(lnk, z_emu).reshape(-1)

    ell = log_grid(cfg.ell_min, cfg.ell_max, cfg.n_ell)
    r = (cfg.ell_max / cfg.ell_min) ** (1.0 / (cfg.n_ell - 1))
    delta_ell = ell * (np.sqrt(r) - 1.0 / np.sqrt(r))

    D = cfg.n_data
    rng_n = np.random.default_rng(cfg.seed_noise)
    noise_eps = rng_n.standard_normal(D)
    rng_c = np.random.default_rng(cfg.seed_cov)
    cov_V = rng_c.standard_normal((D, cfg.cov_rank))
    tmpl_g = rng_c.standard_normal((D, cfg.n_tmpl))

    return dict(
        kind="shear", name=cfg.name,
        n_params=cfg.n_params, param_names=cfg.param_names,
        priors=priors, fiducial=np.array(cfg.fiducial()),
        n_bins=cfg.n_bins, nz_mean=np.array(cfg.nz_mean, float),
        nz_sigma=np.array(cfg.nz_sigma, float),
        ell=ell, delta_ell=delta_ell,
        n_k=cfg.n_k, lnk_min=lnk_min, lnk_max=lnk_max,
        n_z=cfg.n_z, z_max=cfg.z_max, n_z_emu=cfg.n_z_emu, z_interp=cfg.z_interp,
        n_chi=cfg.n_chi, a_min=cfg.a_min,
        emu_W=Ws, emu_b=bs, emu_act="tanh",
        emu_inputs=np.array(cfg.emu_inputs, dtype=np.int32),
        emu_in_center=np.array(centers), emu_in_scale=np.array(scales),
        emu_out_mu=mu, emu_out_sigma=float(cfg.emu_out_sigma),
        n_tmpl=cfg.n_tmpl, tmpl_g=tmpl_g,
        ia_pivot=cfg.ia_pivot, c1rho=cfg.c1rho,
        cov_kind=cfg.cov_kind,
        n_gal_sr=cfg.n_gal_arcmin2 * ARCMIN2_PER_SR, sigma_e=cfg.sigma_e,
        f_sky=cfg.f_sky, cov_V=cov_V, cov_rank_amp=cfg.cov_rank_amp,
        noise_eps=noise_eps,
    )


def make_gauss_inputs(cfg: GaussConfig) -> dict:
    return dict(kind="gauss", name=cfg.name, n_params=cfg.d,
                priors=[("U", 0.0, 1.0)] * cfg.d, mu=cfg.mu, sigma=cfg.sigma)


def make_cmb_inputs(cfg: CMBConfig) -> dict:
    """CMB stand-in: emulator 6 -> hidden -> 3*n_ell with CosmoPower's
    sigmoid-linear activation f(x) = [g + (1-g) sigmoid(beta x)] x, per-unit
    g ~ U(0, 0.5) and beta ~ U(0.5, 1.5); outputs de-standardised as
    mu_ell + sigma_ell * y with a synthetic smooth spectrum mu_ell."""
    priors = cfg.priors()
    dims = cfg.emu_dims
    rng_e = np.random.default_rng(cfg.seed_emulator)
    Ws, bs = _mlp_weights(rng_e, dims, cfg.emu_bias_sd)
    act_g = [rng_e.uniform(0.0, 0.5, n) for n in dims[1:-1]]
    act_beta = [rng_e.uniform(0.5, 1.5, n) for n in dims[1:-1]]
    centers = np.array([0.5 * (p[1] + p[2]) for p in priors])
    scales = np.array([0.5 * (p[2] - p[1]) for p in priors])
    ell = np.arange(2, 2 + cfg.n_ell, dtype=float)
    # Smooth positive stand-ins for the TT, TE, EE spectra (muK^2), and a
    # per-multipole output scale.
    tt = 5e3 * (ell / 200.0) ** 0.2 / (1.0 + (ell / 1000.0) ** 2.5) / (ell * (ell + 1) / (2 * np.pi))
    te = 0.1 * tt * np.cos(ell / 150.0)
    ee = 0.05 * tt * (1.0 + 0.3 * np.sin(ell / 200.0))
    mu = np.concatenate([tt, te, ee])
    sig = cfg.emu_out_sigma * np.abs(np.concatenate([tt, tt * 0.1, ee]))
    D = cfg.n_data
    rng_n = np.random.default_rng(cfg.seed_noise)
    noise_eps = rng_n.standard_normal(D)
    # cosmic-variance TT mock: k d_ell / C_ell ~ chi^2 with k = 2 ell + 1
    tt_chi2 = rng_n.chisquare(2.0 * ell + 1.0)
    nu = cfg.nu_factor * D
    return dict(kind="cmb", name=cfg.name, n_params=6, priors=priors,
                fiducial=np.array(cfg.fiducial), emu_W=Ws, emu_b=bs,
                emu_act="sigmoid_linear", act_g=act_g, act_beta=act_beta,
                emu_inputs=np.arange(6), emu_in_center=centers, emu_in_scale=scales,
                emu_out_mu=mu, emu_out_sig=sig, ell=ell, n_data=D,
                noise_eps=noise_eps, wishart_nu=nu, seed_cov=cfg.seed_cov,
                cov_rel=0.1, tt_chi2=tt_chi2)


_WISHART_CACHE: dict = {}


def wishart_base(D: int, nu: int, seed: int) -> np.ndarray:
    """W = A A^T / nu with A ~ N(0, 1) of size D x nu (seeded), accumulated in
    column blocks of A: a dense SPD matrix with E[W] = I whose spectrum follows
    the Marchenko-Pastur law (condition number near ((1 + r)/(1 - r))^2,
    r = sqrt(D / nu)).  The CMB covariance is this matrix times a scale set
    from the fiducial model by each side.  Cached per process (the D = 7521
    case takes seconds)."""
    key = (int(D), int(nu), int(seed))
    if key not in _WISHART_CACHE:
        rng = np.random.default_rng(seed)
        W = np.zeros((D, D))
        blk = 1024
        for c0 in range(0, nu, blk):
            A = rng.standard_normal((D, min(blk, nu - c0)))
            W += A @ A.T
        W /= nu
        W = 0.5 * (W + W.T)
        _WISHART_CACHE.clear()
        _WISHART_CACHE[key] = W
    return _WISHART_CACHE[key]
