"""Pins of the oracle's shear likelihood (App. A of the paper) against closed
forms, independent adaptive quadrature, library routines and invariants."""

import math

import numpy as np
import pytest
from scipy import integrate, linalg

import workloads as w
from oracle.shear import ShearOracle, C_KMS


@pytest.fixture(scope="module")
def tiny():
    inp = w.make_shear_inputs(w.shear_tiny())
    return inp, ShearOracle(inp)


@pytest.fixture(scope="module")
def big():
    inp = w.make_shear_inputs(w.shear39())
    return inp, ShearOracle(inp)


def theta_with(inp, **kw):
    t = np.array(inp["fiducial"], float)
    names = inp["param_names"]
    for k, v in kw.items():
        t[names.index(k)] = v
    return t


def E_ref(z, om, w0, wa):
    zp1 = 1 + z
    return math.sqrt(om * zp1 ** 3 + (1 - om) * zp1 ** (3 * (1 + w0 + wa)) * math.exp(-3 * wa * z / zp1))


def test_chi_einstein_de_sitter_closed_form(big):
    inp, o = big
    h = 0.7
    t = theta_with(inp, h=h, omega_b=0.02, omega_cdm=h * h - 0.02, w0=-1.0, wa=0.0)
    chi = o.chi_nodes(t)
    # 1 - 1/sqrt(1+z) written without cancellation at small z
    sq = np.sqrt(1 + o.z)
    exact = 2 * C_KMS / (100 * h) * o.z / (sq * (sq + 1))
    assert np.allclose(chi[1:], exact[1:], rtol=1e-13, atol=0)
    assert chi[0] == 0.0


@pytest.mark.parametrize("w0,wa", [(-1.0, 0.0), (-0.8, 0.3), (-1.3, -0.4)])
def test_chi_against_adaptive_quadrature(big, w0, wa):
    inp, o = big
    t = theta_with(inp, w0=w0, wa=wa)
    h = t[2]
    om = (t[0] + t[1]) / h ** 2
    chi = o.chi_nodes(t)
    for n in [1, 17, 300, 700, 1024]:
        ref = C_KMS / (100 * h) * integrate.quad(lambda z: 1 / E_ref(z, om, w0, wa), 0, o.z[n],
                                                 epsabs=0, epsrel=1e-13, limit=200)[0]
        assert abs(chi[n] / ref - 1) < 1e-12


def test_growth_einstein_de_sitter_is_a(big):
    inp, o = big
    h = 0.7
    t = theta_with(inp, h=h, omega_b=0.02, omega_cdm=h * h - 0.02, w0=-1.0, wa=0.0)
    D = o.growth_nodes(t)
    assert np.allclose(D, o.a, rtol=1e-13, atol=0)


def test_growth_converges_to_integral_second_order():
    # ln D(a) = -int_a^1 Omega_m(a')^gamma dln a': trapezoid on the grid vs quad,
    # error O(N^-2): halving the spacing must cut it ~4x.
    errs = []
    for n_chi in (257, 513):
        cfg = w.shear39()
        from dataclasses import replace
        inp = w.make_shear_inputs(replace(cfg, n_chi=n_chi))
        o = ShearOracle(inp, data=np.zeros(cfg.n_data), cov=np.eye(cfg.n_data))
        t = theta_with(inp, w0=-0.9, wa=0.2)
        h = t[2]
        om = (t[0] + t[1]) / h ** 2
        w0, wa = t[5], t[6]
        gamma = 0.55 + 0.05 * (1 + w0 + 0.5 * wa)
        f = lambda a: (om * a ** -3 / E_ref(1 / a - 1, om, w0, wa) ** 2) ** gamma / a
        D = o.growth_nodes(t)
        n = n_chi - 1
        ref = math.exp(-integrate.quad(f, o.a[n], 1.0, epsrel=1e-13)[0])
        errs.append(abs(D[n] / ref - 1))
    assert errs[1] < 1e-5
    assert 3.0 < errs[0] / errs[1] < 5.0


def _n_chi_continuous(inp, t, i):
    """Normalised n_i(chi) as a function of z, by adaptive quadrature."""
    h, om, w0, wa = t[2], (t[0] + t[1]) / t[2] ** 2, t[5], t[6]
    zmax = 1.0 / inp["a_min"] - 1.0
    dz = t[11 + i]
    mu, sg = inp["nz_mean"][i], inp["nz_sigma"][i]
    nz = lambda z: math.exp(-0.5 * ((z - dz - mu) / sg) ** 2)
    norm = integrate.quad(nz, 0, zmax, epsrel=1e-13, limit=200)[0]
    return lambda z: nz(z) / norm * (100 * h / C_KMS) * E_ref(z, om, w0, wa), zmax


def test_shear_window_against_quadrature():
    """Eq. 5 by nested adaptive quadrature in z vs the oracle's trapezoid sums on
    two grids (97 and 385 nodes, same a-values): the error must fall at second
    order and be small on the fine grid."""
    from dataclasses import replace
    errs = {}
    for n_chi, step in ((97, 1), (385, 4)):
        cfg = replace(w.shear_tiny(), n_chi=n_chi)
        inp = w.make_shear_inputs(cfg)
        o = ShearOracle(inp, data=np.zeros(cfg.n_data), cov=np.eye(cfg.n_data))
        t = theta_with(inp, A_IA=0.0, Dz_1=0.02)
        h, om, w0, wa = t[2], (t[0] + t[1]) / t[2] ** 2, t[5], t[6]
        chi = o.chi_nodes(t)
        E = o.E_of_z(o.z, om, w0, wa)
        W, _omega = o.windows(t, chi, E, o.growth_nodes(t), o.nz_chi(t, E))
        chi_of_z = lambda z: C_KMS / (100 * h) * integrate.quad(
            lambda x: 1 / E_ref(x, om, w0, wa), 0, z, epsrel=1e-13)[0]
        for i in range(o.nb):
            nfun, zmax = _n_chi_continuous(inp, t, i)
            for n0 in [5, 20, 48, 80]:
                n = n0 * step
                zn, cn = o.z[n], chi[n]
                # int_chi^chiH n(chi')(chi'-chi)/chi' dchi' in z: n(z) dchi/dz (1 - chi/chi(z))
                integ = integrate.quad(
                    lambda z: nfun(z) * C_KMS / (100 * h) / E_ref(z, om, w0, wa)
                    * (1 - cn / chi_of_z(z)), zn, zmax, epsrel=1e-11, limit=200)[0]
                ref = 1.5 * om * (100 * h / C_KMS) ** 2 * cn / o.a[n] * integ
                if abs(W[i, n]) > 1e-6 * np.abs(W[i]).max():   # skip the far tail
                    errs.setdefault((i, n0), []).append(abs(W[i, n] / ref - 1))
    assert len(errs) >= 8
    for key, (e_coarse, e_fine) in errs.items():
        # trapezoid error O(h^2): a 4x finer grid cuts it ~16x
        assert e_fine < 2e-2, (key, e_fine)
        assert e_fine < e_coarse / 10 or e_fine < 1e-7, (key, e_coarse, e_fine)


def test_ia_window_sign_and_scaling(tiny):
    """W^I (Eq. 6) is linear in A_IA, negative for A_IA > 0, and scales as
    ((1+z)/1.62)^eta: compare windows at two A_IA and two eta values."""
    inp, o = tiny
    def Wset(**kw):
        t = theta_with(inp, **kw)
        _h, om, w0, wa = o.cosmo(t)
        chi = o.chi_nodes(t)
        E = o.E_of_z(o.z, om, w0, wa)
        return o.windows(t, chi, E, o.growth_nodes(t), o.nz_chi(t, E))[0]
    W0 = Wset(A_IA=0.0, eta_IA=0.0)
    W1 = Wset(A_IA=1.0, eta_IA=0.0)
    W2 = Wset(A_IA=2.0, eta_IA=0.0)
    We = Wset(A_IA=1.0, eta_IA=1.5)
    WI1 = W1 - W0
    atol = 1e-12 * np.abs(W0).max()   # differences of windows cancel to round-off of W^gamma
    assert np.allclose(W2 - W0, 2 * WI1, rtol=1e-9, atol=atol)
    assert np.all(WI1[:, 1:] <= 0)
    ratio = ((1 + o.z) / 1.62) ** 1.5
    mask = np.abs(WI1) > 1e-4 * np.abs(WI1).max()
    assert np.allclose(((We - W0) / np.where(mask, WI1, 1))[mask], np.broadcast_to(ratio, WI1.shape)[mask],
                       rtol=1e-8)


def test_limber_constant_power_converges():
    """Eq. 4 with a constant P and pure lensing windows (A_IA = 0, so the
    integrand W W / chi^2 stays finite at chi -> 0): the sums on grids of 97,
    193 and 385 nodes must converge to a common limit.  Leaving out the chi = 0
    node (finite lensing integrand there, singular IA term) makes the rule
    first order: e(h) ~ c h gives e2 / e1 = (1/2 - 1/4) / (1 - 1/4) = 1/3."""
    vals = []
    for n_chi in (97, 193, 385):
        from dataclasses import replace
        cfg = replace(w.shear_tiny(), n_chi=n_chi)
        inp = w.make_shear_inputs(cfg)
        o = ShearOracle(inp, data=np.zeros(cfg.n_data), cov=np.eye(cfg.n_data))
        t = theta_with(inp, A_IA=0.0)
        _h, om, w0, wa = o.cosmo(t)
        chi = o.chi_nodes(t)
        E = o.E_of_z(o.z, om, w0, wa)
        W, omega = o.windows(t, chi, E, o.growth_nodes(t), o.nz_chi(t, E))
        Pl = np.ones((o.n_ell, o.N))
        vals.append(o.limber(W, omega, chi, Pl)[:, 0])
    e1 = np.abs(vals[0] - vals[2])
    e2 = np.abs(vals[1] - vals[2])
    assert np.all((e2 > 0.25 * e1) & (e2 < 0.45 * e1))
    assert np.max(e2 / np.abs(vals[2])) < 2e-2


def test_limber_brute_force_single_bin_tiny_grid():
    """Brute force on a 9-node grid: one bin, two ell, an explicit double loop
    over nodes for Eq. 5 and Eq. 4 with a bilinear log10 P table (reproduced
    exactly by the Catmull-Rom lookup)."""
    from dataclasses import replace
    cfg = replace(w.shear_tiny(), n_bins=1, nz_mean=(0.8,), nz_sigma=(0.3,), n_ell=2, n_chi=9,
                  n_tmpl=0)
    inp = w.make_shear_inputs(cfg)
    o = ShearOracle(inp, data=np.zeros(cfg.n_data), cov=np.eye(cfg.n_data))
    t = theta_with(inp, A_IA=0.0)
    h, om, w0, wa = t[2], (t[0] + t[1]) / t[2] ** 2, t[5], t[6]
    chi = o.chi_nodes(t)
    a = o.a
    N = 9
    da = (1 - inp["a_min"]) / (N - 1)
    wts = [da * (0.5 if n in (0, N - 1) else 1.0) for n in range(N)]
    Ez = [E_ref(1 / a[n] - 1, om, w0, wa) for n in range(N)]
    nz = [math.exp(-0.5 * ((1 / a[n] - 1 - t[11] - 0.8) / 0.3) ** 2) for n in range(N)]
    norm = sum(wts[n] * nz[n] / a[n] ** 2 for n in range(N))
    nchi = [nz[n] / norm * (100 * h / C_KMS) * Ez[n] for n in range(N)]
    om_w = [wts[n] * (C_KMS / (100 * h)) / (a[n] ** 2 * Ez[n]) for n in range(N)]
    Wg = [0.0] * N
    for n in range(1, N):
        s = 0.0
        for m in range(n, N):
            s += om_w[m] * nchi[m] * (chi[m] - chi[n]) / chi[m]
        Wg[n] = 1.5 * om * (100 * h / C_KMS) ** 2 * chi[n] / a[n] * s
    # bilinear table in (ln k, z)
    lnk = np.linspace(o.lnk_min, o.lnk_max, o.n_k)
    zt = np.linspace(0, o.z_max, o.n_z)
    T = 2.0 - 0.3 * (lnk[None, :] - lnk[0]) + 0.1 * zt[:, None] + 0.02 * zt[:, None] * lnk[None, :]
    Pl = o.lookup(T, chi)
    for l, ell in enumerate(o.ell):
        ref = 0.0
        for n in range(1, N):
            s = min(max(math.log((ell + 0.5) / chi[n]), o.lnk_min), o.lnk_max)
            zz = 1 / a[n] - 1
            lp = 2.0 - 0.3 * (s - lnk[0]) + 0.1 * zz + 0.02 * zz * s
            assert abs(Pl[l, n] / 10 ** lp - 1) < 1e-12
            ref += om_w[n] * Wg[n] ** 2 / chi[n] ** 2 * 10 ** lp
        E = o.E_of_z(o.z, om, w0, wa)
        W, omega = o.windows(t, chi, E, o.growth_nodes(t), o.nz_chi(t, E))
        C = o.limber(W, omega, chi, Pl)
        assert abs(C[0, l] / ref - 1) < 1e-12


def test_lookup_reproduces_quadratics_in_interior(tiny):
    inp, o = tiny
    lnk = np.linspace(o.lnk_min, o.lnk_max, o.n_k)
    zt = np.linspace(0, o.z_max, o.n_z)
    f = lambda s, z: 0.3 * s * s - 0.2 * s * z + 0.1 * z * z + 0.5 * s - z + 1.0
    T = f(lnk[None, :], zt[:, None])
    P = o.pad_table(T)
    rng = np.random.default_rng(5)
    for _ in range(200):
        s = rng.uniform(lnk[1], lnk[-2])
        z = rng.uniform(zt[1], zt[-2])
        ik, tk = o.bracket(s, o.lnk_min, o.dlnk, o.n_k)
        jz, tz = o.bracket(z, 0.0, o.dz, o.n_z)
        wk, wz = o.catmull_rom_weights(tk), o.catmull_rom_weights(tz)
        v = sum(wz[p] * wk[q] * P[jz + p, ik + q] for p in range(4) for q in range(4))
        assert abs(v - f(s, z)) < 1e-12
    # at the nodes the interpolant is the table value
    for ik in range(0, o.n_k - 1, 5):
        for jz in range(0, o.n_z - 1, 3):
            wk, wz = o.catmull_rom_weights(0.0), o.catmull_rom_weights(0.0)
            v = sum(wz[p] * wk[q] * P[jz + p, ik + q] for p in range(4) for q in range(4))
            assert v == pytest.approx(T[jz, ik], abs=1e-14)


def test_emulator_small_signal_jacobian(tiny):
    """Around x = 0 the emulator is y ~ y0 + sigma J x with
    J = W_L diag(1 - h_{L-1}^2) W_{L-1} ... diag(1 - h_1^2) W_1: a central
    difference of the oracle's forward must match that matrix chain."""
    inp, o = tiny
    Ws, bs = inp["emu_W"], inp["emu_b"]
    hs = []
    h = np.zeros(Ws[0].shape[1])
    for l in range(len(Ws) - 1):
        h = np.tanh(Ws[l] @ h + bs[l])
        hs.append(h)
    J = Ws[0]
    for l in range(1, len(Ws)):
        J = Ws[l] @ (np.diag(1 - hs[l - 1] ** 2) @ J)
    rng = np.random.default_rng(3)
    x = rng.standard_normal(Ws[0].shape[1])
    eps = 1e-5
    t = np.array(inp["fiducial"], float)
    idx = inp["emu_inputs"]
    def emu_at(xn):
        tt = t.copy()
        tt[idx] = inp["emu_in_center"] + inp["emu_in_scale"] * xn
        return o.emulator(tt).reshape(-1)
    fd = (emu_at(eps * x) - emu_at(-eps * x)) / (2 * eps)
    assert np.allclose(fd, inp["emu_out_sigma"] * (J @ x), rtol=1e-6, atol=1e-9)


def test_chi2_identity_covariance_and_triangular_solve(tiny):
    inp, o = tiny
    t = theta_with(inp)
    m = o.model(t)
    rng = np.random.default_rng(1)
    d = m + 1e-10 * rng.standard_normal(o.D)
    oi = ShearOracle(inp, data=d, cov=np.eye(o.D))
    assert oi.chi2(t) == pytest.approx(np.sum((d - oi.model(t)) ** 2), rel=1e-13)
    r = rng.standard_normal(o.D)
    y = o.forward_subst(r)
    assert np.allclose(y, linalg.solve_triangular(o.L, r, lower=True), rtol=1e-11, atol=1e-6)
    sign, logdet = np.linalg.slogdet(2 * np.pi * o.cov)
    assert sign > 0
    assert o.c0 == pytest.approx(-0.5 * logdet, rel=1e-12)


def test_multiplicative_bias_and_templates_are_exact(tiny):
    inp, o = tiny
    t0 = theta_with(inp, **{f"m_{i}": 0.0 for i in range(o.nb)})
    mvals = [0.03, -0.02, 0.05]
    t1 = theta_with(inp, **{f"m_{i}": mvals[i] for i in range(o.nb)})
    m0 = o.model(t0, with_templates=False).reshape(o.n_pairs, o.n_ell)
    m1 = o.model(t1, with_templates=False).reshape(o.n_pairs, o.n_ell)
    for p, (i, j) in enumerate(o.pairs):
        assert np.allclose(m1[p], (1 + mvals[i]) * (1 + mvals[j]) * m0[p], rtol=1e-13)
    b = np.arange(1, o.n_tmpl + 1) * 0.3
    tb = t0.copy()
    tb[11 + 2 * o.nb:] = b
    sig = np.sqrt(np.diag(o.cov))
    assert np.allclose(o.model(tb) - o.model(t0), 0.1 * sig * (inp["tmpl_g"] @ b), rtol=1e-9, atol=1e-25)


def test_knox_covariance_structure(tiny):
    inp, o = tiny
    C = o.cov
    assert np.allclose(C, C.T, rtol=1e-14, atol=0)
    assert np.all(np.linalg.eigvalsh(C) > 0)


def test_complex_step_matches_central_differences(tiny):
    inp, o = tiny
    t = np.array(inp["fiducial"], float)
    rng = np.random.default_rng(9)
    t = t + 0.01 * np.abs(t + 0.1) * rng.standard_normal(t.size)
    g = o.grad_complex_step(t)
    for i in range(t.size):
        hstep = 1e-5 * max(abs(t[i]), 1e-2)
        tp, tm = t.copy(), t.copy()
        tp[i] += hstep
        tm[i] -= hstep
        fd = (o.loglike(tp) - o.loglike(tm)) / (2 * hstep)
        assert abs(fd - g[i]) <= 1e-5 * max(abs(g[i]), 1.0), (i, fd, g[i])


def test_bf16_rounding_matches_library_conversion():
    import torch
    rng = np.random.default_rng(12)
    a = np.concatenate([rng.standard_normal(2000) * 10.0 ** rng.integers(-6, 6, 2000),
                        [1.0, 1.00390625, 1.005859375, -0.0, 65504.0]])
    ref = torch.tensor(a, dtype=torch.float32).to(torch.bfloat16).double().numpy()
    assert np.array_equal(ShearOracle.to_bf16(a), ref)


def test_zinterp_catmull_rom_and_linear():
    """Coarse-z interpolation: Catmull-Rom reproduces linear functions of z
    everywhere and quadratics away from the edges; linear interpolation
    reproduces linear functions and the coarse values at the coarse nodes."""
    from dataclasses import replace as dc_replace
    for mode in ("catmull_rom", "linear"):
        cfg = dc_replace(w.shear_tiny(), coarse_z=5, z_interp=mode)
        inp = w.make_shear_inputs(cfg)
        o = ShearOracle.__new__(ShearOracle)   # only the grid attributes zinterp reads
        o.inp, o.n_z, o.n_k, o.z_max = inp, inp["n_z"], inp["n_k"], inp["z_max"]
        zc = np.linspace(0.0, o.z_max, 5)
        zf = np.linspace(0.0, o.z_max, o.n_z)
        lin = (1.5 + 0.7 * zc)[:, None] * np.ones((1, o.n_k))
        assert np.allclose(o.zinterp(lin), (1.5 + 0.7 * zf)[:, None] * np.ones((1, o.n_k)), rtol=1e-13, atol=1e-13)
        if mode == "catmull_rom":
            q = (zc ** 2)[:, None] * np.ones((1, o.n_k))
            interior = (zf >= zc[1]) & (zf <= zc[-2])
            assert np.allclose(o.zinterp(q)[interior], (zf[interior] ** 2)[:, None], rtol=1e-12, atol=1e-12)
        else:
            rng = np.random.default_rng(3)
            T = rng.standard_normal((5, o.n_k))
            out = o.zinterp(T)
            for i, z in enumerate(zc):
                j = np.argmin(np.abs(zf - z))
                if abs(zf[j] - z) < 1e-12:
                    assert np.allclose(out[j], T[i], rtol=0, atol=1e-14)
