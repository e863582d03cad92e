"""Cosmic-shear likelihood of arXiv:2509.13307, App. A, in plain FP64 NumPy.
Test infrastructure only.

Steps, each following the cited passage (names as in the paper):
  grid        N_chi nodes uniform in scale factor from a = 1 down to a_min
              (App. A, the paragraph after the nuisance list); trapezoid weights.
  background  E(z) of flat w0-wa (CPL) dark energy; comoving distance
              chi(z) = (c/H0) int_0^z dz'/E(z') by a 64-point Gauss-Legendre rule
              on [0, z] at every node; growth D(a) from
              ln D = -int_a^1 Omega_m(a')^gamma dln a' (trapezoid in ln a),
              gamma = 0.55 + 0.05 (1 + w0 + wa/2).
  n(z)        Gaussian source bins shifted n_i(z) -> n_i(z - D_z,i) (App. A,
              photometric-redshift item), normalised on the grid.
  windows     W^gamma (Eq. 5) by the direct double sum over nodes; W^I (Eq. 6)
              with A(z) = A_IA ((1+z)/1.62)^eta_IA and C_1 rho_cr = 0.013875;
              W^eps = W^gamma + W^I, which makes one Limber sum of W^eps W^eps
              equal to the four-term sum of Eq. 3.
  emulator    MLP stand-in for the CosmoPower P(k, z) emulator (Sec. 2.5).
  lookup      P(k = (ell + 1/2)/chi, z) (Eq. 4) by Catmull-Rom bicubic
              interpolation of log10 P in (ln k, z), ln k clamped to the table.
  limber      C_ij(ell) = sum_n w_n W_i W_j / chi_n^2 P (Eq. 4), the chi = 0
              node excluded.
  model       (1 + m_i)(1 + m_j) C_ij(ell) (App. A, multiplicative-bias item)
              plus linear noise templates T b.
  loglike     Gaussian: -1/2 |L^-1 (d - m)|^2 - sum ln L_aa - D/2 ln 2 pi, the
              whitening by explicit forward substitution.

Mock data and covariance (App. A: LSST-like Gaussian covariance with
sigma_e = 0.3, f_sky = 0.35) are built here from the oracle's own fiducial
model: a Knox-formula covariance plus a seeded low-rank term, or a diagonal at
10% of the fiducial, and data = model + L eps.

Complex inputs are supported (brackets and clamps use real parts) so that the
complex-step derivative of loglike is exact to round-off.
"""

from __future__ import annotations

import math

import numpy as np

from .priors import cube_to_theta, theta_free_to_full

C_KMS = 299792.458  # speed of light [km/s]
GL64_X, GL64_W = np.polynomial.legendre.leggauss(64)


def _re(x):
    return np.real(x)


class ShearOracle:
    def __init__(self, inp: dict, data=None, cov=None):
        self.inp = inp
        self.priors = inp["priors"]
        self.nb = int(inp["n_bins"])
        self.n_ell = len(inp["ell"])
        self.ell = np.asarray(inp["ell"], float)
        self.pairs = [(i, j) for i in range(self.nb) for j in range(i, self.nb)]
        self.n_pairs = len(self.pairs)
        self.D = self.n_pairs * self.n_ell
        self.n_tmpl = int(inp["n_tmpl"])
        # chi grid: N nodes uniform in a, node 0 at a = 1.
        N = int(inp["n_chi"])
        self.N = N
        self.da = (1.0 - inp["a_min"]) / (N - 1)
        self.a = 1.0 - self.da * np.arange(N)
        self.z = 1.0 / self.a - 1.0
        self.wa = np.full(N, self.da)
        self.wa[0] *= 0.5
        self.wa[-1] *= 0.5
        # emulator table grids
        self.n_k = int(inp["n_k"])
        self.lnk_min, self.lnk_max = float(inp["lnk_min"]), float(inp["lnk_max"])
        self.dlnk = (self.lnk_max - self.lnk_min) / (self.n_k - 1)
        self.n_z = int(inp["n_z"])
        self.z_max = float(inp["z_max"])
        self.dz = self.z_max / (self.n_z - 1)
        self.n_z_emu = int(inp["n_z_emu"])
        self.tmpl = None
        if data is None or cov is None:
            data, cov = self.make_mock()
        self.set_data(data, cov)

    # ----------------------------------------------------------- background
    @staticmethod
    def cosmo(theta):
        h = theta[2]
        om = (theta[0] + theta[1]) / (h * h)
        return h, om, theta[5], theta[6]

    @staticmethod
    def E_of_z(z, om, w0, wa):
        zp1 = 1.0 + z
        de = (1.0 - om) * zp1 ** (3.0 * (1.0 + w0 + wa)) * np.exp(-3.0 * wa * z / zp1)
        return np.sqrt(om * zp1 ** 3 + de)

    def chi_nodes(self, theta):
        """chi(z_n) by a 64-point Gauss-Legendre rule on [0, z_n] at each node."""
        h, om, w0, wa = self.cosmo(theta)
        zn = self.z[:, None]
        zz = 0.5 * zn * (GL64_X[None, :] + 1.0)
        integ = 1.0 / self.E_of_z(zz, om, w0, wa)
        return (C_KMS / (100.0 * h)) * 0.5 * self.z * np.sum(GL64_W[None, :] * integ, axis=1)

    def growth_nodes(self, theta):
        """D(a_n) normalised to D(1) = 1, trapezoid in ln a on the chi grid."""
        _h, om, w0, wa = self.cosmo(theta)
        E = self.E_of_z(self.z, om, w0, wa)
        om_a = om * (1.0 + self.z) ** 3 / (E * E)
        gamma = 0.55 + 0.05 * (1.0 + w0 + 0.5 * wa)
        f = om_a ** gamma
        lna = np.log(self.a)
        seg = 0.5 * (f[:-1] + f[1:]) * (lna[:-1] - lna[1:])
        lnD = -np.concatenate([[0.0 * seg[0]], np.cumsum(seg)])
        return np.exp(lnD)

    # ---------------------------------------------------------------- n(z)
    def nz_chi(self, theta, E):
        """n_i(chi_m): shifted Gaussian in z, normalised so int n_i dchi = 1 on the grid."""
        h = theta[2]
        nb = self.nb
        dzs = theta[11:11 + nb]
        mu = self.inp["nz_mean"]
        sg = self.inp["nz_sigma"]
        out = []
        for i in range(nb):
            raw = np.exp(-0.5 * ((self.z - dzs[i] - mu[i]) / sg[i]) ** 2)
            norm = np.sum(self.wa * raw / self.a ** 2)
            out.append(raw * (100.0 * h / C_KMS) * E / norm)
        return np.array(out)

    # ------------------------------------------------------------- windows
    def windows(self, theta, chi, E, D, nchi):
        """W^eps_i(chi_n) = W^gamma_i (Eq. 5, direct double sum) + W^I_i (Eq. 6)."""
        h, om, _w0, _wa = self.cosmo(theta)
        N = self.N
        omega = self.wa * (C_KMS / (100.0 * h)) / (self.a ** 2 * E)   # trapezoid weight in chi
        pref = 1.5 * om * (100.0 * h / C_KMS) ** 2
        # K[n, m] = (chi_m - chi_n)/chi_m for m >= n >= 1, else 0
        n_idx = np.arange(N)
        chi_safe = np.where(_re(chi) > 0, chi, 1.0)
        K = (chi[None, :] - chi[:, None]) / chi_safe[None, :]
        mask = (n_idx[None, :] >= n_idx[:, None]) & (n_idx[:, None] >= 1)
        K = np.where(mask, K, 0.0)
        A_IA, eta = theta[9], theta[10]
        amp = A_IA * ((1.0 + self.z) / self.inp["ia_pivot"]) ** eta
        W = []
        for i in range(self.nb):
            integ = K @ (omega * nchi[i])
            Wg = pref * chi / self.a * integ
            WI = -amp * self.inp["c1rho"] * om / D * nchi[i]
            W.append(Wg + WI)
        return np.array(W), omega

    # ------------------------------------------------------------ emulator
    @staticmethod
    def to_bf16(a):
        """Round to the nearest bfloat16 (ties to even) through float32, returned as float64."""
        f = np.asarray(a, dtype=np.float32).copy()
        u = f.view(np.uint32)
        u += np.uint32(0x7FFF) + ((u >> np.uint32(16)) & np.uint32(1))
        u &= np.uint32(0xFFFF0000)
        return u.view(np.float32).astype(np.float64)

    def emulator(self, theta, bf16=False, bf16_weights=False):
        """log10 P on the emulator's (z, k) grid, shape (n_z_emu, n_k).  With
        bf16=True the weights of layers >= 1 and every hidden activation are
        rounded to bfloat16 (arithmetic stays FP64): the model the tensor-core
        path computes, up to its FP32 accumulation order.  With
        bf16_weights=True only those weights are rounded (activations exact):
        the model whose gradient the split-bf16 adjoint computes, and a smooth
        function of theta, so complex-step differentiation goes through it."""
        inp = self.inp
        x = (theta[inp["emu_inputs"]] - inp["emu_in_center"]) / inp["emu_in_scale"]
        Ws, bs = inp["emu_W"], inp["emu_b"]
        rw = bf16 or bf16_weights
        h = x
        for l in range(len(Ws) - 1):
            W = self.to_bf16(Ws[l]) if (rw and l >= 1) else Ws[l]
            h = np.tanh(W @ h + bs[l])
            if bf16:
                h = self.to_bf16(h)
        Wl = self.to_bf16(Ws[-1]) if rw else Ws[-1]
        y = Wl @ h + bs[-1]
        t = inp["emu_out_mu"] + inp["emu_out_sigma"] * y
        return t.reshape(self.n_z_emu, self.n_k)

    @staticmethod
    def catmull_rom_weights(t):
        t2 = t * t
        t3 = t2 * t
        return (0.5 * (-t + 2.0 * t2 - t3), 0.5 * (2.0 - 5.0 * t2 + 3.0 * t3),
                0.5 * (t + 4.0 * t2 - 3.0 * t3), 0.5 * (-t2 + t3))

    @staticmethod
    def bracket(s, lo, step, n):
        """Cell index i in [0, n-2] and fraction t for s on a uniform grid."""
        u = (s - lo) / step
        i = np.clip(np.floor(_re(u)).astype(int), 0, n - 2)
        return i, u - i

    @staticmethod
    def pad_table(T):
        """Ghost rows/columns by linear extrapolation: p[-1] = 2 p[0] - p[1], p[n] = 2 p[n-1] - p[n-2]."""
        nz, nk = T.shape
        P = np.zeros((nz + 2, nk + 2), dtype=T.dtype)
        P[1:-1, 1:-1] = T
        P[0, 1:-1] = 2 * T[0] - T[1]
        P[-1, 1:-1] = 2 * T[-1] - T[-2]
        P[:, 0] = 2 * P[:, 1] - P[:, 2]
        P[:, -1] = 2 * P[:, -2] - P[:, -3]
        return P

    def zinterp(self, Tc):
        """Coarse-z emulator table -> the n_z table (coarse grid uniform on
        [0, z_max]): Catmull-Rom in z, or linear between the bracketing coarse
        nodes (inp["z_interp"] == "linear", the paper's interpolated P(k))."""
        nzc = Tc.shape[0]
        zf = np.linspace(0.0, self.z_max, self.n_z)
        if self.inp.get("z_interp", "catmull_rom") == "linear":
            u = zf / (self.z_max / (nzc - 1))
            i = np.clip(np.floor(_re(u)).astype(int), 0, nzc - 2)
            t = u - i
            return (1.0 - t)[:, None] * Tc[i] + t[:, None] * Tc[i + 1]
        P = self.pad_table(Tc)[:, 1:-1]
        j, t = self.bracket(zf, 0.0, self.z_max / (nzc - 1), nzc)
        w = self.catmull_rom_weights(t)
        out = np.zeros((self.n_z, self.n_k), dtype=Tc.dtype)
        for q in range(4):
            out += w[q][:, None] * P[j + q]
        return out

    def lookup(self, T, chi):
        """P(ell, n) for nodes n >= 1 (column 0 unused, set 0)."""
        P = self.pad_table(T)
        N = self.N
        lnchi = np.log(np.where(_re(chi[1:]) > 0, chi[1:], 1.0))
        jz, tz = self.bracket(self.z[1:], 0.0, self.dz, self.n_z)
        wz = self.catmull_rom_weights(tz)
        out = np.zeros((self.n_ell, N), dtype=np.result_type(T, chi))
        for l, ell in enumerate(self.ell):
            s = math.log(ell + 0.5) - lnchi
            s = np.where(_re(s) < self.lnk_min, self.lnk_min,
                         np.where(_re(s) > self.lnk_max, self.lnk_max, s))
            ik, tk = self.bracket(s, self.lnk_min, self.dlnk, self.n_k)
            wk = self.catmull_rom_weights(tk)
            v = 0.0
            for p in range(4):
                for q in range(4):
                    v = v + wz[p] * wk[q] * P[jz + p, ik + q]
            out[l, 1:] = 10.0 ** v
        return out

    # -------------------------------------------------------------- limber
    def limber(self, W, omega, chi, Pl):
        """C_p(ell) = sum_{n>=1} omega_n W_i(n) W_j(n) / chi_n^2 P(ell, n)."""
        chi2 = np.where(_re(chi) > 0, chi * chi, 1.0)
        q = np.where(np.arange(self.N) >= 1, omega / chi2, 0.0)
        C = np.zeros((self.n_pairs, self.n_ell), dtype=np.result_type(W, Pl))
        for p, (i, j) in enumerate(self.pairs):
            g = q * W[i] * W[j]
            for l in range(self.n_ell):
                C[p, l] = np.sum(g * Pl[l])
        return C

    # --------------------------------------------------------------- model
    def spectra(self, theta):
        """Tomographic C_ij(ell) (shape n_pairs x n_ell) at full parameters theta."""
        theta = np.asarray(theta)
        _h, om, w0, wa = self.cosmo(theta)
        chi = self.chi_nodes(theta)
        E = self.E_of_z(self.z, om, w0, wa)
        D = self.growth_nodes(theta)
        nchi = self.nz_chi(theta, E)
        W, omega = self.windows(theta, chi, E, D, nchi)
        T = self.emulator(theta)
        if self.n_z_emu != self.n_z:
            T = self.zinterp(T)
        Pl = self.lookup(T, chi)
        return self.limber(W, omega, chi, Pl)

    def model(self, theta, with_templates=True):
        theta = np.asarray(theta)
        C = self.spectra(theta)
        mb = theta[11 + self.nb:11 + 2 * self.nb]
        m = np.array([(1.0 + mb[i]) * (1.0 + mb[j]) * C[p] for p, (i, j) in enumerate(self.pairs)])
        m = m.reshape(-1)
        if with_templates and self.n_tmpl:
            b = theta[11 + 2 * self.nb:]
            m = m + self.tmpl @ b
        return m

    # --------------------------------------------------------- data / cov
    def make_mock(self):
        inp = self.inp
        fid = np.asarray(inp["fiducial"], float)
        mfid = self.model(fid, with_templates=False)
        if inp["cov_kind"] == "diag10":
            cov = np.diag((0.1 * mfid) ** 2)
        elif inp["cov_kind"] == "knox":
            cov = self.knox_cov(mfid)
        else:
            raise ValueError(inp["cov_kind"])
        L = np.linalg.cholesky(cov)
        data = mfid + L @ inp["noise_eps"]
        return data, cov

    def knox_cov(self, mfid):
        """Gaussian (Knox) covariance at the fiducial spectra with shape noise,
        plus a seeded dense low-rank term scaled to the diagonal."""
        inp = self.inp
        nb, nl = self.nb, self.n_ell
        Ct = np.zeros((nb, nb, nl))
        M = mfid.reshape(self.n_pairs, nl)
        for p, (i, j) in enumerate(self.pairs):
            Ct[i, j] = Ct[j, i] = M[p]
        noise = inp["sigma_e"] ** 2 / inp["n_gal_sr"]
        for i in range(nb):
            Ct[i, i] += noise
        cov = np.zeros((self.D, self.D))
        for p, (i, j) in enumerate(self.pairs):
            for q, (k, l) in enumerate(self.pairs):
                for e in range(nl):
                    v = (Ct[i, k, e] * Ct[j, l, e] + Ct[i, l, e] * Ct[j, k, e]) / (
                        (2.0 * self.ell[e] + 1.0) * inp["delta_ell"][e] * inp["f_sky"])
                    cov[p * nl + e, q * nl + e] = v
        V = inp["cov_V"]
        s = np.sqrt(np.diag(cov))
        cov = cov + inp["cov_rank_amp"] * (s[:, None] * (V @ V.T) / V.shape[1] * s[None, :])
        return cov

    def set_data(self, data, cov):
        self.data = np.asarray(data, float)
        self.cov = np.asarray(cov, float)
        self.L = np.linalg.cholesky(self.cov)
        self.c0 = -np.sum(np.log(np.diag(self.L))) - 0.5 * self.D * math.log(2.0 * math.pi)
        if self.n_tmpl:
            sig = np.sqrt(np.diag(self.cov))
            self.tmpl = 0.1 * sig[:, None] * self.inp["tmpl_g"]

    # ----------------------------------------------------------- likelihood
    def forward_subst(self, r):
        """Solve L y = r by explicit forward substitution."""
        L = self.L
        y = np.zeros(self.D, dtype=r.dtype)
        for a in range(self.D):
            y[a] = (r[a] - L[a, :a] @ y[:a]) / L[a, a]
        return y

    def chi2(self, theta):
        r = self.data - self.model(theta)
        y = self.forward_subst(r)
        return np.sum(y * y)

    def loglike_full(self, theta):
        return -0.5 * self.chi2(theta) + self.c0

    def loglike(self, theta_free):
        """Physical free parameters -> log L."""
        return self.loglike_full(theta_free_to_full(self.priors, np.asarray(theta_free)))

    def loglike_cube(self, cube):
        return self.loglike_full(cube_to_theta(self.priors, cube))

    def grad_complex_step(self, theta_free, h=1e-30):
        """d log L / d theta_free by the complex-step method (Squire & Trapp 1998)."""
        theta_free = np.asarray(theta_free, float)
        g = np.zeros_like(theta_free)
        for i in range(theta_free.size):
            t = theta_free.astype(complex)
            t[i] += 1j * h
            g[i] = np.imag(self.loglike(t)) / h
        return g
