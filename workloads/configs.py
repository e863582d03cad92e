"""Workload definitions: sizes, grid extents, prior boxes and fiducial values.

Parameter conventions follow Table 1 of arXiv:2509.13307 (priors and fiducial
values of the cosmic-shear model) and its Appendix A (tomographic bins,
chi-grid uniform in scale factor from a=1 to a_min).  The 5-bin / 39-parameter
layout and the synthetic stand-ins (random-init emulator, noise templates) are
the readings recorded in the design notes; none of this module computes any
part of the method.
"""

from __future__ import annotations

from dataclasses import dataclass, field, replace
from typing import Optional

# Full shear parameter vector, in this order, followed by D_z[i], m[i], b[t].
SHEAR_BASE_NAMES = ("omega_b", "omega_cdm", "h", "n_s", "ln10As", "w0", "wa",
                    "c_min", "eta0", "A_IA", "eta_IA")

# (kind, a, b, fiducial): kind "U" = uniform on [a, b]; "N" = Gaussian mean a, sd b.
# Table 1 of the paper for the first nine; A_IA/eta_IA per the 2-parameter
# intrinsic-alignment reading; D_z, m per Table 1 (m's 0.02 read as a standard
# deviation); noise-template amplitudes b ~ N(0, 1).
_BASE_PRIORS = {
    "omega_b": ("U", 0.01875, 0.02625, 0.02242),
    "omega_cdm": ("U", 0.05, 0.255, 0.11933),
    "h": ("U", 0.64, 0.982, 0.6766),
    "n_s": ("U", 0.84, 1.1, 0.9665),
    "ln10As": ("U", 1.61, 3.91, 3.047),
    "w0": ("U", -1.5, -0.5, -1.0),
    "wa": ("U", -0.5, 0.5, 0.0),
    "c_min": ("U", 2.0, 4.0, 2.6),
    "eta0": ("U", 0.5, 1.0, 0.7),
    "A_IA": ("U", -6.0, 6.0, 1.0),
    "eta_IA": ("U", -5.0, 5.0, 0.0),
}
_DZ_PRIOR = ("N", 0.0, 0.01, 0.0)
_M_PRIOR = ("N", 0.01, 0.02, 0.01)
_B_PRIOR = ("N", 0.0, 1.0, 0.0)


def shear_param_names(n_bins: int, n_tmpl: int) -> list[str]:
    return (list(SHEAR_BASE_NAMES) + [f"Dz_{i}" for i in range(n_bins)]
            + [f"m_{i}" for i in range(n_bins)] + [f"b_{t}" for t in range(n_tmpl)])


@dataclass(frozen=True)
class SamplerConfig:
    n_live: int
    n_delete: int                 # k: points deleted and chains evolved per iteration
    repeats: Optional[int] = None  # slice moves per chain; None -> 5 * d
    tol: float = 1e-3             # stop when ln(Z_dead + Z_live) - ln Z_dead < tol
    seed: int = 3
    max_iters: int = 1_000_000
    width: float = 1.0            # initial slice width along a unit-Mahalanobis direction
    step_cap: int = 100           # cap on stepping-out and on shrinkage steps
    ridge: float = 1e-12          # added to the live covariance diagonal

    def n_repeats(self, d: int) -> int:
        return 5 * d if self.repeats is None else self.repeats


@dataclass(frozen=True)
class ShearConfig:
    name: str
    n_bins: int
    nz_mean: tuple
    nz_sigma: tuple
    n_ell: int
    n_k: int
    n_z: int
    z_max: float
    n_chi: int
    a_min: float
    emu_hidden: tuple
    emu_inputs: tuple             # indices into the full parameter vector
    n_tmpl: int
    fixed: dict                   # name -> value for parameters held fixed
    cov_kind: str                 # "diag10" (10% of fiducial) or "knox"
    sampler: SamplerConfig
    ell_min: float = 30.0
    ell_max: float = 3000.0
    k_min: float = 1e-3
    k_max: float = 10.0
    n_gal_arcmin2: float = 6.0    # per bin (30 arcmin^-2 over 5 bins)
    sigma_e: float = 0.3
    f_sky: float = 0.35
    cov_rank: int = 5             # seeded dense low-rank addition to the Knox covariance
    cov_rank_amp: float = 0.05
    ia_pivot: float = 1.62        # A(z) = A_IA ((1+z)/ia_pivot)^eta_IA
    c1rho: float = 5e-14 * 2.775e11   # C_1 rho_cr (dimensionless, h cancels)
    emu_out_sigma: float = 0.05   # emulator output scale in dex about the mean table
    emu_bias_sd: float = 0.1
    emu_smooth_out: bool = False  # output layer a smooth function of (ln k, z) (Chebyshev bases), so
                                  # the coarse-z emulator is the full one evaluated at fewer z nodes
    coarse_z: Optional[int] = None    # if set: emulator on this many z nodes, interpolated to n_z
    z_interp: str = "catmull_rom"     # coarse -> fine z: "catmull_rom" or "linear" (the paper's)
    seed_emulator: int = 0
    seed_noise: int = 1
    seed_cov: int = 2

    @property
    def n_params(self) -> int:
        return len(SHEAR_BASE_NAMES) + 2 * self.n_bins + self.n_tmpl

    @property
    def param_names(self) -> list[str]:
        return shear_param_names(self.n_bins, self.n_tmpl)

    @property
    def n_pairs(self) -> int:
        return self.n_bins * (self.n_bins + 1) // 2

    @property
    def n_data(self) -> int:
        return self.n_pairs * self.n_ell

    @property
    def n_z_emu(self) -> int:
        return self.coarse_z if self.coarse_z else self.n_z

    @property
    def emu_dims(self) -> tuple:
        return (len(self.emu_inputs),) + tuple(self.emu_hidden) + (self.n_k * self.n_z_emu,)

    def priors(self):
        """List of (kind, a, b) per full parameter; kind "F" = fixed at a."""
        out = []
        for name in self.param_names:
            if name in _BASE_PRIORS:
                kind, a, b, fid = _BASE_PRIORS[name]
            elif name.startswith("Dz_"):
                kind, a, b, fid = _DZ_PRIOR
            elif name.startswith("m_"):
                kind, a, b, fid = _M_PRIOR
            else:
                kind, a, b, fid = _B_PRIOR
            if name in self.fixed:
                out.append(("F", float(self.fixed[name]), 0.0))
            else:
                out.append((kind, a, b))
        return out

    def fiducial(self):
        """Parameters the mock data is generated at (fixed values where fixed)."""
        out = []
        for name in self.param_names:
            if name in _BASE_PRIORS:
                fid = _BASE_PRIORS[name][3]
            elif name.startswith("Dz_"):
                fid = _DZ_PRIOR[3]
            elif name.startswith("m_"):
                fid = _M_PRIOR[3]
            else:
                fid = _B_PRIOR[3]
            out.append(float(self.fixed.get(name, fid)))
        return out

    @property
    def d_free(self) -> int:
        return sum(1 for p in self.priors() if p[0] != "F")

    def with_sampler(self, **kw) -> "ShearConfig":
        return replace(self, sampler=replace(self.sampler, **kw))


def _fixed_all_but_cosmo5(n_bins: int) -> dict:
    f = {"w0": -1.0, "wa": 0.0, "c_min": 2.6, "eta0": 0.7, "A_IA": 0.0, "eta_IA": 0.0}
    for i in range(n_bins):
        f[f"Dz_{i}"] = 0.0
        f[f"m_{i}"] = 0.0
    return f


def shear5(**sampler_kw) -> ShearConfig:
    """5-parameter cosmic-shear toy: 5->64->64->320 emulator (40 k x 8 z),
    2 bins, 10 ell, 129 chi nodes on a in [0.25, 1], diagonal covariance."""
    return ShearConfig(
        name="shear5", n_bins=2, nz_mean=(0.5, 1.0), nz_sigma=(0.2, 0.2),
        n_ell=10, n_k=40, n_z=8, z_max=3.0, n_chi=129, a_min=0.25,
        emu_hidden=(64, 64), emu_inputs=(0, 1, 2, 3, 4), n_tmpl=0,
        fixed=_fixed_all_but_cosmo5(2), cov_kind="diag10",
        sampler=SamplerConfig(n_live=100, n_delete=1, **sampler_kw))


def shear39(**sampler_kw) -> ShearConfig:
    """39-parameter w0-wa shear: 7 cosmology + 2 baryon + 2 IA + 5 D_z + 5 m +
    18 noise-template amplitudes; 5 bins x 20 ell (D = 300); emulator
    7->4x1024->(200 k x 50 z); 1025 chi nodes uniform in a on [1/6.02, 1]."""
    kw = dict(n_live=1000, n_delete=500)
    kw.update(sampler_kw)
    return ShearConfig(
        name="shear39", n_bins=5, nz_mean=(0.4, 0.7, 1.0, 1.3, 1.6),
        nz_sigma=(0.15,) * 5, n_ell=20, n_k=200, n_z=50, z_max=5.02,
        n_chi=1025, a_min=1.0 / 6.02, emu_hidden=(1024,) * 4,
        emu_inputs=(0, 1, 2, 3, 4, 7, 8), n_tmpl=18, fixed={}, cov_kind="knox",
        emu_smooth_out=True, sampler=SamplerConfig(**kw))


def shear37_lcdm(**sampler_kw) -> ShearConfig:
    """The nested LCDM twin of shear39: w0 = -1 and wa = 0 held fixed."""
    c = shear39(**sampler_kw)
    return replace(c, name="shear37_lcdm", fixed={"w0": -1.0, "wa": 0.0})


def shear33(**sampler_kw) -> ShearConfig:
    """A 33-dimensional w0-wa variant: the last six template amplitudes fixed at 0."""
    c = shear39(**sampler_kw)
    return replace(c, name="shear33", fixed={f"b_{t}": 0.0 for t in range(12, 18)})


def shear_tiny(**sampler_kw) -> ShearConfig:
    """A small full-physics shear problem (all nuisance types active) sized so the
    CPU oracle runs in well under a second per evaluation; spans several GEMM
    tiles with ragged tails (hidden 192, output 24 k x 10 z = 240)."""
    kw = dict(n_live=64, n_delete=16)
    kw.update(sampler_kw)
    return ShearConfig(
        name="shear_tiny", n_bins=3, nz_mean=(0.5, 0.9, 1.3), nz_sigma=(0.2,) * 3,
        n_ell=6, n_k=24, n_z=10, z_max=4.0, n_chi=97, a_min=0.2,
        emu_hidden=(192, 192), emu_inputs=(0, 1, 2, 3, 4, 7, 8), n_tmpl=4,
        fixed={}, cov_kind="knox", sampler=SamplerConfig(**kw))


@dataclass(frozen=True)
class GaussConfig:
    """Isotropic Gaussian likelihood on the unit cube (uniform prior)."""
    name: str
    d: int
    mu: float = 0.5
    sigma: float = 0.05
    sampler: SamplerConfig = field(default_factory=lambda: SamplerConfig(n_live=100, n_delete=1))

    @property
    def d_free(self) -> int:
        return self.d

    def with_sampler(self, **kw) -> "GaussConfig":
        return replace(self, sampler=replace(self.sampler, **kw))


def gauss_test(d: int = 5, **sampler_kw) -> GaussConfig:
    kw = dict(n_live=100, n_delete=1)
    kw.update(sampler_kw)
    return GaussConfig(name=f"gauss{d}", d=d, sampler=SamplerConfig(**kw))


@dataclass(frozen=True)
class CMBConfig:
    """6-parameter CMB-like problem: emulator 6->4x512->3x2507 (TT, TE, EE on
    ell = 2..2508) with a dense seeded covariance."""
    name: str
    n_ell: int
    emu_hidden: tuple
    sampler: SamplerConfig
    # (omega_b, omega_cdm, h, tau, n_s, ln10As): Planck 2018 best fit
    fiducial: tuple = (0.02237, 0.1200, 0.6736, 0.0544, 0.9649, 3.044)
    box_frac: float = 0.2
    tau_range: tuple = (0.02, 0.12)
    nu_factor: int = 2            # Wishart degrees of freedom = nu_factor * D
    emu_out_sigma: float = 0.05
    emu_bias_sd: float = 0.1
    seed_emulator: int = 0
    seed_noise: int = 1
    seed_cov: int = 2

    @property
    def n_data(self) -> int:
        return 3 * self.n_ell

    @property
    def d_free(self) -> int:
        return 6

    @property
    def emu_dims(self) -> tuple:
        return (6,) + tuple(self.emu_hidden) + (self.n_data,)

    def priors(self):
        out = []
        for i, f in enumerate(self.fiducial):
            if i == 3:
                out.append(("U", self.tau_range[0], self.tau_range[1]))
            else:
                out.append(("U", f * (1 - self.box_frac), f * (1 + self.box_frac)))
        return out


def cmb6(n_ell: int = 2507, **sampler_kw) -> CMBConfig:
    kw = dict(n_live=500, n_delete=250)
    kw.update(sampler_kw)
    return CMBConfig(name="cmb6", n_ell=n_ell, emu_hidden=(512,) * 4,
                     sampler=SamplerConfig(**kw))


def cmb_tiny(**sampler_kw) -> CMBConfig:
    """A small CMB-like problem for parity tests: 40 multipoles (D = 120),
    emulator 6 -> 96 -> 80 -> 120, spanning several tiles with ragged tails."""
    kw = dict(n_live=60, n_delete=30)
    kw.update(sampler_kw)
    return CMBConfig(name="cmb_tiny", n_ell=40, emu_hidden=(96, 80), sampler=SamplerConfig(**kw))


def shear39_interp(**sampler_kw) -> ShearConfig:
    """shear39 with the emulator evaluated on 10 coarse z nodes, Catmull-Rom
    interpolated to the 50-node table (output 200 k x 10 z = 2000)."""
    return replace(shear39(**sampler_kw), name="shear39_interp", coarse_z=10)


def shear37_interp(**sampler_kw) -> ShearConfig:
    return replace(shear37_lcdm(**sampler_kw), name="shear37_interp", coarse_z=10)


def shear39_interp_linear(**sampler_kw) -> ShearConfig:
    """shear39 on 10 coarse z nodes linearly interpolated in z (the paper's
    interpolated-P(k) runs)."""
    return replace(shear39(**sampler_kw), name="shear39_interp_linear", coarse_z=10, z_interp="linear")


def uneven_runs():
    """The packed-runs workload: (model, dimension, n_live) for eight runs with
    k = n_live / 2, all on the interpolated emulator."""
    spec = [("lcdm", 250), ("w0wa", 500), ("lcdm", 1000), ("w0wa", 2000), ("w0wa33", 250),
            ("w0wa", 1000), ("lcdm", 500), ("w0wa", 250)]
    out = []
    for i, (model, n) in enumerate(spec):
        base = {"lcdm": shear37_interp, "w0wa": shear39_interp,
                "w0wa33": lambda **kw: replace(shear39_interp(**kw), name="shear33_interp",
                                               fixed={f"b_{t}": 0.0 for t in range(12, 18)})}[model]
        out.append(base(n_live=n, n_delete=n // 2, seed=3 + i))
    return out
