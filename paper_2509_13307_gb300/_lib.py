"""ctypes binding of libgpuns.so: structures mirroring include/gpuns.h and the
exported functions with their argument types.  Argument marshalling only."""

from __future__ import annotations

import ctypes as C
import os

_PKG = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_PKG, "libgpuns.so")

NS_OK, NS_EINVAL, NS_ECUDA, NS_ENOMEM, NS_ETIMEOUT, NS_ESLICE, NS_ENONFINITE, NS_ENOTSUP = 0, -1, -2, -3, -4, -5, -6, -7
NS_BIT_SLICE_CAP, NS_BIT_NONFINITE, NS_BIT_TIMEOUT = 1, 2, 4
NS_KIND_GAUSS, NS_KIND_SHEAR, NS_KIND_CMB = 0, 1, 2
NS_ACT = {"tanh": 0, "sigmoid_linear": 1}
NS_SOLVE = {"fold": 0, "literal": 1}
NS_CMB_FORM = {"gauss": 0, "tt_cv": 1}
NS_PREC = {"fp64": 0, "fp32": 1, "bf16": 2, "bf16_f64chi2": 3}
NS_PRIOR = {"U": 0, "N": 1, "F": 2}

EXPORTS = ["ns_strerror", "ns_problem_create", "ns_problem_free", "ns_problem_dim", "ns_prior_transform",
           "loglike_batch", "ns_model_batch", "ns_emulator_batch", "ns_problem_status", "ns_problem_tiles", "ns_problem_fused", "loglike_grad_batch", "ns_init", "ns_step", "ns_evidence",
           "ns_live_points", "ns_dead_points", "ns_last_iteration", "ns_profile_stage", "ns_profile_read",
           "ns_evidence_noalloc", "ns_multi_init", "ns_multi_step", "ns_multi_run",
           "ns_multi_free", "ns_nuts_run", "ns_shard_evolve", "ns_shard_export", "ns_shard_insert",
           "ns_shard_range", "ns_free"]


class Prior(C.Structure):
    _fields_ = [("kind", C.c_int), ("a", C.c_double), ("b", C.c_double)]


class EmulatorDesc(C.Structure):
    _fields_ = [("n_layers", C.c_int), ("dims", C.POINTER(C.c_int)),
                ("W", C.POINTER(C.POINTER(C.c_double))), ("b", C.POINTER(C.POINTER(C.c_double))),
                ("activation", C.c_int), ("inputs", C.POINTER(C.c_int)),
                ("in_center", C.POINTER(C.c_double)), ("in_scale", C.POINTER(C.c_double)),
                ("out_mu", C.POINTER(C.c_double)), ("out_sigma", C.c_double),
                ("out_sigma_vec", C.POINTER(C.c_double)),
                ("act_g", C.POINTER(C.POINTER(C.c_double))), ("act_beta", C.POINTER(C.POINTER(C.c_double)))]


class ShearDesc(C.Structure):
    _fields_ = [("n_bins", C.c_int), ("nz_mean", C.POINTER(C.c_double)), ("nz_sigma", C.POINTER(C.c_double)),
                ("n_ell", C.c_int), ("ell", C.POINTER(C.c_double)),
                ("n_k", C.c_int), ("lnk_min", C.c_double), ("lnk_max", C.c_double),
                ("n_z", C.c_int), ("z_max", C.c_double), ("n_z_emu", C.c_int),
                ("n_chi", C.c_int), ("a_min", C.c_double), ("ia_pivot", C.c_double), ("c1rho", C.c_double),
                ("n_tmpl", C.c_int), ("tmpl", C.POINTER(C.c_double)), ("z_interp", C.c_int)]


class GaussDesc(C.Structure):
    _fields_ = [("mu", C.c_double), ("sigma", C.c_double)]


class CmbDesc(C.Structure):
    _fields_ = [("solve", C.c_int), ("form", C.c_int), ("n_tt", C.c_int), ("ell", C.POINTER(C.c_double))]


class ProblemDesc(C.Structure):
    _fields_ = [("kind", C.c_int), ("precision", C.c_int), ("n_params", C.c_int),
                ("priors", C.POINTER(Prior)), ("n_data", C.c_int),
                ("data", C.POINTER(C.c_double)), ("cov", C.POINTER(C.c_double)),
                ("emu", EmulatorDesc), ("shear", ShearDesc), ("gauss", GaussDesc), ("max_batch", C.c_int),
                ("cmb", CmbDesc), ("hidden_tile", C.c_int)]


class Config(C.Structure):
    _fields_ = [("n_live", C.c_int), ("n_delete", C.c_int), ("repeats", C.c_int), ("tol", C.c_double),
                ("seed", C.c_ulonglong), ("width", C.c_double), ("step_cap", C.c_int), ("ridge", C.c_double),
                ("rounds_per_sync", C.c_int), ("chain_groups", C.c_int), ("n_shards", C.c_int),
                ("shard", C.c_int)]


class NutsConfig(C.Structure):
    _fields_ = [("n_chains", C.c_int), ("n_warmup", C.c_int), ("n_samples", C.c_int), ("seed", C.c_ulonglong),
                ("target_accept", C.c_double), ("max_depth", C.c_int), ("init_step", C.c_double),
                ("adapt_mass", C.c_int)]


class NutsStats(C.Structure):
    _fields_ = [("gradient_evals", C.c_longlong), ("batched_calls", C.c_longlong), ("divergences", C.c_int),
                ("mean_depth", C.c_double), ("mean_accept", C.c_double)]


class Status(C.Structure):
    _fields_ = [("iterations", C.c_longlong), ("evaluations", C.c_longlong), ("rounds", C.c_longlong),
                ("converged", C.c_int), ("status_bits", C.c_int), ("logZ", C.c_double), ("logX", C.c_double),
                ("lstar", C.c_double), ("nonfinite", C.c_longlong)]


_lib = None


def load():
    """Load libgpuns.so; raises if it has not been built (there is no fallback)."""
    global _lib
    if _lib is not None:
        return _lib
    if not os.path.exists(LIB_PATH):
        raise RuntimeError(f"{LIB_PATH} is missing: build it with paper_2509_13307_gb300.build.build() "
                           "(nvcc, sm_103a); the library has no CPU fallback")
    lib = C.CDLL(LIB_PATH)
    vp, dp, ip = C.c_void_p, C.POINTER(C.c_double), C.POINTER(C.c_int)
    lib.ns_strerror.restype = C.c_char_p
    lib.ns_strerror.argtypes = [C.c_int]
    lib.ns_problem_create.argtypes = [C.POINTER(ProblemDesc), C.POINTER(vp)]
    lib.ns_problem_free.argtypes = [vp]
    lib.ns_problem_dim.argtypes = [vp, ip]
    lib.ns_prior_transform.argtypes = [vp, vp, C.c_int, vp, vp]
    lib.loglike_batch.argtypes = [vp, vp, C.c_int, vp, vp]
    lib.ns_model_batch.argtypes = [vp, vp, C.c_int, vp, vp]
    lib.ns_emulator_batch.argtypes = [vp, vp, C.c_int, vp, vp]
    lib.ns_problem_status.argtypes = [vp, C.POINTER(C.c_int), C.c_int]
    lib.ns_nuts_run.argtypes = [vp, C.POINTER(NutsConfig), dp, dp, dp, dp, C.POINTER(NutsStats), vp]
    lib.ns_problem_tiles.argtypes = [vp, C.POINTER(C.c_int), C.POINTER(C.c_float), C.c_int]
    lib.ns_problem_fused.argtypes = [vp, C.POINTER(C.c_int)]
    lib.loglike_grad_batch.argtypes = [vp, vp, C.c_int, vp, vp, vp]
    lib.ns_init.argtypes = [vp, C.POINTER(Config), vp, C.POINTER(vp)]
    lib.ns_step.argtypes = [vp, C.c_int, C.POINTER(Status)]
    lib.ns_evidence.argtypes = [vp, C.c_int, dp, dp, dp, dp, C.POINTER(C.c_longlong)]
    lib.ns_live_points.argtypes = [vp, vp, vp]
    lib.ns_dead_points.argtypes = [vp, C.c_longlong, vp, vp, vp, C.POINTER(C.c_longlong)]
    lib.ns_last_iteration.argtypes = [vp, dp, vp, vp, vp]
    lib.ns_profile_stage.argtypes = [vp, C.c_int]
    lib.ns_profile_read.argtypes = [vp, dp, C.POINTER(C.c_longlong), C.POINTER(C.c_longlong)]
    lib.ns_evidence_noalloc.argtypes = [vp, vp, C.c_longlong, C.c_ulonglong, C.c_int, vp, vp]
    lib.ns_multi_init.argtypes = [C.POINTER(vp), C.c_int, C.POINTER(Config), vp, C.POINTER(vp)]
    lib.ns_multi_step.argtypes = [vp, C.c_int, C.POINTER(Status)]
    lib.ns_multi_run.argtypes = [vp, C.c_int, C.POINTER(vp)]
    lib.ns_multi_free.argtypes = [vp]
    lib.ns_shard_evolve.argtypes = [vp, C.POINTER(Status)]
    lib.ns_shard_export.argtypes = [vp, vp]
    lib.ns_shard_insert.argtypes = [vp, vp, C.POINTER(Status)]
    lib.ns_shard_range.argtypes = [vp, ip, ip]
    lib.ns_free.argtypes = [vp]
    for name in EXPORTS:
        getattr(lib, name).restype = C.c_char_p if name == "ns_strerror" else C.c_int
    _lib = lib
    return lib


class GpunsError(RuntimeError):
    def __init__(self, code, where):
        msg = load().ns_strerror(code).decode()
        super().__init__(f"{where}: {msg} (status {code})")
        self.code = code


def check(code, where):
    if code != NS_OK:
        raise GpunsError(code, where)
