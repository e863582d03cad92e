"""Thin Python layer over the C ABI: builds problem descriptors from the seeded
workload inputs, passes torch CUDA tensors by pointer on torch's current stream,
and wraps runs.  Every numerical step runs inside libgpuns.so."""

from __future__ import annotations

import ctypes as C
from dataclasses import dataclass

import numpy as np
import torch

from . import _lib as L
from .mock import diagonal_covariance, knox_covariance


def _dptr(a: np.ndarray):
    return a.ctypes.data_as(C.POINTER(C.c_double))


def _iptr(a: np.ndarray):
    return a.ctypes.data_as(C.POINTER(C.c_int))


def _stream(stream=None):
    s = torch.cuda.current_stream() if stream is None else stream
    return C.c_void_p(s.cuda_stream)


def _require_cuda(t: torch.Tensor, name: str, dtype=torch.float64):
    if not t.is_cuda or t.dtype != dtype or t.dim() != 2:
        raise ValueError(f"{name} must be a 2-D CUDA {dtype} tensor")
    return t.contiguous()


class Problem:
    """A likelihood problem resident on the current CUDA device."""

    def __init__(self, inp: dict, precision: str = "fp64", max_batch: int = 1024, data=None, cov=None,
                 solve: str = "fold", form: str = "gauss", hidden_tile: int = 0):
        self.lib = L.load()
        self.hidden_tile = int(hidden_tile)
        self.inp = inp
        self.kind = inp["kind"]
        self.precision = precision
        self.max_batch = int(max_batch)
        self.solve = solve
        self.form = form
        self._h = C.c_void_p()
        if self.kind == "shear" and (data is None or cov is None):
            data, cov = self._make_mock()
        elif self.kind == "cmb" and form == "tt_cv" and data is None:
            data = self._make_mock_tt()
        elif self.kind == "cmb" and form != "tt_cv" and (data is None or cov is None):
            data, cov = self._make_mock_cmb()
        self.data = None if data is None else np.ascontiguousarray(data, dtype=np.float64)
        self.cov = None if cov is None else np.ascontiguousarray(cov, dtype=np.float64)
        self._create(precision, self.max_batch, self.data, self.cov, self._templates(self.cov))
        d = C.c_int()
        L.check(self.lib.ns_problem_dim(self._h, C.byref(d)), "ns_problem_dim")
        self.d = d.value

    # ------------------------------------------------------------ set-up
    def _templates(self, cov):
        inp = self.inp
        if self.kind != "shear" or inp["n_tmpl"] == 0:
            return None
        if cov is None:
            return np.zeros((len(inp["noise_eps"]), inp["n_tmpl"]))
        sig = np.sqrt(np.diag(cov))
        return np.ascontiguousarray(0.1 * sig[:, None] * inp["tmpl_g"])

    def _make_mock(self):
        """data = model(fiducial) + L eps with the library's FP64 model vector."""
        inp = self.inp
        D = len(inp["noise_eps"])
        self._create("fp64", 1, np.zeros(D), np.eye(D),
                     np.zeros((D, inp["n_tmpl"])) if inp["n_tmpl"] else None)
        fid = np.asarray(inp["fiducial"], float)
        free = [i for i, p in enumerate(inp["priors"]) if p[0] != "F"]
        th = torch.tensor(fid[free][None, :], dtype=torch.float64, device="cuda")
        mfid = self.model(th)[0].cpu().numpy()
        self._free()
        if inp["cov_kind"] == "diag10":
            cov = diagonal_covariance(mfid)
        else:
            cov = knox_covariance(mfid, inp["n_bins"], inp["ell"], inp["delta_ell"], inp["f_sky"],
                                  inp["sigma_e"] ** 2 / inp["n_gal_sr"], inp["cov_V"], inp["cov_rank_amp"])
        data = mfid + np.linalg.cholesky(cov) @ inp["noise_eps"]
        return data, cov

    def _make_mock_tt(self):
        """Cosmic-variance TT mock: d_ell = C_fid,ell X_ell / (2 ell + 1) with the
        seeded chi-squared draws X_ell and the library's FP64 fiducial spectra."""
        inp = self.inp
        form, self.form = self.form, "gauss"
        self._create("fp64", 1, None, None, None)
        self.form = form
        th = torch.tensor(np.asarray(inp["fiducial"], float)[None, :], dtype=torch.float64, device="cuda")
        mfid = self.model(th)[0].cpu().numpy()
        self._free()
        n = len(inp["ell"])
        return mfid[:n] * inp["tt_chi2"] / (2.0 * np.asarray(inp["ell"], float) + 1.0)

    def _make_mock_cmb(self):
        """C = s W (seeded Wishart base, s from the library's FP64 fiducial
        model: mean variance (cov_rel * rms m_fid)^2) and data = m_fid + L eps."""
        from workloads import wishart_base
        inp = self.inp
        self._create("fp64", 1, None, None, None)
        th = torch.tensor(np.asarray(inp["fiducial"], float)[None, :], dtype=torch.float64, device="cuda")
        mfid = self.model(th)[0].cpu().numpy()
        self._free()
        W = wishart_base(int(inp["n_data"]), int(inp["wishart_nu"]), int(inp["seed_cov"]))
        s = (inp["cov_rel"] * np.sqrt(np.mean(mfid * mfid))) ** 2 / np.mean(np.diag(W))
        cov = s * W
        data = mfid + np.linalg.cholesky(cov) @ inp["noise_eps"]
        return data, cov

    def _create(self, precision, max_batch, data, cov, tmpl):
        inp = self.inp
        keep = []   # arrays that must stay alive during ns_problem_create
        desc = L.ProblemDesc()
        desc.kind = {"shear": L.NS_KIND_SHEAR, "cmb": L.NS_KIND_CMB}.get(self.kind, L.NS_KIND_GAUSS)
        desc.precision = L.NS_PREC[precision]
        pri = inp["priors"]
        desc.n_params = len(pri)
        parr = (L.Prior * len(pri))(*[L.Prior(L.NS_PRIOR[k], a, b) for (k, a, b) in pri])
        keep.append(parr)
        desc.priors = parr
        desc.max_batch = max_batch
        # BF16 layer mode: 0 autotuned per-layer GEMMs, 16..128 a forced N-tile, -1 the fused stack
        desc.hidden_tile = self.hidden_tile if precision.startswith("bf16") else 0
        if self.kind == "gauss":
            desc.gauss = L.GaussDesc(inp["mu"], inp["sigma"])
        else:
            D = len(inp["noise_eps"])
            desc.n_data = D
            for arr, field in ((data, "data"), (cov, "cov")):
                if arr is None:
                    continue
                a = np.ascontiguousarray(arr, dtype=np.float64)
                keep.append(a)
                setattr(desc, field, _dptr(a))
            Ws = [np.ascontiguousarray(w, dtype=np.float64) for w in inp["emu_W"]]
            bs = [np.ascontiguousarray(b, dtype=np.float64) for b in inp["emu_b"]]
            keep += Ws + bs
            nl = len(Ws)
            dims = np.array([Ws[0].shape[1]] + [w.shape[0] for w in Ws], dtype=np.int32)
            Wp = (C.POINTER(C.c_double) * nl)(*[_dptr(w) for w in Ws])
            bp = (C.POINTER(C.c_double) * nl)(*[_dptr(b) for b in bs])
            ins = np.ascontiguousarray(inp["emu_inputs"], dtype=np.int32)
            cen = np.ascontiguousarray(inp["emu_in_center"], dtype=np.float64)
            scl = np.ascontiguousarray(inp["emu_in_scale"], dtype=np.float64)
            mu = np.ascontiguousarray(inp["emu_out_mu"], dtype=np.float64)
            keep += [dims, Wp, bp, ins, cen, scl, mu]
            e = desc.emu
            e.n_layers = nl
            e.dims = _iptr(dims)
            e.W = C.cast(Wp, C.POINTER(C.POINTER(C.c_double)))
            e.b = C.cast(bp, C.POINTER(C.POINTER(C.c_double)))
            e.inputs = _iptr(ins)
            e.in_center = _dptr(cen)
            e.in_scale = _dptr(scl)
            e.out_mu = _dptr(mu)
            e.activation = L.NS_ACT[inp.get("emu_act", "tanh")]
            if e.activation == L.NS_ACT["sigmoid_linear"]:
                gs = [np.ascontiguousarray(g, dtype=np.float64) for g in inp["act_g"]]
                bs_ = [np.ascontiguousarray(b, dtype=np.float64) for b in inp["act_beta"]]
                gp = (C.POINTER(C.c_double) * len(gs))(*[_dptr(g) for g in gs])
                bp2 = (C.POINTER(C.c_double) * len(bs_))(*[_dptr(b) for b in bs_])
                keep += gs + bs_ + [gp, bp2]
                e.act_g = C.cast(gp, C.POINTER(C.POINTER(C.c_double)))
                e.act_beta = C.cast(bp2, C.POINTER(C.POINTER(C.c_double)))
            if self.kind == "cmb":
                sv = np.ascontiguousarray(inp["emu_out_sig"], dtype=np.float64)
                keep.append(sv)
                e.out_sigma = 1.0
                e.out_sigma_vec = _dptr(sv)
                desc.cmb.solve = L.NS_SOLVE[self.solve]
                desc.cmb.form = L.NS_CMB_FORM[self.form]
                if self.form == "tt_cv":
                    ell = np.ascontiguousarray(inp["ell"], dtype=np.float64)
                    keep.append(ell)
                    desc.cmb.n_tt = len(ell)
                    desc.cmb.ell = _dptr(ell)
                    desc.n_data = len(ell) if data is not None else 0
                    desc.cov = C.POINTER(C.c_double)()
                h = C.c_void_p()
                L.check(self.lib.ns_problem_create(C.byref(desc), C.byref(h)), "ns_problem_create")
                self._h = h
                return
            e.out_sigma = float(inp["emu_out_sigma"])
            s = desc.shear
            nzm = np.ascontiguousarray(inp["nz_mean"], dtype=np.float64)
            nzs = np.ascontiguousarray(inp["nz_sigma"], dtype=np.float64)
            ell = np.ascontiguousarray(inp["ell"], dtype=np.float64)
            keep += [nzm, nzs, ell]
            s.n_bins = inp["n_bins"]
            s.nz_mean = _dptr(nzm)
            s.nz_sigma = _dptr(nzs)
            s.n_ell = len(ell)
            s.ell = _dptr(ell)
            s.n_k = inp["n_k"]
            s.lnk_min = inp["lnk_min"]
            s.lnk_max = inp["lnk_max"]
            s.n_z = inp["n_z"]
            s.z_max = inp["z_max"]
            s.n_z_emu = inp["n_z_emu"]
            s.n_chi = inp["n_chi"]
            s.a_min = inp["a_min"]
            s.ia_pivot = inp["ia_pivot"]
            s.c1rho = inp["c1rho"]
            s.n_tmpl = inp["n_tmpl"]
            s.z_interp = {"catmull_rom": 0, "linear": 1}[inp.get("z_interp", "catmull_rom")]
            if inp["n_tmpl"]:
                t = np.ascontiguousarray(tmpl, dtype=np.float64)
                keep.append(t)
                s.tmpl = _dptr(t)
        h = C.c_void_p()
        L.check(self.lib.ns_problem_create(C.byref(desc), C.byref(h)), "ns_problem_create")
        self._h = h

    def _free(self):
        if self._h:
            self.lib.ns_problem_free(self._h)
            self._h = C.c_void_p()

    def close(self):
        self._free()

    def __del__(self):
        try:
            self._free()
        except Exception:
            pass

    @property
    def handle(self):
        return self._h

    # ------------------------------------------------------------ calls
    def loglike(self, theta: torch.Tensor, stream=None) -> torch.Tensor:
        """log L at physical free parameters theta (B x d, float64, CUDA)."""
        theta = _require_cuda(theta, "theta")
        B = theta.shape[0]
        out = torch.empty(B, dtype=torch.float64, device=theta.device)
        L.check(self.lib.loglike_batch(self._h, C.c_void_p(theta.data_ptr()), B, C.c_void_p(out.data_ptr()),
                                       _stream(stream)), "loglike_batch")
        return out

    def model(self, theta: torch.Tensor, stream=None) -> torch.Tensor:
        theta = _require_cuda(theta, "theta")
        B = theta.shape[0]
        D = len(self.inp["noise_eps"])
        out = torch.empty((B, D), dtype=torch.float64, device=theta.device)
        L.check(self.lib.ns_model_batch(self._h, C.c_void_p(theta.data_ptr()), B, C.c_void_p(out.data_ptr()),
                                        _stream(stream)), "ns_model_batch")
        return out

    def emulator(self, theta: torch.Tensor, stream=None) -> torch.Tensor:
        """Raw emulator output (B x n_out) in the problem precision, returned as float64."""
        theta = _require_cuda(theta, "theta")
        B = theta.shape[0]
        n_out = int(np.asarray(self.inp["emu_out_mu"]).size)
        out = torch.empty((B, n_out), dtype=torch.float64, device=theta.device)
        L.check(self.lib.ns_emulator_batch(self._h, C.c_void_p(theta.data_ptr()), B, C.c_void_p(out.data_ptr()),
                                           _stream(stream)), "ns_emulator_batch")
        return out

    def tiles(self):
        """BF16: (N-tile width per layer, autotuned time per launch [ms]) of the tensor-core layers."""
        n = len(self.inp["emu_W"])
        t = (C.c_int * n)()
        ms = (C.c_float * n)()
        L.check(self.lib.ns_problem_tiles(self._h, t, ms, n), "ns_problem_tiles")
        return list(t), list(ms)

    def fused_cluster(self) -> int:
        """BF16: cluster size of the fused input + hidden-layer kernel, 0 if the layers run separately."""
        c = C.c_int(0)
        L.check(self.lib.ns_problem_fused(self._h, C.byref(c)), "ns_problem_fused")
        return c.value

    def device_status(self, clear: bool = False) -> int:
        """Status bits of earlier batch calls (NS_BIT_TIMEOUT = 4: a bounded
        device wait gave up and the affected rows are NaN).  Synchronises."""
        bits = C.c_int(0)
        L.check(self.lib.ns_problem_status(self._h, C.byref(bits), int(clear)), "ns_problem_status")
        return bits.value

    def prior_transform(self, cube: torch.Tensor, stream=None) -> torch.Tensor:
        cube = _require_cuda(cube, "cube")
        out = torch.empty_like(cube)
        L.check(self.lib.ns_prior_transform(self._h, C.c_void_p(cube.data_ptr()), cube.shape[0],
                                            C.c_void_p(out.data_ptr()), _stream(stream)), "ns_prior_transform")
        return out

    def loglike_grad(self, theta: torch.Tensor, stream=None):
        theta = _require_cuda(theta, "theta")
        B = theta.shape[0]
        out = torch.empty(B, dtype=torch.float64, device=theta.device)
        g = torch.empty_like(theta)
        L.check(self.lib.loglike_grad_batch(self._h, C.c_void_p(theta.data_ptr()), B, C.c_void_p(out.data_ptr()),
                                            C.c_void_p(g.data_ptr()), _stream(stream)), "loglike_grad_batch")
        return out, g


class LogLike(torch.autograd.Function):
    """log L(theta) as a differentiable torch op: forward calls the library's
    hand-written adjoint (loglike_grad_batch) once and keeps the gradient;
    backward scales it by the incoming gradient."""

    @staticmethod
    def forward(ctx, theta, problem):
        logL, grad = problem.loglike_grad(theta.detach())
        ctx.save_for_backward(grad)
        return logL

    @staticmethod
    def backward(ctx, grad_out):
        (grad,) = ctx.saved_tensors
        return grad_out[:, None] * grad, None


def loglike_autograd(problem: "Problem", theta: torch.Tensor) -> torch.Tensor:
    return LogLike.apply(theta, problem)


@dataclass
class RunStatus:
    iterations: int
    evaluations: int
    rounds: int
    converged: bool
    status_bits: int
    logZ: float
    logX: float
    lstar: float
    nonfinite: int = 0


class NestedRun:
    """One nested-sampling run on a problem (ns_init / ns_step / ns_evidence)."""

    def __init__(self, problem: Problem, n_live: int, n_delete: int, repeats: int | None = None,
                 tol: float = 1e-3, seed: int = 3, width: float = 1.0, step_cap: int = 100,
                 ridge: float = 1e-12, rounds_per_sync: int = 0, chain_groups: int = 0, stream=None,
                 n_shards: int = 1, shard: int = 0):
        self.lib = problem.lib
        self.problem = problem
        self.n_live, self.n_delete, self.d = n_live, n_delete, problem.d
        cfg = L.Config(n_live, n_delete, 0 if repeats is None else repeats, tol, seed, width, step_cap, ridge,
                       rounds_per_sync, chain_groups, n_shards, shard)
        self._stream_obj = stream if stream is not None else torch.cuda.current_stream()
        h = C.c_void_p()
        L.check(self.lib.ns_init(problem.handle, C.byref(cfg), _stream(self._stream_obj), C.byref(h)), "ns_init")
        self._h = h
        self.n_shards, self.shard = max(1, n_shards), shard
        b, e = C.c_int(), C.c_int()
        L.check(self.lib.ns_shard_range(self._h, C.byref(b), C.byref(e)), "ns_shard_range")
        self.chain_range = (b.value, e.value)

    @staticmethod
    def _status(st) -> "RunStatus":
        return RunStatus(st.iterations, st.evaluations, st.rounds, bool(st.converged), st.status_bits,
                         st.logZ, st.logX, st.lstar, st.nonfinite)

    # ---- one run split over devices (ns_shard_*): see ShardedRun
    def shard_evolve(self) -> "RunStatus":
        st = L.Status()
        L.check(self.lib.ns_shard_evolve(self._h, C.byref(st)), "ns_shard_evolve")
        return self._status(st)

    def shard_export(self) -> torch.Tensor:
        """This shard's final chain states, (chains x (d + 2)) float64 on the device."""
        b, e = self.chain_range
        out = torch.empty((e - b, self.d + 2), dtype=torch.float64, device="cuda")
        L.check(self.lib.ns_shard_export(self._h, C.c_void_p(out.data_ptr())), "ns_shard_export")
        return out

    def shard_insert(self, finals: torch.Tensor) -> "RunStatus":
        finals = finals.contiguous()
        if finals.shape != (self.n_delete, self.d + 2) or finals.dtype != torch.float64 or not finals.is_cuda:
            raise ValueError("finals must be a (k, d + 2) float64 CUDA tensor")
        st = L.Status()
        L.check(self.lib.ns_shard_insert(self._h, C.c_void_p(finals.data_ptr()), C.byref(st)), "ns_shard_insert")
        return self._status(st)

    @classmethod
    def from_config(cls, problem, sc, **kw):
        return cls(problem, sc.n_live, sc.n_delete, sc.repeats, sc.tol, sc.seed, sc.width, sc.step_cap, sc.ridge, **kw)

    def step(self, n_iters: int = 1) -> RunStatus:
        st = L.Status()
        L.check(self.lib.ns_step(self._h, n_iters, C.byref(st)), "ns_step")
        return RunStatus(st.iterations, st.evaluations, st.rounds, bool(st.converged), st.status_bits,
                         st.logZ, st.logX, st.lstar, st.nonfinite)

    def run(self, max_iters: int = 10 ** 9, chunk: int = 64) -> RunStatus:
        st = self.step(0)
        while not st.converged and st.iterations < max_iters:
            st = self.step(min(chunk, max_iters - st.iterations))
        return st

    def evidence(self, n_replays: int = 200) -> dict:
        lz, err, lx, H = C.c_double(), C.c_double(), C.c_double(), C.c_double()
        nd = C.c_longlong()
        L.check(self.lib.ns_evidence(self._h, n_replays, C.byref(lz), C.byref(err), C.byref(lx), C.byref(H),
                                     C.byref(nd)), "ns_evidence")
        return dict(logZ=lz.value, logZ_err=err.value, logX=lx.value, H=H.value, n_dead=nd.value)

    def live_points(self):
        x = np.empty((self.n_live, self.d))
        lg = np.empty(self.n_live)
        L.check(self.lib.ns_live_points(self._h, x.ctypes.data_as(C.c_void_p), lg.ctypes.data_as(C.c_void_p)),
                "ns_live_points")
        return x, lg

    def dead_points(self, max_out: int = 1 << 40):
        st = self.step(0)
        n = min(max_out, st.iterations * self.n_delete)
        x = np.empty((max(n, 1), self.d))
        lg = np.empty(max(n, 1))
        nl = np.empty(max(n, 1), dtype=np.int32)
        cnt = C.c_longlong()
        L.check(self.lib.ns_dead_points(self._h, n, x.ctypes.data_as(C.c_void_p), lg.ctypes.data_as(C.c_void_p),
                                        nl.ctypes.data_as(C.c_void_p), C.byref(cnt)), "ns_dead_points")
        m = cnt.value
        return x[:m], lg[:m], nl[:m]

    def posterior(self):
        """Posterior samples of the run: the dead points, then the live points in
        ascending log L, as (cube x, log L, log w) with the normalised
        importance weights of Eq. 1, w_i = L_i (X_{i-1} - X_i) / Z and the
        expected shrinkage ln X_i = ln X_{i-1} - 1/n_i (host-side analysis of
        the copied-out points)."""
        xd, ld, nd = self.dead_points()
        xl, ll = self.live_points()
        o = np.argsort(ll, kind="stable")
        x = np.vstack([xd, xl[o]])
        lg = np.concatenate([ld, ll[o]])
        nl = np.concatenate([nd, self.n_live - np.arange(self.n_live)]).astype(float)
        lnX_prev = np.concatenate([[0.0], -np.cumsum(1.0 / nl)[:-1]])
        logw = lg + lnX_prev + np.log(-np.expm1(-1.0 / nl))
        m = np.max(logw)
        logw = logw - (m + np.log(np.sum(np.exp(logw - m))))
        return x, lg, logw

    def last_iteration(self):
        k = self.n_delete
        lstar = C.c_double()
        dele = np.empty(k, dtype=np.int32)
        sta = np.empty(k, dtype=np.int32)
        ev = np.empty(k, dtype=np.int32)
        L.check(self.lib.ns_last_iteration(self._h, C.byref(lstar), dele.ctypes.data_as(C.c_void_p),
                                           sta.ctypes.data_as(C.c_void_p), ev.ctypes.data_as(C.c_void_p)),
                "ns_last_iteration")
        return lstar.value, dele, sta, ev

    STAGES = {"off": 0, "projection": 1, "emu_out": 2, "chi2": 3, "emu_hidden": 4, "windows": 5}

    def profile_stage(self, stage: str):
        L.check(self.lib.ns_profile_stage(self._h, self.STAGES[stage]), "ns_profile_stage")

    def profile_read(self):
        ms, n, rows = C.c_double(), C.c_longlong(), C.c_longlong()
        L.check(self.lib.ns_profile_read(self._h, C.byref(ms), C.byref(n), C.byref(rows)), "ns_profile_read")
        return dict(ms=ms.value, launches=n.value, rows=rows.value)

    def close(self):
        if self._h:
            self.lib.ns_free(self._h)
            self._h = C.c_void_p()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


def shard_bounds(k: int, n_shards: int):
    """Chain ranges of the shards of a run split over n_shards devices: shard s
    evolves chains [floor(k s / G), floor(k (s + 1) / G)) (as ns_init sets them)."""
    return [(k * s // n_shards, k * (s + 1) // n_shards) for s in range(n_shards)]


class ShardedRun:
    """One nested-sampling run split over the ranks of a torch.distributed
    group, one device per rank (the k chains of an iteration are independent,
    Sec. 2.2).  Every rank holds a shard run (NestedRun with n_shards = world
    size, shard = rank; any object with the same shard_* methods works) of the
    same problem and seed.  Per iteration the shards evolve their chains, then
    one all-gather of every shard's final chain states (rows padded to the
    largest shard, unpadded here in shard order) hands all k to every rank,
    which inserts them; the deletion, covariance and evidence work is
    redundant, so no other exchange is needed and every rank ends each
    iteration with the single-device run's state."""

    def __init__(self, shard_run, group=None):
        import torch.distributed as dist
        self.dist = dist
        self.run = shard_run
        self.group = group
        self.world = dist.get_world_size(group)
        self.rank = dist.get_rank(group)
        self.k, self.d = shard_run.n_delete, shard_run.d
        self.bounds = shard_bounds(self.k, self.world)
        if tuple(shard_run.chain_range) != tuple(self.bounds[self.rank]):
            raise ValueError(f"rank {self.rank} holds chains {shard_run.chain_range}, expected {self.bounds[self.rank]}")
        self.rows = max(e - b for b, e in self.bounds)

    def gather(self, local: torch.Tensor) -> torch.Tensor:
        """All shards' rows (k x (d + 2)) in chain order from this rank's rows."""
        w = self.d + 2
        pad = torch.zeros((self.rows, w), dtype=local.dtype, device=local.device)
        pad[:local.shape[0]] = local
        parts = [torch.empty_like(pad) for _ in range(self.world)]
        self.dist.all_gather(parts, pad, group=self.group)
        return torch.cat([parts[s][:e - b] for s, (b, e) in enumerate(self.bounds)])

    def step(self, n_iters: int = 1):
        st = None
        for _ in range(n_iters):
            st = self.run.shard_evolve()
            if st.converged:
                break
            st = self.run.shard_insert(self.gather(self.run.shard_export()))
        return st

    def run_until_converged(self, max_iters: int = 10 ** 9):
        st = None
        for _ in range(max_iters):
            st = self.step(1)
            if st.converged:
                break
        return st


class MultiRun:
    """Several nested-sampling runs of one model packed into shared likelihood
    batches (ns_multi_*).  problems share the model; each has its own priors."""

    def __init__(self, problems, samplers, stream=None):
        self.lib = problems[0].lib
        self.problems = problems
        n = len(problems)
        arr = (C.c_void_p * n)(*[p.handle.value for p in problems])
        cfgs = (L.Config * n)(*[L.Config(sc.n_live, sc.n_delete, 0 if sc.repeats is None else sc.repeats, sc.tol,
                                         sc.seed, sc.width, sc.step_cap, sc.ridge, 0, 1, 0, 0) for sc in samplers])
        self._stream_obj = stream if stream is not None else torch.cuda.current_stream()
        h = C.c_void_p()
        L.check(self.lib.ns_multi_init(arr, n, cfgs, _stream(self._stream_obj), C.byref(h)), "ns_multi_init")
        self._h = h
        self.n = n
        self.samplers = samplers

    def step(self, n_iters: int = 1):
        st = (L.Status * self.n)()
        L.check(self.lib.ns_multi_step(self._h, n_iters, st), "ns_multi_step")
        return [RunStatus(s.iterations, s.evaluations, s.rounds, bool(s.converged), s.status_bits, s.logZ, s.logX,
                          s.lstar, s.nonfinite) for s in st]

    def run(self, max_iters: int = 10 ** 9, chunk: int = 64):
        sts = self.step(0)
        while not all(s.converged for s in sts) and min(s.iterations for s in sts) < max_iters:
            sts = self.step(chunk)
        return sts

    def _run(self, i):
        r = C.c_void_p()
        L.check(self.lib.ns_multi_run(self._h, i, C.byref(r)), "ns_multi_run")
        return r

    def evidence(self, i: int, n_replays: int = 200) -> dict:
        lz, err, lx, H = C.c_double(), C.c_double(), C.c_double(), C.c_double()
        nd = C.c_longlong()
        L.check(self.lib.ns_evidence(self._run(i), n_replays, C.byref(lz), C.byref(err), C.byref(lx), C.byref(H),
                                     C.byref(nd)), "ns_evidence")
        return dict(logZ=lz.value, logZ_err=err.value, logX=lx.value, H=H.value, n_dead=nd.value)

    def last_iteration(self, i: int):
        k = self.samplers[i].n_delete
        lstar = C.c_double()
        dele = np.empty(k, dtype=np.int32)
        sta = np.empty(k, dtype=np.int32)
        ev = np.empty(k, dtype=np.int32)
        L.check(self.lib.ns_last_iteration(self._run(i), C.byref(lstar), dele.ctypes.data_as(C.c_void_p),
                                           sta.ctypes.data_as(C.c_void_p), ev.ctypes.data_as(C.c_void_p)),
                "ns_last_iteration")
        return lstar.value, dele, sta, ev

    def close(self):
        if self._h:
            self.lib.ns_multi_free(self._h)
            self._h = C.c_void_p()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


def nuts(problem: Problem, n_chains: int, n_warmup: int, n_samples: int, z0=None, seed: int = 5,
         target_accept: float = 0.8, max_depth: int = 10, init_step: float = 0.1, adapt_mass: bool = True,
         stream=None) -> dict:
    """No-U-Turn sampling of the problem's posterior (ns_nuts_run): returns the
    unconstrained samples z (chains x samples x d), the physical parameters
    theta (prior transform of the logistic of z, on the device), log p(z), the
    final step sizes and the run statistics."""
    d = problem.d
    z0 = np.zeros((n_chains, d)) if z0 is None else np.ascontiguousarray(z0, dtype=np.float64)
    z0 = np.ascontiguousarray(z0, dtype=np.float64)
    cfg = L.NutsConfig(n_chains, n_warmup, n_samples, seed, target_accept, max_depth, init_step, int(adapt_mass))
    samples = np.empty((n_chains, n_samples, d))
    logp = np.empty((n_chains, n_samples))
    eps = np.empty(n_chains)
    st = L.NutsStats()
    L.check(problem.lib.ns_nuts_run(problem.handle, C.byref(cfg), _dptr(z0), _dptr(samples), _dptr(logp),
                                    _dptr(eps), C.byref(st), _stream(stream)), "ns_nuts_run")
    flat = torch.tensor(1.0 / (1.0 + np.exp(-samples.reshape(-1, d))), dtype=torch.float64, device="cuda")
    theta = torch.cat([problem.prior_transform(flat[i:i + problem.max_batch])
                       for i in range(0, flat.shape[0], problem.max_batch)]).cpu().numpy()
    return dict(z=samples, theta=theta.reshape(n_chains, n_samples, d), logp=logp, step_size=eps,
                stats=dict(gradient_evals=st.gradient_evals, batched_calls=st.batched_calls,
                           divergences=st.divergences, mean_depth=st.mean_depth, mean_accept=st.mean_accept))
