#!/usr/bin/env python
"""Benchmark of the batched nested-slice-sampling step (arXiv:2509.13307) on
the 39-parameter w0-wa cosmic-shear workload, one JSON line on rank 0.

A step is one nested-sampling iteration: delete the k = 500 lowest of
n = 1000 live points (FP64 evidence update), live covariance + Cholesky,
500 chains x 5d = 195 hit-and-run slice moves, every proposal scored by the
fused likelihood (BF16 tcgen05 emulator 7 -> 4x1024 -> 10000, chi(z), windows,
P(k, z) lookup, Limber, whitened chi^2).  The metric is likelihood
evaluations per second over the timed steps (device time, CUDA events on the
run's stream, L2 flushed between steps).  Also reported: the plain FP32 form
on the same workload, iterations/s, wall time to a converged log Z, the
end-to-end rate through the public API with host buffers, the roofline of the
dominant kernel, and the CPU oracle as a baseline.

Multi-GPU (torchrun): each rank runs an independent nested-sampling run with
its own seed (runs are independent problems: weak scaling, no collective on the
data path); the value is the sum of evaluations over the max of rank times.

--impl reference times the CPU oracle on the same workload (bounded sample of
likelihood evaluations per step) and prints the same JSON line.
"""

from __future__ import annotations

import argparse
import json
import math
import os
import subprocess
import sys
import tempfile
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = "logL evals/s and seconds to converged logZ (39-d shear), BF16+adjoint vs plain FP32"
UNIT = "evals/s"
WORKLOAD = ("shear39: 39-parameter w0-wa cosmic shear (7 cosmology + 2 baryon + 2 IA + 5 D_z + 5 m + "
            "18 template amplitudes), 5 tomographic bins x 20 ell (D = 300), emulator 7->4x1024->(200 k x 50 z), "
            "1025 chi nodes uniform in a on [1/6.02, 1], dense Knox + rank-5 covariance; n_live = 1000, "
            "k = 500 chains, 5d = 195 slice moves per chain")


def _env_int(name, default):
    try:
        return int(os.environ.get(name, default))
    except ValueError:
        return default


def cpu_oracle_rate(seconds: float = 12.0, threads: int = 1) -> dict:
    """Oracle log-likelihood evaluations/s on the host (bounded sample), in a
    subprocess with BLAS/OpenMP pinned to `threads`."""
    code = r"""
import os, sys, time, json
sys.path.insert(0, %r)
import numpy as np
import workloads as w
from oracle.shear import ShearOracle
from oracle.priors import cube_to_theta
inp = w.make_shear_inputs(w.shear39())
o = ShearOracle(inp)
rng = np.random.default_rng(0)
n = 0; t0 = time.time()
while time.time() - t0 < %f:
    o.loglike_cube(rng.uniform(0.02, 0.98, 39)); n += 1
dt = time.time() - t0
print(json.dumps({"n": n, "s": dt}))
""" % (ROOT, seconds)
    env = dict(os.environ)
    for k in ("OMP_NUM_THREADS", "OPENBLAS_NUM_THREADS", "MKL_NUM_THREADS", "NUMEXPR_NUM_THREADS"):
        env[k] = str(threads)
    env["CUDA_VISIBLE_DEVICES"] = ""
    r = subprocess.run([sys.executable, "-c", code], capture_output=True, text=True, env=env, timeout=600)
    if r.returncode != 0:
        return {"value": None, "unit": UNIT, "cores": threads, "kind": "oracle", "error": r.stderr[-300:]}
    d = json.loads(r.stdout.strip().splitlines()[-1])
    return {"value": d["n"] / d["s"], "unit": UNIT, "cores": threads, "kind": "oracle",
            "sample": f"{d['n']} oracle log-likelihood evaluations of the 39-d shear problem at random "
                      f"prior points ({d['s']:.1f} s, FP64 NumPy, {threads} thread)"}


class ClockSampler:
    """nvidia-smi clocks / throttle reasons sampled every 200 ms."""

    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, index: int):
        self.index = index
        self.f = tempfile.NamedTemporaryFile("w+", suffix=".csv", delete=False)
        self.p = None

    def start(self):
        try:
            self.p = subprocess.Popen(["nvidia-smi", "-i", str(self.index), f"--query-gpu={self.FIELDS}",
                                       "--format=csv,noheader,nounits", "-lms", "200"],
                                      stdout=self.f, stderr=subprocess.DEVNULL)
        except OSError:
            self.p = None

    def stop(self) -> dict:
        if self.p is None:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        self.p.terminate()
        try:
            self.p.wait(timeout=5)
        except subprocess.TimeoutExpired:
            self.p.kill()
        self.f.flush()
        self.f.seek(0)
        sm, smax, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for line in self.f.read().splitlines():
            parts = [x.strip() for x in line.split(",")]
            if len(parts) < 9:
                continue
            try:
                sm.append(float(parts[1]))
                smax.append(float(parts[2]))
            except ValueError:
                continue
            for nm, v in zip(names, parts[5:9]):
                if v.lower().startswith("active"):
                    reasons.add(nm)
        os.unlink(self.f.name)
        sm.sort()
        return {"sm_mhz": sm[len(sm) // 2] if sm else None, "sm_max_mhz": max(smax) if smax else None,
                "reasons": sorted(reasons), "samples": len(sm)}


def limber_method_flops_per_eval(cfg) -> float:
    """The method's FLOPs of the Limber stage per evaluation (the roofline
    numerator): per (ell, chi node) the 16-tap bicubic lookup of Eq. 4 (16
    FMA) and one FMA per bin pair of the Limber sum (Eq. 3-4), 2 FLOP per FMA:
    2 n_ell N_chi (16 + n_pairs) = 1.271 MFLOP on the 39-d problem."""
    return 2.0 * cfg.n_ell * cfg.n_chi * (16 + cfg.n_pairs)


def limber_flops_per_eval(cfg) -> float:
    """Every FLOP the Limber kernel (k_limber) executes per evaluation, a
    larger count than the method's (reported beside it): per (ell, chi-node)
    a 16-tap bicubic lookup (32) + bracket and Catmull-Rom weights (10) + nb
    window products + 2 n_pairs pair-sum FLOPs (one FMA each); per data
    element the bias product and the template sum (3 + 2 n_tmpl)."""
    N = cfg.n_chi
    nb = cfg.n_bins
    npairs = nb * (nb + 1) // 2
    D = cfg.n_data
    return cfg.n_ell * (N - 1) * (32 + 10 + nb + 2 * npairs) + D * (3 + 2 * cfg.n_tmpl)


# DRAM traffic of k_limber per evaluation from one ncu capture (29,979,904 bytes
# read and 0 written at 460 evaluations per launch, cold L2, the summary in
# profiles/k_limber_bf16_shear39_B460.md).  It equals the kernel's algorithmic
# input bytes, so it scales with the rows of a launch; it is reported only while
# the kernel's sources are the ones the capture was taken on.
LIMBER_TRAFFIC_BYTES_PER_EVAL = 29979904 / 460
LIMBER_TRAFFIC_SOURCES = ("paper_2509_13307_gb300/csrc/projection.cu", "paper_2509_13307_gb300/csrc/async_copy.cuh")
# the whitening kernel and its launcher share projection.cu; that section does not enter the digest
LIMBER_DIGEST_SKIP = ("// Whitening Y = R L^-T", "template <typename T>\nstatic size_t windows_smem")
LIMBER_TRAFFIC_SHA256 = "52f6dbc59c1dce38ca2e5c08ab54174a9a1aec25b3ae3bace81f87e79b41af4f"


def limber_source_digest() -> str:
    """SHA-256 of the Limber kernel's sources (projection.cu without its
    whitening section, and async_copy.cuh)."""
    import hashlib
    h = hashlib.sha256()
    a, b = LIMBER_DIGEST_SKIP
    for f in LIMBER_TRAFFIC_SOURCES:
        with open(os.path.join(ROOT, f), encoding="utf-8") as fh:
            txt = fh.read()
        if a in txt and b in txt and txt.index(a) < txt.index(b):
            txt = txt[:txt.index(a)] + txt[txt.index(b):]
        h.update(txt.encode("utf-8"))
    return h.hexdigest()


def limber_traffic(avg_rows: float):
    """Measured DRAM bytes per k_limber launch of avg_rows evaluations, or None
    when the kernel's sources changed since the capture."""
    return LIMBER_TRAFFIC_BYTES_PER_EVAL * avg_rows if limber_source_digest() == LIMBER_TRAFFIC_SHA256 else None


def windows_flops_per_eval(cfg) -> float:
    """Algorithmic FLOPs of the windows stage (k_windows) per evaluation: per
    node interval the 4-point distance quadrature (4 x 12), per node the
    growth and weights (12), per node and bin the n(z) and window work (25)."""
    N = cfg.n_chi
    return (N - 1) * 48 + N * 12 + N * cfg.n_bins * 25


def job_totals(t_local: float, ev_local, world: int, device):
    """Whole-job totals over the ranks of one node: the timed region is the
    slowest rank's (max) and the evaluations are every rank's (sum); each rank
    runs an independent sampler (weak scaling, no data-path collective)."""
    if world == 1:
        return t_local, float(ev_local)
    import torch
    import torch.distributed as dist
    t = torch.tensor([t_local], dtype=torch.float64, device=device)
    e = torch.tensor([float(ev_local)], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    dist.all_reduce(e, op=dist.ReduceOp.SUM)
    return t.item(), e.item()


def replace_seed(sc, rank):
    from dataclasses import replace
    return replace(sc, seed=sc.seed + 100 * rank)


def measured_peaks() -> dict:
    """The measured HBM copy bandwidth and bf16 GEMM throughput of
    the GB300s, else the recipe's fallback figures."""
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as fh:
            d = json.load(fh)
        return {"hbm_gbs": float(d["hbm_gbs"]), "bf16_tflops_sustained": float(d["bf16_tflops_sustained"]),
                "source": "measured"}
    except (OSError, KeyError, ValueError):
        return {"hbm_gbs": 6800.0, "bf16_tflops_sustained": 1700.0, "source": "fallback"}


def fp32_alu_peak_tflops(sm_mhz: float) -> float:
    """152 SMs x 128 FP32 lanes x 2 FLOP (FMA) x clock."""
    return 152 * 128 * 2 * sm_mhz * 1e6 / 1e12


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=5)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--precision", default="bf16")
    ap.add_argument("--no-full-run", action="store_true", help="skip the time-to-converged-logZ runs")
    ap.add_argument("--no-fp32-run", action="store_true",
                    help="skip the plain FP32 form's time-to-converged-logZ run (about two minutes)")
    ap.add_argument("--no-cpu", action="store_true", help="skip the CPU oracle baseline")
    ap.add_argument("--no-multi", action="store_true", help="skip the packed-runs measurement")
    ap.add_argument("--no-cmb", action="store_true", help="skip the CMB (D = 7521) measurement")
    ap.add_argument("--no-nuts", action="store_true", help="skip the NUTS measurement")
    ap.add_argument("--nuts-warmup", type=int, default=10, help="NUTS warm-up iterations (bench line; "
                    "--study nuts: use e.g. 500)")
    ap.add_argument("--nuts-samples", type=int, default=10)
    ap.add_argument("--profile", choices=["loglike", "round", "cmb", "grad"], default=None,
                    help="run a short fixed workload for a profiler and exit (no timing line): "
                         "'loglike' = 4 loglike_batch calls of --batch rows on the 39-d shear problem, "
                         "'round' = two warm NS iterations then one more inside an NVTX range 'prof', "
                         "'cmb' = 4 loglike_batch calls on the D = 7521 CMB problem, "
                         "'grad' = 4 loglike_grad_batch calls of --batch rows on the 39-d shear problem")
    ap.add_argument("--batch", type=int, default=500)
    ap.add_argument("--hidden-tile", type=int, default=0,
                    help="--profile: force the N-tile width (16/32/64/128) of the BF16 hidden layers (0: autotuned)")
    ap.add_argument("--study", choices=["evidence", "oracle", "nuts"], default=None,
                    help="one-off measurements printed as one JSON line (no timing line): 'evidence' = log Z and "
                         "log B01 of the 39-d w0-wa vs 37-d LCDM runs over --seeds in each of --precisions, the "
                         "interpolated-P(k) runs on the same data and the full - interpolated log L offset over "
                         "the posterior; 'oracle' = the CPU oracle's evaluation rates (1 and all host threads) and "
                         "full nested-sampling runs, with the 6-d CMB and 39-d shear times extrapolated from "
                         "rates x the GPU runs' evaluation counts; 'nuts' = the HMC comparison: NUTS on the "
                         "hand-written adjoint (64 chains, --nuts-warmup + --nuts-samples iterations) against the "
                         "nested-sampling posterior of the same problem")
    ap.add_argument("--seeds", default="3,4,5")
    ap.add_argument("--precisions", default="bf16,fp32")
    ap.add_argument("--oracle-limit", type=float, default=900.0, help="seconds allowed per full oracle run")
    ap.add_argument("--oracle-parts", default="rates,runs,gpu",
                    help="--study oracle: any of rates (oracle evaluation rates), runs (full oracle runs), gpu (the "
                         "GPU runs and the extrapolations; run alone, nothing else on the GPU)")
    args = ap.parse_args()
    if args.profile:
        return profile_workload(args)
    if args.study == "evidence":
        return evidence_study(args)
    if args.study == "oracle":
        return oracle_study(args)
    if args.study == "nuts":
        return nuts_study(args)
    if args.impl == "reference":
        return reference_arm(args)
    return ours(args)


def profile_workload(args):
    """Short fixed workloads to run under ncu (the launch list and single-kernel
    captures of profiles/); prints nothing but a completion line."""
    import numpy as np
    import torch
    from paper_2509_13307_gb300.build import build
    build()
    import workloads as w
    from paper_2509_13307_gb300 import Problem, NestedRun
    if args.profile == "cmb":
        inp = w.make_cmb_inputs(w.cmb6())
        prob = Problem(inp, args.precision if args.precision != "bf16" else "fp32", max_batch=args.batch)
    else:
        inp = w.make_shear_inputs(w.shear39())
        prob = Problem(inp, args.precision, max_batch=max(args.batch, 1000),   # grad: max_batch sizes its workspace
                       hidden_tile=args.hidden_tile)
    if args.profile == "round":
        sc = w.shear39().sampler
        run = NestedRun.from_config(prob, sc)
        run.step(2)
        torch.cuda.synchronize()
        torch.cuda.nvtx.range_push("prof")
        run.step(1)
        torch.cuda.nvtx.range_pop()
        torch.cuda.synchronize()
    else:
        free = [i for i, p in enumerate(inp["priors"]) if p[0] != "F"]
        cube = torch.tensor(np.random.default_rng(9).uniform(0.02, 0.98, (args.batch, len(free))), device="cuda")
        th = prob.prior_transform(cube)
        for _ in range(4):
            if args.profile == "grad":
                prob.loglike_grad(th)
            else:
                prob.loglike(th)
        torch.cuda.synchronize()
    print(f"profile workload {args.profile} done", flush=True)
    return 0


def evidence_study(args):
    """The benchmark spec's evidence check on the 39-d shear problem: nested
    sampling to a converged log Z of the w0-wa (39-d) and LCDM (37-d, w0 = -1,
    wa = 0 fixed) models on the same mock data, per seed and precision; log
    B01 = ln Z_LCDM - ln Z_w0wa (Eq. 2) with error sqrt(s0^2 + s1^2); the same
    with the emulator on 10 coarse z nodes interpolated to the 50-node table
    (Catmull-Rom, and linear as in the paper's interpolated likelihood, App. B)
    on the full problem's data; and the full - interpolated log L offset over
    posterior samples of the full BF16 runs (FP64 likelihoods)."""
    from dataclasses import replace
    import numpy as np
    import torch
    from paper_2509_13307_gb300.build import build
    build()
    import workloads as w
    from paper_2509_13307_gb300 import Problem, NestedRun
    seeds = [int(x) for x in args.seeds.split(",") if x]
    precs = [x for x in args.precisions.split(",") if x]
    models = {"w0wa": w.shear39(), "lcdm": w.shear37_lcdm()}
    interp = {"catmull_rom": {"w0wa": w.shear39_interp(), "lcdm": w.shear37_interp()},
              "linear": {"w0wa": w.shear39_interp_linear(),
                         "lcdm": replace(w.shear37_interp(), name="shear37_interp_linear", z_interp="linear")}}
    inps = {m: w.make_shear_inputs(c) for m, c in models.items()}
    base = Problem(inps["w0wa"], "fp64", max_batch=8)
    data, cov = base.data, base.cov
    base.close()
    out = {"workload": WORKLOAD, "seeds": seeds, "runs": [], "bayes": {}}
    posts = {}

    def one(cfg, inp, prec, seed, tag):
        sc = cfg.sampler
        p = Problem(inp, prec, max_batch=sc.n_live, data=data, cov=cov)
        torch.cuda.synchronize()
        t0 = time.time()
        r = NestedRun(p, sc.n_live, sc.n_delete, sc.repeats, sc.tol, seed, sc.width, sc.step_cap, sc.ridge)
        st = r.run(max_iters=5000)
        ev = r.evidence()
        dt = time.time() - t0
        rec = dict(tag=tag, precision=prec, seed=seed, d=p.d, seconds=dt, iterations=st.iterations,
                   evaluations=st.evaluations, converged=st.converged, status_bits=st.status_bits,
                   nonfinite=st.nonfinite, logZ=ev["logZ"], logZ_err=ev["logZ_err"], H=ev["H"])
        if prec == "bf16" and tag.startswith("full") and seed == seeds[0]:
            posts[tag] = (r.posterior(), inp)
        r.close()
        p.close()
        out["runs"].append(rec)
        print(json.dumps(rec), file=sys.stderr, flush=True)
        return rec

    def bayes(recs0, recs1):
        lb = [a["logZ"] - b["logZ"] for a, b in zip(recs0, recs1)]
        eb = [math.hypot(a["logZ_err"], b["logZ_err"]) for a, b in zip(recs0, recs1)]
        return dict(logB01_per_seed=lb, err_per_seed=eb, logB01_mean=float(np.mean(lb)),
                    logB01_seed_sd=float(np.std(lb, ddof=1)) if len(lb) > 1 else None,
                    logZ_lcdm=[a["logZ"] for a in recs0], logZ_w0wa=[b["logZ"] for b in recs1])

    for prec in precs:
        rl = [one(models["lcdm"], inps["lcdm"], prec, sd, "full_lcdm") for sd in seeds]
        rw = [one(models["w0wa"], inps["w0wa"], prec, sd, "full_w0wa") for sd in seeds]
        out["bayes"][f"full_{prec}"] = bayes(rl, rw)
    for kind, cf in interp.items():
        ii = {m: w.make_shear_inputs(c) for m, c in cf.items()}
        rl = [one(cf["lcdm"], ii["lcdm"], "bf16", sd, f"interp_{kind}_lcdm") for sd in seeds]
        rw = [one(cf["w0wa"], ii["w0wa"], "bf16", sd, f"interp_{kind}_w0wa") for sd in seeds]
        out["bayes"][f"interp_{kind}_bf16"] = bayes(rl, rw)
        # full - interpolated log L (FP64) over posterior samples of the full runs
        for m in ("w0wa", "lcdm"):
            key = f"full_{m}"
            if key not in posts:
                continue
            (x, lg, logw), inp_full = posts[key]
            rng = np.random.default_rng(11)
            idx = rng.choice(len(logw), size=512, p=np.exp(logw))
            cube = torch.tensor(x[idx], dtype=torch.float64, device="cuda")
            pf = Problem(inp_full, "fp64", max_batch=512, data=data, cov=cov)
            pi = Problem(ii[m], "fp64", max_batch=512, data=data, cov=cov)
            th = pf.prior_transform(cube)
            dl = (pf.loglike(th) - pi.loglike(th)).cpu().numpy()
            out.setdefault("offset", {})[f"{kind}_{m}"] = dict(
                mean=float(np.mean(dl)), sd=float(np.std(dl, ddof=1)), min=float(np.min(dl)), max=float(np.max(dl)),
                samples=512, how="FP64 log L_full - log L_interp at 512 posterior draws of the full BF16 run")
            pf.close()
            pi.close()
    print(json.dumps(out), flush=True)
    return 0


def posterior_moments(theta, logw):
    """Weighted mean and standard deviation of nested-sampling posterior
    samples, and the Kish effective sample size of the weights."""
    import numpy as np
    w = np.exp(logw - np.max(logw))
    w /= w.sum()
    mean = w @ theta
    sd = np.sqrt(np.maximum(w @ (theta - mean) ** 2, 0.0))
    return mean, sd, 1.0 / np.sum(w * w)


def nuts_study(args):
    """The HMC comparison of the paper (Sec. 3.2, Table 2's NUTS rows) on the
    39-d shear problem: NUTS (64 chains in lockstep on the hand-written
    adjoint, dual averaging to a 0.8 acceptance target, diagonal mass matrix
    from warm-up) started from nested-sampling posterior draws, and its
    posterior means and standard deviations against the weighted dead points
    of a converged nested-sampling run of the same problem and precision."""
    import numpy as np
    import torch
    from paper_2509_13307_gb300.build import build
    build()
    import workloads as w
    from paper_2509_13307_gb300 import Problem, NestedRun, nuts
    cfg = w.shear39()
    inp = w.make_shear_inputs(cfg)
    sc = cfg.sampler
    prob = Problem(inp, args.precision, max_batch=sc.n_live)
    t0 = time.time()
    run = NestedRun.from_config(prob, sc)
    st = run.run(max_iters=5000)
    ev = run.evidence()
    t_ns = time.time() - t0
    x, lg, logw = run.posterior()
    run.close()
    B = prob.max_batch
    theta = np.concatenate([prob.prior_transform(torch.tensor(x[i:i + B], device="cuda")).cpu().numpy()
                            for i in range(0, len(x), B)])
    m_ns, s_ns, ess_ns = posterior_moments(theta, logw)
    n_ch = 64
    rng = np.random.default_rng(12)
    pick = rng.choice(len(logw), size=n_ch, p=np.exp(logw))
    xc = np.clip(x[pick], 1e-9, 1 - 1e-9)
    z0 = np.log(xc) - np.log1p(-xc)
    pn = Problem(inp, args.precision, max_batch=n_ch, data=prob.data, cov=prob.cov)
    torch.cuda.synchronize()
    t0 = time.time()
    out = nuts(pn, n_ch, args.nuts_warmup, args.nuts_samples, z0=z0, seed=5, init_step=0.02, max_depth=10)
    t_nuts = time.time() - t0
    th = out["theta"]                                   # chains x samples x d
    m_hmc = th.reshape(-1, th.shape[-1]).mean(axis=0)
    s_hmc = th.reshape(-1, th.shape[-1]).std(axis=0)
    se_hmc = th.mean(axis=1).std(axis=0, ddof=1) / np.sqrt(n_ch)   # spread of chain means
    se_ns = s_ns / np.sqrt(ess_ns)
    zsc = (m_hmc - m_ns) / np.sqrt(se_hmc ** 2 + se_ns ** 2)
    names = [inp["param_names"][i] for i, p in enumerate(inp["priors"]) if p[0] != "F"]
    stn = out["stats"]
    res = {"workload": WORKLOAD, "precision": args.precision,
           "ns": {"seconds": t_ns, "evaluations": st.evaluations, "logZ": ev["logZ"], "logZ_err": ev["logZ_err"],
                  "ess": ess_ns, "status_bits": st.status_bits},
           "nuts": {"chains": n_ch, "warmup": args.nuts_warmup, "samples": args.nuts_samples, "seconds": t_nuts,
                    "gradient_evals": stn["gradient_evals"], "grad_evals_per_s": stn["gradient_evals"] / t_nuts,
                    "batched_calls": stn["batched_calls"], "mean_depth": stn["mean_depth"],
                    "mean_accept": stn["mean_accept"], "divergences": stn["divergences"],
                    "init": "64 draws from the nested-sampling posterior"},
           "compare": {"param": names, "mean_ns": m_ns.tolist(), "sd_ns": s_ns.tolist(), "mean_nuts": m_hmc.tolist(),
                       "sd_nuts": s_hmc.tolist(), "z_mean": zsc.tolist(), "max_abs_z": float(np.max(np.abs(zsc))),
                       "sd_ratio_min": float(np.min(s_hmc / s_ns)), "sd_ratio_max": float(np.max(s_hmc / s_ns)),
                       "how": "z = (mean_nuts - mean_ns) / sqrt(se_nuts^2 + se_ns^2); se_nuts from the spread of "
                              "the 64 chain means, se_ns = sd / sqrt(Kish ESS of the NS weights)"}}
    print(json.dumps(res), flush=True)
    return 0


def _host_info():
    info = {"nproc": os.cpu_count(), "machine": os.uname().machine}
    try:
        with open("/proc/cpuinfo") as fh:
            txt = fh.read()
        for key in ("model name", "CPU part", "Hardware"):
            for line in txt.splitlines():
                if line.startswith(key):
                    info[key.replace(" ", "_")] = line.split(":", 1)[1].strip()
                    break
    except OSError:
        pass
    try:
        r = subprocess.run(["lscpu"], capture_output=True, text=True, timeout=20)
        for line in r.stdout.splitlines():
            if line.startswith("Model name"):
                info["model_name"] = line.split(":", 1)[1].strip()
    except (OSError, subprocess.SubprocessError):
        pass
    return info


def _oracle_subprocess(code: str, threads: int, timeout: float):
    env = dict(os.environ)
    for k in ("OMP_NUM_THREADS", "OPENBLAS_NUM_THREADS", "MKL_NUM_THREADS", "NUMEXPR_NUM_THREADS"):
        env[k] = str(threads)
    env["CUDA_VISIBLE_DEVICES"] = ""
    r = subprocess.run([sys.executable, "-c", code], capture_output=True, text=True, env=env, timeout=timeout)
    if r.returncode != 0:
        return {"error": r.stderr[-400:]}
    return json.loads(r.stdout.strip().splitlines()[-1])


_ORACLE_RATE = r"""
import sys, time, json
sys.path.insert(0, %(root)r)
import numpy as np
import workloads as w
kind = %(kind)r
if kind == "cmb6":
    from oracle.cmb import CMBOracle
    o = CMBOracle(w.make_cmb_inputs(w.cmb6()))
    d = 6
else:
    from oracle.shear import ShearOracle
    cfg = getattr(w, kind)()
    o = ShearOracle(w.make_shear_inputs(cfg))
    d = cfg.d_free
rng = np.random.default_rng(0)
o.loglike_cube(rng.uniform(0.02, 0.98, d))
n = 0; t0 = time.time()
while time.time() - t0 < %(seconds)f or n < 2:
    o.loglike_cube(rng.uniform(0.02, 0.98, d)); n += 1
print(json.dumps({"n": n, "s": time.time() - t0}))
"""

_ORACLE_RUN = r"""
import sys, time, json
sys.path.insert(0, %(root)r)
import numpy as np
import workloads as w
from oracle.ns import NestedSampler
kind = %(kind)r
if kind == "gauss5":
    from oracle.gauss import GaussOracle
    cfg = w.gauss_test(5)
    f = GaussOracle(w.make_gauss_inputs(cfg)).loglike
    d = 5
else:
    from oracle.shear import ShearOracle
    cfg = getattr(w, kind)()
    f = ShearOracle(w.make_shear_inputs(cfg)).loglike_cube
    d = cfg.d_free
ns = NestedSampler.from_config(f, d, cfg.sampler)
t0 = time.time()
ns.initialise()
while not ns.converged() and time.time() - t0 < %(limit)f:
    ns.iterate()
dt = time.time() - t0
ev = ns.evidence(n_replays=200) if ns.converged() else {}
print(json.dumps({"seconds": dt, "converged": ns.converged(), "iterations": ns.it, "evaluations": ns.n_evals,
                  "logZ": ev.get("logZ"), "logZ_err": ev.get("logZ_err")}))
"""


def oracle_study(args):
    """The oracle as a baseline (FP64 NumPy on the host cores of the machine that runs the bench):
    evaluation rates at 1 and all threads for the 5-d toy, the 6-d CMB problem
    and the 39-d shear problem; full nested-sampling runs of the 5-d Gaussian
    test problem and the 5-d shear toy (bounded by --oracle-limit seconds);
    for the 6-d CMB and 39-d shear problems, whose oracle runs would take
    hours to days, the time to a converged log Z is extrapolated as the GPU
    run's evaluation count / the oracle's rate, and labelled as such."""
    nproc = os.cpu_count() or 1
    parts = set(args.oracle_parts.split(","))
    out = {"host": _host_info(), "rates": {}, "runs": {}, "extrapolated": {}}
    secs = {"shear5": 15.0, "cmb6": 20.0, "shear39": 15.0} if "rates" in parts else {}
    for kind, sec in secs.items():
        for th in sorted({1, nproc}):
            r = _oracle_subprocess(_ORACLE_RATE % dict(root=ROOT, kind=kind, seconds=sec), th, 1800)
            if "n" in r:
                r = {"evals_per_s": r["n"] / r["s"], "evals": r["n"], "seconds": r["s"]}
            out["rates"][f"{kind}_threads{th}"] = r
            print(json.dumps({kind: r, "threads": th}), file=sys.stderr, flush=True)
    for kind in (("gauss5", "shear5") if "runs" in parts else ()):
        r = _oracle_subprocess(_ORACLE_RUN % dict(root=ROOT, kind=kind, limit=args.oracle_limit), 1,
                               args.oracle_limit + 600)
        r["threads"] = 1
        out["runs"][kind] = r
        print(json.dumps({kind: r}), file=sys.stderr, flush=True)
    if "gpu" not in parts:
        print(json.dumps(out), flush=True)
        return 0
    # GPU runs for the evaluation counts of the extrapolations (and the GPU's own times)
    import torch
    from paper_2509_13307_gb300.build import build
    build()
    import workloads as w
    from paper_2509_13307_gb300 import Problem, NestedRun
    gpu = {}
    for kind, cfg, inp_fn, prec in (("gauss5", w.gauss_test(5), w.make_gauss_inputs, "fp64"),
                                    ("shear5", w.shear5(), w.make_shear_inputs, "fp64"),
                                    ("cmb6", w.cmb6(), w.make_cmb_inputs, "fp32"),
                                    ("shear39", w.shear39(), w.make_shear_inputs, "bf16")):
        sc = cfg.sampler
        p = Problem(inp_fn(cfg), prec, max_batch=max(sc.n_live, 2 * sc.n_delete))
        torch.cuda.synchronize()
        t0 = time.time()
        r = NestedRun.from_config(p, sc)
        st = r.run(max_iters=100000)
        ev = r.evidence()
        gpu[kind] = dict(seconds=time.time() - t0, evaluations=st.evaluations, iterations=st.iterations,
                         precision=prec, logZ=ev["logZ"], logZ_err=ev["logZ_err"])
        r.close()
        p.close()
    out["gpu_runs"] = gpu
    for kind in ("shear5", "cmb6", "shear39"):
        for th in sorted({1, nproc}):
            rate = out["rates"].get(f"{kind}_threads{th}", {}).get("evals_per_s")
            if rate:
                out["extrapolated"][f"{kind}_threads{th}"] = dict(
                    seconds=gpu[kind]["evaluations"] / rate, label="extrapolated: GPU run's evaluation count / "
                    "oracle evaluations per second (not a measured oracle run)")
    print(json.dumps(out), flush=True)
    return 0


def reference_arm(args):
    world = _env_int("WORLD_SIZE", 1)
    rank = _env_int("RANK", 0)
    if world > 1 and rank != 0:
        return 0
    import numpy as np
    import workloads as w
    from oracle.shear import ShearOracle
    inp = w.make_shear_inputs(w.shear39())
    o = ShearOracle(inp)
    rng = np.random.default_rng(0)
    per_step = 24
    for _ in range(args.warmup):
        for _ in range(per_step):
            o.loglike_cube(rng.uniform(0.02, 0.98, 39))
    t0 = time.time()
    for _ in range(args.steps):
        for _ in range(per_step):
            o.loglike_cube(rng.uniform(0.02, 0.98, 39))
    dt = time.time() - t0
    val = args.steps * per_step / dt
    threads = os.environ.get("OPENBLAS_NUM_THREADS") or os.environ.get("OMP_NUM_THREADS") or str(os.cpu_count())
    line = {"impl": "reference", "metric": METRIC, "value": val, "unit": UNIT, "n_gpus": args.gpus,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": 1e3 * dt / args.steps,
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
            "data": "synthetic", "config": {"workload": WORKLOAD, "sample": f"{per_step} evaluations per step"},
            "cpu_baseline": {"value": val, "unit": UNIT, "cores": int(threads), "kind": "oracle",
                             "sample": f"{per_step} oracle log-likelihood evaluations per step at random prior points"},
            "e2e": {"value": val, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)
    return 0


def ours(args):
    import numpy as np
    import torch
    import torch.distributed as dist

    world = _env_int("WORLD_SIZE", 1)
    rank = _env_int("RANK", 0)
    local = _env_int("LOCAL_RANK", 0)
    if world > 1:
        torch.cuda.set_device(local)
        dist.init_process_group("nccl")
    dev = torch.device("cuda", torch.cuda.current_device())

    from paper_2509_13307_gb300.build import build
    build()
    import workloads as w
    from paper_2509_13307_gb300 import Problem, NestedRun

    cfg = w.shear39()
    inp = w.make_shear_inputs(cfg)
    sc = cfg.sampler
    seed = sc.seed + rank

    def barrier():
        if world > 1:
            dist.barrier()

    flush = torch.empty(256 * 1024 * 1024 // 4, dtype=torch.float32, device=dev)
    stream = torch.cuda.current_stream()

    def timed_steps(prob, n_warm, n_steps, profile=None):
        run = NestedRun(prob, sc.n_live, sc.n_delete, sc.repeats, sc.tol, seed, sc.width, sc.step_cap, sc.ridge)
        for _ in range(n_warm):
            run.step(1)
        if profile:
            run.profile_stage(profile)
        st0 = run.step(0)
        ms = 0.0
        for _ in range(n_steps):
            flush.fill_(1.0)
            torch.cuda.synchronize()
            barrier()
            e0 = torch.cuda.Event(enable_timing=True)
            e1 = torch.cuda.Event(enable_timing=True)
            e0.record(stream)
            run.step(1)
            e1.record(stream)
            torch.cuda.synchronize()
            ms += e0.elapsed_time(e1)
        barrier()
        st1 = run.step(0)
        prof = run.profile_read() if profile else None
        out = dict(ms=ms, evals=st1.evaluations - st0.evaluations, rounds=st1.rounds - st0.rounds,
                   iters=st1.iterations - st0.iterations, prof=prof, status=st1.status_bits,
                   nonfinite=st1.nonfinite)
        run.close()
        return out

    # ---------------- main arm: BF16 likelihood, timed NS steps
    prob = Problem(inp, args.precision, max_batch=sc.n_live)
    clocks = ClockSampler(torch.cuda.current_device() if world == 1 else local)
    clocks.start()
    res = timed_steps(prob, args.warmup, args.steps, profile="projection")
    clk = clocks.stop()

    t_local, ev_local = res["ms"] / 1e3, res["evals"]
    t_job, ev_job = job_totals(t_local, ev_local, world, dev)
    value = ev_job / t_job

    # per round (one chain group): slice (with the prior transform and the
    # next round's batch-counter reset), windows, the emulator (the fused
    # input + hidden-layer kernel and the output GEMM, or the input layer and
    # one GEMM per further layer), Limber, whitening; per iteration 7 more
    # (sort and delete, column means, covariance, Cholesky, directions, chain
    # starts, insert).
    n_layers = len(inp["emu_W"])
    per_round = 4 + (2 if prob.fused_cluster() else n_layers)
    gpu_launches = res["rounds"] * per_round + 7 * res["iters"]

    # ---------------- roofline of the dominant kernel (Limber stage), timed live
    prof = res["prof"]
    flops = limber_method_flops_per_eval(cfg)
    peak = fp32_alu_peak_tflops(2070.0)
    roofline = None
    if prof and prof["launches"] > 0 and prof["ms"] > 0:
        achieved = prof["rows"] * flops / (prof["ms"] * 1e-3) / 1e12
        roofline = {"bound": "alu", "achieved": achieved, "peak": peak, "unit": "TFLOP/s",
                    "frac": achieved / peak, "traffic": limber_traffic(prof["rows"] / prof["launches"]),
                    "traffic_unit": "bytes per launch (ncu dram__bytes_read.sum + dram__bytes_write.sum, "
                                    "scaled from 460 evaluations)",
                    "kernel": "k_limber<float,5,fast> (A10-A12: P lookup, Limber sums, data vector)",
                    "flop_per_eval": flops,
                    "flop_basis": "A10 + A11L method count 2 n_ell N_chi (16 + n_pairs); the kernel's full "
                                  "instruction-level count incl. weights and indexing is kernel_flop_per_eval",
                    "kernel_flop_per_eval": limber_flops_per_eval(cfg),
                    "avg_launch_ms": prof["ms"] / prof["launches"],
                    "avg_rows_per_launch": prof["rows"] / prof["launches"],
                    "peak_basis": "FP32 ALU 152 SM x 128 lanes x 2 x 2070 MHz (no measured FP32 peak in MEASURED_PEAKS.json)"}
        if roofline["traffic"]:
            # the same kernel against HBM: measured bytes per launch / launch time
            gbs = roofline["traffic"] / (roofline["avg_launch_ms"] * 1e-3) / 1e9
            roofline["hbm_achieved_GBps"] = gbs
            roofline["hbm_frac"] = gbs / measured_peaks()["hbm_gbs"]

    extra = {}
    # ---------------- the emulator's output layer (tcgen05) against the
    # measured sustained bf16 tensor peak, timed live in the rounds
    try:
        r_emu = timed_steps(prob, 1, 2, profile="emu_out")
        pe = r_emu["prof"]
        if pe and pe["launches"] > 0 and pe["ms"] > 0:
            k_out = inp["emu_W"][-1].shape
            flop_row = 2.0 * k_out[0] * k_out[1]
            ach = pe["rows"] * flop_row / (pe["ms"] * 1e-3) / 1e12
            pk = measured_peaks()["bf16_tflops_sustained"]
            extra["roofline_emulator_output_gemm"] = {
                "bound": "tensor", "achieved": ach, "peak": pk, "unit": "TFLOP/s", "frac": ach / pk,
                "kernel": "k_gemm_tc_swap<256> (emulator output layer %d -> %d, bf16 x bf16 -> fp32)" % (k_out[1], k_out[0]),
                "avg_launch_ms": pe["ms"] / pe["launches"], "avg_rows_per_launch": pe["rows"] / pe["launches"],
                "peak_basis": "measured cuBLAS bf16 sustained (MEASURED_PEAKS.json)"}
    except Exception as exc:
        extra["roofline_emulator_output_gemm_error"] = repr(exc)[:200]
    # ---------------- plain FP32 form on the same workload
    if args.precision != "fp32":
        p32 = Problem(inp, "fp32", max_batch=sc.n_live)
        r32 = timed_steps(p32, 1, 2)
        p32.close()
        extra["fp32_evals_per_s"] = r32["evals"] / (r32["ms"] / 1e3)
        extra["speedup_vs_fp32"] = value / extra["fp32_evals_per_s"] if world == 1 else \
            (ev_local / t_local) / extra["fp32_evals_per_s"]
    extra["iters_per_s"] = res["iters"] / t_local
    extra["rounds_per_step"] = res["rounds"] / max(res["iters"], 1)

    # ---------------- adjoint throughput (B = 4096 parameter vectors, hand-written adjoint)
    try:
        Bg = 4096
        pg = Problem(inp, args.precision, max_batch=Bg)
        rng_g = np.random.default_rng(4 + rank)
        free_g = [i for i, p in enumerate(inp["priors"]) if p[0] != "F"]
        thg = pg.prior_transform(torch.tensor(rng_g.uniform(0.02, 0.98, (Bg, len(free_g))), device=dev))
        for _ in range(2):
            pg.loglike_grad(thg)
        torch.cuda.synchronize()
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        for _ in range(3):
            pg.loglike_grad(thg)
        e1.record(stream)
        torch.cuda.synchronize()
        extra["grad_evals_per_s"] = 3 * Bg / (e0.elapsed_time(e1) / 1e3)
        extra["grad_batch"] = Bg
        pg.close()
    except Exception as exc:  # report, do not hide, a failure of this extra measurement
        extra["grad_error"] = repr(exc)[:200]

    # ---------------- packed uneven runs (8 runs, interpolated emulator)
    if not args.no_multi:
        try:
            from paper_2509_13307_gb300 import MultiRun
            cfgs = w.uneven_runs()
            base = w.make_shear_inputs(cfgs[1])
            probs = []
            for c in cfgs:
                ci = w.make_shear_inputs(c)
                probs.append(Problem(ci, args.precision, max_batch=c.sampler.n_live,
                                     data=None if not probs else probs[0].data,
                                     cov=None if not probs else probs[0].cov))
            mr = MultiRun(probs, [replace_seed(c.sampler, rank) for c in cfgs])
            mr.step(1)
            torch.cuda.synchronize()
            e0 = torch.cuda.Event(enable_timing=True)
            e1 = torch.cuda.Event(enable_timing=True)
            ev0 = sum(s.evaluations for s in mr.step(0))
            e0.record(stream)
            sts = mr.step(2)
            e1.record(stream)
            torch.cuda.synchronize()
            extra["packed_runs_evals_per_s"] = (sum(s.evaluations for s in sts) - ev0) / (e0.elapsed_time(e1) / 1e3)
            extra["packed_runs"] = "8 runs, d in {37, 39, 33}, n_live in {250, 500, 1000, 2000}, k = n/2, emulator on 10 z nodes interpolated to 50"
            mr.close()
            for q in probs:
                q.close()
            del base
        except Exception as exc:
            extra["packed_runs_error"] = repr(exc)[:200]

    # ---------------- wall time to a converged log Z (BF16), from ns_init
    if not args.no_full_run:
        torch.cuda.synchronize()
        t0 = time.time()
        run = NestedRun(prob, sc.n_live, sc.n_delete, sc.repeats, sc.tol, seed, sc.width, sc.step_cap, sc.ridge)
        st = run.run(max_iters=2000)
        ev = run.evidence()
        t1 = time.time()
        extra.update(time_to_logZ_s=t1 - t0, logZ=ev["logZ"], logZ_err=ev["logZ_err"], logZ_iters=st.iterations,
                     logZ_evals=st.evaluations, logZ_converged=st.converged, logZ_status_bits=st.status_bits,
                     logZ_nonfinite_evals=st.nonfinite)
        run.close()
        # the nested LCDM model (w0 = -1, wa = 0 fixed, 37-d) on the same data:
        # the Bayes factor B01 = Z_LCDM / Z_w0wa (Eq. 2)
        try:
            c37 = w.shear37_lcdm()
            p37 = Problem(w.make_shear_inputs(c37), args.precision, max_batch=sc.n_live, data=prob.data,
                          cov=prob.cov)
            torch.cuda.synchronize()
            t0 = time.time()
            r37 = NestedRun(p37, sc.n_live, sc.n_delete, sc.repeats, sc.tol, seed, sc.width, sc.step_cap, sc.ridge)
            s37 = r37.run(max_iters=2000)
            e37 = r37.evidence()
            extra["bayes"] = {"logZ_w0wa": ev["logZ"], "logZ_w0wa_err": ev["logZ_err"],
                              "logZ_lcdm": e37["logZ"], "logZ_lcdm_err": e37["logZ_err"],
                              "logB01": e37["logZ"] - ev["logZ"],
                              "logB01_err": math.hypot(e37["logZ_err"], ev["logZ_err"]),
                              "lcdm_time_to_logZ_s": time.time() - t0, "lcdm_evals": s37.evaluations,
                              "lcdm_status_bits": s37.status_bits, "precision": args.precision,
                              "models": "B01 = Z(LCDM, 37-d) / Z(w0-wa, 39-d), same mock data, seed %d" % seed}
            r37.close()
            p37.close()
        except Exception as exc:
            extra["bayes_error"] = repr(exc)[:200]
        # the plain FP32 form's wall time to a converged log Z on the same problem
        if not args.no_fp32_run and args.precision != "fp32":
            p32 = Problem(inp, "fp32", max_batch=sc.n_live, data=prob.data, cov=prob.cov)
            torch.cuda.synchronize()
            t0 = time.time()
            r32 = NestedRun(p32, sc.n_live, sc.n_delete, sc.repeats, sc.tol, seed, sc.width, sc.step_cap, sc.ridge)
            s32 = r32.run(max_iters=2000)
            e32 = r32.evidence()
            extra.update(fp32_time_to_logZ_s=time.time() - t0, fp32_logZ=e32["logZ"], fp32_logZ_err=e32["logZ_err"],
                         fp32_logZ_evals=s32.evaluations, fp32_logZ_status_bits=s32.status_bits,
                         time_to_logZ_speedup_vs_fp32=(time.time() - t0) / extra["time_to_logZ_s"])
            r32.close()
            p32.close()

    # ---------------- NUTS on the adjoint (the HMC comparison of the 39-d
    # shear problem): 64 chains in lockstep, a short warm-up and sample
    if not args.no_nuts:
        try:
            from paper_2509_13307_gb300 import nuts
            pn = Problem(inp, args.precision, max_batch=64)
            torch.cuda.synchronize()
            t0 = time.time()
            out = nuts(pn, 64, args.nuts_warmup, args.nuts_samples, seed=5 + rank, init_step=0.02, max_depth=8)
            dt = time.time() - t0
            stn = out["stats"]
            extra.update(nuts_chains=64, nuts_warmup=args.nuts_warmup, nuts_samples=args.nuts_samples,
                         nuts_seconds=dt, nuts_grad_evals_per_s=stn["gradient_evals"] / dt,
                         nuts_iters_per_s=64 * (args.nuts_warmup + args.nuts_samples) / dt,
                         nuts_mean_depth=stn["mean_depth"], nuts_mean_accept=stn["mean_accept"],
                         nuts_divergences=stn["divergences"])
            pn.close()
        except Exception as exc:
            extra["nuts_error"] = repr(exc)[:200]

    # ---------------- the 6-parameter CMB configuration (D = 7521, dense
    # covariance, whitening fold, FP32 emulator): NS evaluations/s and the wall
    # time to a converged log Z
    if not args.no_cmb:
        try:
            ccfg = w.cmb6()
            cinp = w.make_cmb_inputs(ccfg)
            csc = replace_seed(ccfg.sampler, rank)
            t_setup = time.time()
            pc = Problem(cinp, "fp32", max_batch=csc.n_live)
            torch.cuda.synchronize()
            t_setup = time.time() - t_setup
            crun = NestedRun.from_config(pc, csc)
            crun.step(1)
            torch.cuda.synchronize()
            e0 = torch.cuda.Event(enable_timing=True)
            e1 = torch.cuda.Event(enable_timing=True)
            s0 = crun.step(0)
            e0.record(stream)
            s1 = crun.step(3)
            e1.record(stream)
            torch.cuda.synchronize()
            extra["cmb_evals_per_s"] = (s1.evaluations - s0.evaluations) / (e0.elapsed_time(e1) / 1e3)
            crun.close()
            t0 = time.time()
            crun = NestedRun.from_config(pc, csc)
            cst = crun.run(max_iters=5000)
            cev = crun.evidence()
            extra.update(cmb_time_to_logZ_s=time.time() - t0, cmb_logZ=cev["logZ"], cmb_logZ_err=cev["logZ_err"],
                         cmb_iters=cst.iterations, cmb_evals=cst.evaluations, cmb_converged=cst.converged,
                         cmb_setup_s=t_setup,
                         cmb_workload="cmb6: 6-parameter LCDM CMB-like, emulator 6->4x512->3x2507 sigmoid-linear "
                                      "(FP32), dense 7521 x 7521 Wishart-style covariance, whitening fold, "
                                      "n_live = 500, k = 250")
            crun.close()
            pc.close()
        except Exception as exc:
            extra["cmb_error"] = repr(exc)[:200]
        # the paper's own CMB likelihood form: cosmic-variance-limited TT
        try:
            ptt = Problem(cinp, "fp32", max_batch=csc.n_live, form="tt_cv")
            t0 = time.time()
            trun = NestedRun.from_config(ptt, csc)
            tst = trun.run(max_iters=5000)
            tev = trun.evidence()
            extra.update(cmb_tt_time_to_logZ_s=time.time() - t0, cmb_tt_logZ=tev["logZ"],
                         cmb_tt_logZ_err=tev["logZ_err"], cmb_tt_evals=tst.evaluations,
                         cmb_tt_converged=tst.converged)
            trun.close()
            ptt.close()
        except Exception as exc:
            extra["cmb_tt_error"] = repr(exc)[:200]

    # ---------------- end to end through the public API with host buffers
    B = sc.n_delete
    rng = np.random.default_rng(rank)
    free = [i for i, p in enumerate(inp["priors"]) if p[0] != "F"]
    host_theta = torch.empty((B, len(free)), dtype=torch.float64).pin_memory()
    host_out = torch.empty(B, dtype=torch.float64).pin_memory()
    cube = torch.tensor(rng.uniform(0.05, 0.95, (B, len(free))), device=dev)
    host_theta.copy_(prob.prior_transform(cube).cpu())
    for _ in range(3):
        prob.loglike(host_theta.to(dev, non_blocking=True))
    reps = 40
    torch.cuda.synchronize()
    t0 = time.time()
    for _ in range(reps):
        th = host_theta.to(dev, non_blocking=True)
        host_out.copy_(prob.loglike(th), non_blocking=True)
    torch.cuda.synchronize()
    e2e = {"value": reps * B / (time.time() - t0), "unit": UNIT,
           "h2d_bytes_per_step": B * len(free) * 8, "d2h_bytes_per_step": B * 8,
           "how": "loglike_batch on B = 500 parameter vectors from pinned host memory, H2D + call + D2H per step"}

    cpu = None
    if rank == 0 and not args.no_cpu:
        cpu = cpu_oracle_rate()

    if rank == 0:
        line = {"metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": args.steps,
                "warmup": args.warmup, "ms_per_step": res["ms"] / args.steps, "higher_is_better": True,
                "scaling": "weak", "vs_baseline": None, "dtype": args.precision, "data": "synthetic",
                "config": {"workload": WORKLOAD, "precision": args.precision,
                           "l2": "flushed between timed steps (256 MB write)",
                           "evals_per_step": res["evals"] / max(res["iters"], 1),
                           "status_bits": res["status"], "nonfinite_evals": res["nonfinite"]},
                "roofline": roofline, "cpu_baseline": cpu, "e2e": e2e, "clocks": clk,
                "gpu_launches": gpu_launches}
        line.update(extra)
        print(json.dumps(line), flush=True)
    if world > 1:
        dist.barrier()
        dist.destroy_process_group()
    return 0


if __name__ == "__main__":
    sys.exit(main())
