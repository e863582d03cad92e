"""ns_evidence_noalloc: the evidence of a caller-held dead-point sequence with
no device allocation (for callers whose framework reserves the device memory
for its own pool, or whose loop must not call cudaMalloc / cudaFree).  It must
reproduce ns_evidence on the same run, on two calls in a row (the second call
reuses the library's static scratch array)."""

import ctypes as C

import numpy as np
import pytest
import torch

import workloads as w

pytestmark = pytest.mark.gpu


def test_noalloc_evidence_matches_ns_evidence():
    from paper_2509_13307_gb300 import Problem, NestedRun, _lib
    cfg = w.gauss_test(3, n_live=40, n_delete=4, seed=11)
    prob = Problem(w.make_gauss_inputs(cfg), "fp64", max_batch=40)
    run = NestedRun.from_config(prob, cfg.sampler)
    run.run()
    n_rep = 64
    ref = run.evidence(n_replays=n_rep)
    _xd, ld, nd = run.dead_points()
    _x, lg = run.live_points()
    n = cfg.sampler.n_live
    seq_L = np.concatenate([ld, np.sort(lg)])
    seq_n = np.concatenate([nd, n - np.arange(n)]).astype(np.int32)
    dL = torch.tensor(seq_L, dtype=torch.float64, device="cuda")
    dn = torch.tensor(seq_n, dtype=torch.int32, device="cuda")
    out = torch.full((3,), float("nan"), dtype=torch.float64, device="cuda")
    lib = _lib.load()
    stream = C.c_void_p(torch.cuda.current_stream().cuda_stream)
    for _ in range(2):
        out.fill_(float("nan"))
        rc = lib.ns_evidence_noalloc(C.c_void_p(dL.data_ptr()), C.c_void_p(dn.data_ptr()), len(seq_L),
                                     cfg.sampler.seed, n_rep, C.c_void_p(out.data_ptr()), stream)
        assert rc == 0, lib.ns_strerror(rc)
        logZ, err, logX = out.cpu().numpy()
        assert logZ == pytest.approx(ref["logZ"], rel=1e-11, abs=1e-11)
        assert err == pytest.approx(ref["logZ_err"], rel=1e-8)
        assert logX == pytest.approx(ref["logX"], rel=1e-12)
    # a live count below 1 gives NaN outputs rather than a silent number
    bad = dn.clone()
    bad[5] = 0
    rc = lib.ns_evidence_noalloc(C.c_void_p(dL.data_ptr()), C.c_void_p(bad.data_ptr()), len(seq_L),
                                 cfg.sampler.seed, n_rep, C.c_void_p(out.data_ptr()), stream)
    assert rc == 0 and np.all(np.isnan(out.cpu().numpy()))
    # sizes beyond the static array are rejected
    assert lib.ns_evidence_noalloc(C.c_void_p(dL.data_ptr()), C.c_void_p(dn.data_ptr()), len(seq_L),
                                   cfg.sampler.seed, 4097, C.c_void_p(out.data_ptr()), stream) == -1
