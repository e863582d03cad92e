"""Reduced-precision likelihood paths against the FP64 oracle.

BF16 emulator: compared with the oracle's bf16-aware emulator (weights of
layers >= 1 and every hidden activation rounded to bfloat16, arithmetic FP64),
i.e. the model the tcgen05 path computes up to FP32 accumulation order.  The
accumulation-order differences (~1e-6 relative) flip the bf16 rounding of an
activation now and then; one flip moves that unit by 2^-8 and four stacked
1024-wide layers spread it: measured 1.2e-4 dex on the 39-d emulator (3e-4
against the FP64 emulator); the bound is 2e-4.

FP32 log L: a model vector with relative error eps_m shifts chi^2 by
2 y . L^-1 dm, so |d log L| <= eps_m sum_a |y_a| (|L^-1| |m|)_a with
y = L^-1 (d - m).  The FP32 stages give eps_m ~ 1e-6 (1024-term FP32
contractions in the emulator, 16-tap lookups, 1024-node Limber sums); the test
uses eps_m = 2e-6 (measured errors reach 0.2 of that bound).  BF16 log L is
checked against the oracle fed the GPU's own BF16 emulator table (the
emulator itself is checked against the bf16-aware oracle above): the stages
after the emulator are FP32 and obey the same bound.  (The bf16 rounding flips
of the emulator move log L far from the fiducial by more than this bound, so
the two stages are checked separately.)"""

import numpy as np
import pytest
import torch

from gpu_helpers import cuda_problem, free_theta, oracle_for, random_cube
from oracle.priors import free_indices

pytestmark = pytest.mark.gpu


def _t(a):
    return torch.tensor(np.ascontiguousarray(a), dtype=torch.float64, device="cuda")


def _full(inp, th):
    full = np.array([p[1] for p in inp["priors"]], float)
    full[free_indices(inp["priors"])] = th
    return full


def _fp32_bound(orc, full, eps_m=2e-6):
    m = orc.model(full)
    y = orc.forward_subst(orc.data - m)
    Linv = np.linalg.inv(orc.L)
    return eps_m * np.sum(np.abs(y) * (np.abs(Linv) @ np.abs(m)))


@pytest.mark.parametrize("name", ["shear_tiny", "shear39"])
def test_emulator_bf16_against_bf16_aware_oracle(name):
    inp, orc = oracle_for(name)
    p = cuda_problem(name, "bf16", max_batch=64)
    th = free_theta(inp, random_cube(37 if name == "shear_tiny" else 6, p.d, 31))
    got = p.emulator(_t(th)).cpu().numpy()
    worst_plain = 0.0
    for b in range(len(th)):
        full = _full(inp, th[b])
        ref = orc.emulator(full, bf16=True).reshape(-1)
        err = np.max(np.abs(got[b] - ref))
        worst_plain = max(worst_plain, np.max(np.abs(got[b] - orc.emulator(full).reshape(-1))))
        assert err < 2e-4, (b, err)
    print(f"bf16 emulator vs FP64 emulator: max |d log10 P| = {worst_plain:.2e}")


@pytest.mark.parametrize("name,prec", [("shear5", "fp32"), ("shear39", "fp32"), ("shear_tiny", "fp32"),
                                       ("shear39", "bf16"), ("shear39", "bf16_f64chi2")])
def test_loglike_reduced_precision_bound(name, prec):
    inp, orc = oracle_for(name)
    p = cuda_problem(name, prec, max_batch=64)
    fid = np.asarray(inp["fiducial"])[free_indices(inp["priors"])]
    rng = np.random.default_rng(41)
    near = fid[None, :] * (1 + 1e-3 * rng.standard_normal((3, fid.size))) + 1e-4
    far = free_theta(inp, random_cube(3, p.d, 42))
    th = np.vstack([near, far])
    got = p.loglike(_t(th)).cpu().numpy()
    tab = p.emulator(_t(th)).cpu().numpy() if prec.startswith("bf16") else None
    for b in range(len(th)):
        full = _full(inp, th[b])
        if prec.startswith("bf16"):
            # the oracle's projection and chi^2 of the GPU's own emulator table
            # (checked against the bf16-aware oracle emulator above): the
            # remaining error is the FP32 stages'
            save = orc.emulator
            orc.emulator = lambda t, _tab=tab[b]: _tab.reshape(orc.n_z_emu, orc.n_k)
            try:
                ref = orc.loglike_full(full)
                bound = _fp32_bound(orc, full)
            finally:
                orc.emulator = save
        else:
            ref = orc.loglike_full(full)
            bound = _fp32_bound(orc, full)
        err = abs(got[b] - ref)
        print(f"{name} {prec} row {b}: |dlogL| = {err:.3e}, bound {bound:.3e}, ratio {err / bound:.3f}")
        assert err <= bound


def test_tile_autotuner_choice_is_valid_and_results_identical():
    """The hidden-layer tile autotuner picks one of the supported widths and
    reports the time it measured; the likelihood stays deterministic."""
    import torch
    from gpu_helpers import cuda_problem, free_theta, oracle_for, random_cube
    inp, _ = oracle_for("shear_tiny")
    p = cuda_problem("shear_tiny", "bf16", max_batch=64)
    tiles, ms = p.tiles()
    assert tiles[0] == 0 and all(t in (16, 32, 64, 128) for t in tiles[1:])
    assert all(m > 0 for m in ms[1:-1])
    th = torch.tensor(free_theta(inp, random_cube(40, p.d, 31)), device="cuda")
    a = p.loglike(th).cpu().numpy()
    b = p.loglike(th).cpu().numpy()
    assert (a == b).all()


@pytest.mark.parametrize("prec", ["fp32", "bf16"])
def test_whitened_loglike_full_batch(prec):
    """At the 39-d problem's round size (500 rows, more Limber CTAs than fit
    one wave) every row's log L is checked against the same FP32 model vector
    (ns_model_batch) whitened on the host in FP64: the residual d - m is
    formed in FP32 as the kernels do, and the remaining difference is bounded
    by the FP32 rounding of L^-1 and of the D-term dot products,
    |d log L| <= (D + 16) 2^-24 sum_a |y_a| (|L^-1| |r|)_a + 64 2^-24 chi^2.
    Three sampled rows are also held to the FP32 bound against the oracle."""
    name = "shear39"
    inp, orc = oracle_for(name)
    B = 500
    p = cuda_problem(name, prec, max_batch=B)
    th = free_theta(inp, random_cube(B, p.d, 61))
    thd = _t(th)
    got = p.loglike(thd).cpu().numpy()
    m = p.model(thd).cpu().numpy()
    r = (orc.data.astype(np.float32)[None, :] - m.astype(np.float32)).astype(np.float64)
    Linv = np.linalg.inv(orc.L)
    y = r @ Linv.T
    chi2 = np.sum(y * y, axis=1)
    ref = orc.c0 - 0.5 * chi2
    D = r.shape[1]
    bound = (D + 16) * 2.0 ** -24 * np.sum(np.abs(y) * (np.abs(r) @ np.abs(Linv).T), axis=1) + 64 * 2.0 ** -24 * chi2
    err = np.abs(got - ref)
    assert np.all(np.isfinite(got))
    assert np.all(err <= bound), (int(np.argmax(err / bound)), float(np.max(err / bound)))
    print(f"{prec} whitened log L, 500 rows: max |dlogL| {err.max():.3e}, max ratio to bound {np.max(err / bound):.3f}")
    if prec == "fp32":
        for b in (0, 137, 499):
            full = _full(inp, th[b])
            assert abs(got[b] - orc.loglike_full(full)) <= _fp32_bound(orc, full)
