"""BF16 parity at the batch sizes the nested-sampling rounds run (rows A6-A13).

The 39-d shear likelihood in BF16 (tcgen05 emulator, FP32 projection and
chi^2) is compared element by element with the FP64 oracle's bf16-aware
emulator (weights of layers >= 1 and hidden activations rounded to bf16,
FP64 arithmetic) at 500 and 1000 rows: sampled rows in every 128-row M tile
of the hidden layers and every 256-row tile of the output layer, and their
ragged tails.  Each hidden-layer N-tile width (16, 32, 64, 128) is forced in
turn, and the widths must give bit-identical outputs on every row (the MMA
accumulation order per element does not depend on the width).

Each stage is held to its own tolerance: the emulator table against the
bf16-aware oracle within 2e-4 dex (the FP32 accumulation order flips the bf16
rounding of an activation now and then, see test_gpu_precision); log L
against the oracle's projection and chi^2 of the GPU's own emulator table
(ns_emulator_batch returns exactly the FP32 table the likelihood uses),
within the FP32 model-vector bound eps_m sum_a |y_a| (|L^-1| |m|)_a with
eps_m = 2e-6.  (At random prior points chi^2 reaches ~1e6, so the emulator's
1e-4 dex differences alone move log L by more than the FP32 bound; checking
the stages separately keeps both bounds tight.)"""

import functools

import numpy as np
import pytest
import torch

from gpu_helpers import cuda_problem, free_theta, oracle_for, random_cube
from oracle.priors import cube_to_theta, free_indices

pytestmark = pytest.mark.gpu

WIDTHS = (16, 32, 64, 128)
ROWS = {500: (0, 127, 128, 255, 256, 383, 384, 499),
        1000: (0, 127, 128, 255, 256, 383, 384, 511, 512, 767, 768, 895, 896, 999)}


def _t(a):
    return torch.tensor(np.ascontiguousarray(a), dtype=torch.float64, device="cuda")


def _full(inp, th):
    full = np.array([p[1] for p in inp["priors"]], float)
    full[free_indices(inp["priors"])] = th
    return full


@functools.lru_cache(maxsize=None)
def _linv(name):
    _, orc = oracle_for(name)
    return np.linalg.inv(orc.L)


def _ref_and_bound(name, full, table, eps_m=2e-6):
    """Oracle log L with the emulator table `table` (the GPU's), and the FP32
    bound of the stages after the emulator."""
    _, orc = oracle_for(name)
    save = orc.emulator
    orc.emulator = lambda t, _tab=np.asarray(table, float): _tab.reshape(orc.n_z_emu, orc.n_k)
    try:
        ref = orc.loglike_full(full)
        m = orc.model(full)
    finally:
        orc.emulator = save
    y = orc.forward_subst(orc.data - m)
    bound = eps_m * np.sum(np.abs(y) * (np.abs(_linv(name)) @ np.abs(m)))
    return ref, bound


@functools.lru_cache(maxsize=None)
def _outputs(name, B, width):
    inp, _ = oracle_for(name)
    p = cuda_problem(name, "bf16", max_batch=B, hidden_tile=width)
    tiles, _ = p.tiles()
    th = free_theta(inp, random_cube(B, p.d, 71 + B))
    thd = _t(th)
    emu = p.emulator(thd).cpu().numpy()
    logL = p.loglike(thd).cpu().numpy()
    bits = p.device_status()
    p.close()
    return th, emu, logL, tiles, bits


@pytest.mark.parametrize("B", [500, 1000])
@pytest.mark.parametrize("width", WIDTHS)
def test_bf16_emulator_and_loglike_against_oracle(B, width):
    name = "shear39"
    inp, orc = oracle_for(name)
    th, emu, logL, tiles, bits = _outputs(name, B, width)
    assert bits == 0
    assert all(t == width for t in tiles[1:-1]), tiles
    assert np.all(np.isfinite(logL)) and np.all(np.isfinite(emu))
    worst_e, worst_r = 0.0, 0.0
    for b in ROWS[B]:
        full = _full(inp, th[b])
        ref_e = orc.emulator(full, bf16=True).reshape(-1)
        err_e = np.max(np.abs(emu[b] - ref_e))
        assert err_e < 2e-4, (b, err_e)
        ref, bound = _ref_and_bound(name, full, emu[b])
        err = abs(logL[b] - ref)
        assert err <= bound, (b, err, bound)
        worst_e, worst_r = max(worst_e, err_e), max(worst_r, err / bound)
    print(f"B={B} tile={width}: emulator max |d log10 P| {worst_e:.2e}, log L max error / bound {worst_r:.3f}")


@pytest.mark.parametrize("B", [500, 1000])
def test_hidden_tile_widths_are_bit_identical(B):
    outs = [_outputs("shear39", B, w_) for w_ in WIDTHS]
    for o in outs[1:]:
        assert np.array_equal(o[1], outs[0][1])
        assert np.array_equal(o[2], outs[0][2])


@pytest.mark.parametrize("B", [1, 65, 500, 1000])
def test_fused_emulator_stack(B):
    """The fused emulator stack (hidden_tile = -1): the input layer and the
    three hidden layers as one clustered kernel (8 CTAs per 64-row tile,
    activations kept in shared memory, features as the MMA's M).  Against the
    per-layer path (forced 16-wide tiles, rows as the MMA's M) and the
    bf16-aware oracle: both paths accumulate each product in the same k order
    (measured: bit-identical, printed); every row stays within the emulator
    tolerance of the oracle, including the ragged last tile, and log L
    follows."""
    name = "shear39"
    inp, orc = oracle_for(name)
    pf = cuda_problem(name, "bf16", max_batch=max(B, 64), hidden_tile=-1)
    assert pf.fused_cluster() == 8
    tiles, _ = pf.tiles()
    th = free_theta(inp, random_cube(B, pf.d, 91 + B))
    thd = _t(th)
    ef = pf.emulator(thd).cpu().numpy()
    lf = pf.loglike(thd).cpu().numpy()
    assert pf.device_status() == 0
    pl = cuda_problem(name, "bf16", max_batch=max(B, 64), hidden_tile=16)
    el = pl.emulator(thd).cpu().numpy()
    ll = pl.loglike(thd).cpu().numpy()
    same = np.mean(ef == el)
    print(f"B={B}: fused vs per-layer emulator: {same:.4f} of values identical, max |d| {np.max(np.abs(ef - el)):.2e}")
    assert np.max(np.abs(ef - el)) < 4e-4
    assert np.all(np.isfinite(lf))
    rows = sorted({0, B // 2, B - 1, min(B - 1, 63), min(B - 1, 64)})
    for b in rows:
        full = _full(inp, th[b])
        assert np.max(np.abs(ef[b] - orc.emulator(full, bf16=True).reshape(-1))) < 2e-4, b
        ref, bound = _ref_and_bound(name, full, ef[b])
        assert abs(lf[b] - ref) <= bound, (b, abs(lf[b] - ref), bound)
    pf.close()
    pl.close()


def test_invalid_hidden_tile_is_rejected():
    from paper_2509_13307_gb300._lib import GpunsError
    for bad in (48, 256, -2):
        with pytest.raises(GpunsError):
            cuda_problem("shear_tiny", "bf16", max_batch=8, hidden_tile=bad)
    # the fused stack needs hidden widths of 512 or 1024 (shear_tiny: 192)
    with pytest.raises(GpunsError):
        cuda_problem("shear_tiny", "bf16", max_batch=8, hidden_tile=-1)
    assert cuda_problem("shear39", "bf16", max_batch=8).fused_cluster() == 0


def test_autotuned_problem_matches_forced_widths():
    inp, _ = oracle_for("shear39")
    th, emu, logL, _, _ = _outputs("shear39", 500, 32)
    p = cuda_problem("shear39", "bf16", max_batch=500)
    assert np.array_equal(p.loglike(_t(th)).cpu().numpy(), logL)
    p.close()


@pytest.mark.parametrize("name", ["shear39_interp", "shear39_interp_linear"])
def test_bf16_interpolated_emulator_against_oracle(name):
    """The coarse-z emulator (10 z nodes, interpolated to the 50-node table,
    App. B) in BF16 at 500 rows."""
    inp, orc = oracle_for(name)
    B = 500
    p = cuda_problem(name, "bf16", max_batch=B)
    th = free_theta(inp, random_cube(B, p.d, 83))
    thd = _t(th)
    emu = p.emulator(thd).cpu().numpy()
    logL = p.loglike(thd).cpu().numpy()
    assert np.all(np.isfinite(logL))
    for b in ROWS[B]:
        full = _full(inp, th[b])
        assert np.max(np.abs(emu[b] - orc.emulator(full, bf16=True).reshape(-1))) < 2e-4
        # the coarse-to-fine z step adds a 4-tap FP32 sum to the table: eps_m 4e-6
        ref, bound = _ref_and_bound(name, full, emu[b], eps_m=4e-6)
        assert abs(logL[b] - ref) <= bound, (b, abs(logL[b] - ref), bound)
    p.close()


@pytest.mark.parametrize("prec", ["bf16", "fp32"])
def test_sampler_prior_transform_at_the_cube_edges(prec):
    """Reduced-precision problems take the Gaussian quantile in FP32 (the
    sampler's proposals and ns_prior_transform share it).  Coordinates within
    2^-25 of 1 round to 1.0f, where the FP32 quantile is infinite; the
    transform works on min(c, 1 - c) instead, so every coordinate of the open
    cube maps to a finite parameter close to the FP64 quantile, and the
    likelihood there is finite."""
    name = "shear39"
    inp, orc = oracle_for(name)
    p = cuda_problem(name, prec, max_batch=16)
    pri = inp["priors"]
    gauss = [f for f, i in enumerate(free_indices(pri)) if pri[i][0] == "N"]
    edges = [1e-300, 1e-40, 1e-12, 1e-9, 0.3, 0.5, 1 - 1e-9, 1 - 2.0 ** -30, 1 - 2.0 ** -53]
    cube = np.full((len(edges), p.d), 0.5)
    for r, c in enumerate(edges):
        cube[r, gauss] = c
    got = p.prior_transform(_t(cube)).cpu().numpy()
    ref = cube_to_theta(pri, cube)[:, free_indices(pri)]
    assert np.all(np.isfinite(got))
    # FP32 quantile: relative error ~1e-6 of |z| (FP64 below 1e-37)
    sd = np.array([pri[i][2] if pri[i][0] == "N" else 1.0 for i in free_indices(pri)])
    assert np.all(np.abs(got - ref) <= 2e-6 * (np.abs(ref) + sd)), np.max(np.abs(got - ref))
    logL = p.loglike(_t(got)).cpu().numpy()
    assert np.all(np.isfinite(logL)), logL
    p.close()


def test_bf16_run_has_no_nonfinite_likelihoods():
    """A BF16 run of the 39-d problem: every proposal's log L is finite."""
    import workloads as w
    from paper_2509_13307_gb300 import NestedRun
    sc = w.shear39().sampler
    p = cuda_problem("shear39", "bf16", max_batch=sc.n_live)
    run = NestedRun.from_config(p, sc)
    st = run.step(6)
    assert st.status_bits == 0 and st.nonfinite == 0, st
    run.close()
    p.close()
