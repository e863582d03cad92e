"""GPU parity of the likelihood stages against the FP64 CPU oracle, through the
C ABI (rows A5, A6, A8-A13).

Tolerances: FP64 path 1e-9 relative on log L (the benchmark spec); FP32 path 1e-4
absolute on log L where the arithmetic allows it (the design notes derive the
FP32 bound c * eps32 * sum |terms| for the high-S/N 39-d problem); BF16 path
judged against the bound derived from bf16 rounding of weights/activations."""

import numpy as np
import pytest
import torch

from gpu_helpers import cuda_problem, free_theta, oracle_for, random_cube
from oracle.priors import cube_to_theta, free_indices

pytestmark = pytest.mark.gpu


def _t(a):
    return torch.tensor(np.ascontiguousarray(a), dtype=torch.float64, device="cuda")


@pytest.mark.parametrize("name", ["shear_tiny", "shear39"])
def test_prior_transform(name):
    inp, orc = oracle_for(name)
    p = cuda_problem(name, "fp64", max_batch=64)
    cube = random_cube(53, p.d, 1, 1e-6, 1 - 1e-6)
    got = p.prior_transform(_t(cube)).cpu().numpy()
    ref = cube_to_theta(inp["priors"], cube)[:, free_indices(inp["priors"])]
    assert np.allclose(got, ref, rtol=1e-14, atol=1e-15)


@pytest.mark.parametrize("name,B", [("shear_tiny", 37), ("shear5", 20), ("shear39", 5)])
def test_model_vector_fp64(name, B):
    inp, orc = oracle_for(name)
    p = cuda_problem(name, "fp64", max_batch=64)
    th = free_theta(inp, random_cube(B, p.d, 2))
    got = p.model(_t(th)).cpu().numpy()
    for b in range(B):
        ref = orc.model(_full(inp, th[b]))
        scale = np.max(np.abs(ref))
        assert np.max(np.abs(got[b] - ref)) < 1e-11 * scale, (b, np.max(np.abs(got[b] - ref)) / scale)


def _full(inp, th):
    full = np.array([p[1] for p in inp["priors"]], float)
    full[free_indices(inp["priors"])] = th
    return full


@pytest.mark.parametrize("name,B", [("shear_tiny", 37), ("shear5", 20), ("shear39", 6), ("shear37", 3)])
def test_loglike_fp64_parity(name, B):
    inp, orc = oracle_for(name)
    p = cuda_problem(name, "fp64", max_batch=64)
    th = free_theta(inp, random_cube(B, p.d, 3))
    got = p.loglike(_t(th)).cpu().numpy()
    ref = np.array([orc.loglike(t) for t in th])
    rel = np.abs(got - ref) / np.abs(ref)
    assert np.all(rel < 1e-9), rel.max()


def test_loglike_fp64_near_fiducial_and_own_mock():
    """Near the peak (where chi^2 ~ D and cancellation in d - m is largest) and
    with the library building its own mock data from its FP64 model vector."""
    name = "shear39"
    inp, orc = oracle_for(name)
    p = cuda_problem(name, "fp64", max_batch=8, own_mock=True)
    assert np.max(np.abs(p.data - orc.data)) < 1e-11 * np.max(np.abs(orc.data))
    assert np.allclose(p.cov, orc.cov, rtol=1e-11, atol=0)
    fid = np.asarray(inp["fiducial"])[free_indices(inp["priors"])]
    th = fid[None, :] * (1 + 1e-3 * np.random.default_rng(4).standard_normal((4, fid.size))) + 1e-4
    got = p.loglike(_t(th)).cpu().numpy()
    ref = np.array([orc.loglike(t) for t in th])
    assert np.all(np.abs(got - ref) / np.abs(ref) < 1e-9)


@pytest.mark.parametrize("name", ["shear_tiny", "shear39"])
def test_emulator_fp64_parity(name):
    inp, orc = oracle_for(name)
    p = cuda_problem(name, "fp64", max_batch=64)
    th = free_theta(inp, random_cube(9, p.d, 5))
    got = p.emulator(_t(th)).cpu().numpy()
    for b in range(len(th)):
        ref = orc.emulator(_full(inp, th[b])).reshape(-1)
        assert np.max(np.abs(got[b] - ref)) < 1e-12


def test_batch_edge_cases():
    from paper_2509_13307_gb300._lib import GpunsError
    inp, orc = oracle_for("shear_tiny")
    p = cuda_problem("shear_tiny", "fp64", max_batch=16)
    th = free_theta(inp, random_cube(17, p.d, 6))
    with pytest.raises(GpunsError):
        p.loglike(_t(th))                    # B > max_batch
    out = p.loglike(_t(th[:0]))              # B = 0 is a no-op
    assert out.numel() == 0
    one = p.loglike(_t(th[:1])).cpu().numpy()
    assert abs(one[0] / orc.loglike(th[0]) - 1) < 1e-9


def test_bad_covariance_is_rejected():
    from paper_2509_13307_gb300 import Problem
    from paper_2509_13307_gb300._lib import GpunsError
    inp, orc = oracle_for("shear_tiny")
    cov = orc.cov.copy()
    cov[0, 0] = -1.0
    with pytest.raises(GpunsError):
        Problem(inp, "fp64", max_batch=4, data=orc.data, cov=cov)
