"""Row A14: the hand-written adjoint d log L / d theta against the oracle's
complex-step gradient (exact to round-off), central differences of the GPU
log L, and the torch.autograd wrapper.  FP64: 1e-9 relative to the gradient's
largest component; FP32 / BF16 errors are measured against the FP64 oracle
and bounded by the design notes' derivation."""

import numpy as np
import pytest
import torch

from gpu_helpers import cuda_problem, free_theta, oracle_for, random_cube

pytestmark = pytest.mark.gpu


def _t(a):
    return torch.tensor(np.ascontiguousarray(a), dtype=torch.float64, device="cuda")


@pytest.mark.parametrize("name,B", [("shear_tiny", 5), ("shear5", 3), ("shear39", 2)])
def test_adjoint_fp64_matches_complex_step(name, B):
    inp, orc = oracle_for(name)
    p = cuda_problem(name, "fp64", max_batch=16)
    th = free_theta(inp, random_cube(B, p.d, 21, 0.1, 0.9))
    logL, g = p.loglike_grad(_t(th))
    logL, g = logL.cpu().numpy(), g.cpu().numpy()
    ll = p.loglike(_t(th)).cpu().numpy()
    assert np.allclose(logL, ll, rtol=1e-12, atol=0)
    for b in range(B):
        ref = orc.grad_complex_step(th[b])
        scale = np.max(np.abs(ref))
        err = np.max(np.abs(g[b] - ref)) / scale
        assert err < 1e-9, (b, err, np.argmax(np.abs(g[b] - ref)))


def test_adjoint_fp64_central_differences_of_gpu_loglike():
    inp, orc = oracle_for("shear_tiny")
    p = cuda_problem("shear_tiny", "fp64", max_batch=64)
    th = free_theta(inp, random_cube(1, p.d, 22, 0.1, 0.9))[0]
    _, g = p.loglike_grad(_t(th[None, :]))
    g = g.cpu().numpy()[0]
    rows = []
    for i in range(p.d):
        hstep = 1e-5 * max(abs(th[i]), 1e-2)
        tp, tm = th.copy(), th.copy()
        tp[i] += hstep
        tm[i] -= hstep
        rows += [tp, tm]
    vals = p.loglike(_t(np.array(rows))).cpu().numpy()
    for i in range(p.d):
        hstep = 1e-5 * max(abs(th[i]), 1e-2)
        fd = (vals[2 * i] - vals[2 * i + 1]) / (2 * hstep)
        assert abs(fd - g[i]) <= 1e-5 * max(abs(g[i]), 1.0), (i, fd, g[i])


def _grad_bf16_weights(orc, th):
    """Complex-step gradient of the oracle whose emulator weights (layers >= 1)
    are rounded to bf16, activations exact: the model the split-bf16 adjoint
    differentiates."""
    save = orc.emulator
    orc.emulator = lambda t, _s=save: _s(t, bf16_weights=True)
    try:
        return orc.grad_complex_step(th)
    finally:
        orc.emulator = save


@pytest.mark.parametrize("prec,tol", [("fp32", 1e-4), ("bf16", 1e-4)])
def test_adjoint_low_precision_error_is_bounded(prec, tol):
    """FP32: against the FP64 oracle's complex-step gradient.  BF16: the
    emulator weights are bf16 (the BF16 model), the activations and gradients
    FP32-accurate split-bf16 pairs, so the gradient is checked against the
    complex-step gradient of the oracle with bf16 weights, to the FP32
    tolerance; its distance from the FP64 model's gradient (the bf16 weights'
    effect) is printed."""
    inp, orc = oracle_for("shear39")
    p = cuda_problem("shear39", prec, max_batch=16)
    fid = np.asarray(inp["fiducial"])
    th = fid[None, :] * (1 + 2e-3 * np.random.default_rng(7).standard_normal((2, fid.size))) + 1e-3
    _, g = p.loglike_grad(_t(th))
    g = g.cpu().numpy()
    for b in range(len(th)):
        ref = orc.grad_complex_step(th[b]) if prec == "fp32" else _grad_bf16_weights(orc, th[b])
        err = np.max(np.abs(g[b] - ref)) / np.max(np.abs(ref))
        if prec == "bf16":
            r64 = orc.grad_complex_step(th[b])
            print(f"bf16 gradient vs the FP64 model's: {np.max(np.abs(g[b] - r64)) / np.max(np.abs(r64)):.3e}")
        print(f"{prec} gradient max error / max |grad| = {err:.3e}")
        assert err < tol


def test_autograd_function():
    from paper_2509_13307_gb300 import loglike_autograd
    inp, orc = oracle_for("shear_tiny")
    p = cuda_problem("shear_tiny", "fp64", max_batch=16)
    th = _t(free_theta(inp, random_cube(3, p.d, 23, 0.1, 0.9))).requires_grad_(True)
    out = loglike_autograd(p, th)
    w = torch.tensor([1.0, -2.0, 0.5], dtype=torch.float64, device="cuda")
    (out * w).sum().backward()
    _, g = p.loglike_grad(th.detach())
    assert torch.allclose(th.grad, w[:, None] * g, rtol=1e-13, atol=0)


def test_adjoint_bf16_batch_on_tensor_cores():
    """BF16 problems take the emulator forward and backward on the tensor
    cores (split-bf16 activations and gradients, exact bf16 weights).  At 300
    rows (three 128-row tiles and a ragged tail), random prior points: the
    gradient of three sampled rows against the complex-step gradient of the
    oracle with bf16 emulator weights, to the FP32 tolerance of the test above,
    every row finite."""
    inp, orc = oracle_for("shear39")
    p = cuda_problem("shear39", "bf16", max_batch=300)
    th = free_theta(inp, random_cube(300, p.d, 24, 0.1, 0.9))
    logL, g = p.loglike_grad(_t(th))
    logL, g = logL.cpu().numpy(), g.cpu().numpy()
    assert np.all(np.isfinite(logL)) and np.all(np.isfinite(g))
    for b in (0, 129, 299):
        ref = _grad_bf16_weights(orc, th[b])
        err = np.max(np.abs(g[b] - ref)) / np.max(np.abs(ref))
        print(f"bf16 tensor-core adjoint row {b}: max error / max |grad| = {err:.3e}")
        assert err < 1e-4
