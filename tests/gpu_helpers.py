"""Shared set-up for the GPU parity tests: oracle and CUDA problems built from
the same seeded workload inputs (the oracle's mock data and covariance are
passed to the CUDA problem so that the comparison isolates the arithmetic)."""

import functools

import numpy as np

import workloads as w
from oracle.priors import cube_to_theta, free_indices
from oracle.shear import ShearOracle

CONFIGS = {"shear_tiny": w.shear_tiny, "shear5": w.shear5, "shear39": w.shear39,
           "shear37": w.shear37_lcdm, "shear39_interp": w.shear39_interp,
           "shear39_interp_linear": w.shear39_interp_linear}


@functools.lru_cache(maxsize=None)
def oracle_for(name):
    inp = w.make_shear_inputs(CONFIGS[name]())
    return inp, ShearOracle(inp)


def cuda_problem(name, precision, max_batch=64, own_mock=False, hidden_tile=0):
    from paper_2509_13307_gb300 import Problem
    inp, orc = oracle_for(name)
    if own_mock:
        return Problem(inp, precision, max_batch=max_batch, hidden_tile=hidden_tile)
    return Problem(inp, precision, max_batch=max_batch, data=orc.data, cov=orc.cov, hidden_tile=hidden_tile)


def random_cube(n, d, seed, lo=0.02, hi=0.98):
    return np.random.default_rng(seed).uniform(lo, hi, (n, d))


def free_theta(inp, cube):
    full = cube_to_theta(inp["priors"], cube)
    return np.ascontiguousarray(full[:, free_indices(inp["priors"])])
