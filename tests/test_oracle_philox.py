"""Pins of the oracle's Philox4x32-10 against published known-answer vectors,
and of the uniform / normal conversions against their distributions."""

import os

import numpy as np
import pytest
from scipy import stats

from oracle import philox

GOLD = os.path.join(os.path.dirname(__file__), "golden", "philox4x32_10_kat.txt")


def _kat():
    rows = []
    for line in open(GOLD):
        if line.startswith("#") or not line.strip():
            continue
        v = [int(t, 16) for t in line.split()]
        rows.append((v[:6], v[6:]))
    return rows


@pytest.mark.parametrize("row", _kat())
def test_known_answers(row):
    inp, out = row
    got = [int(x) for x in philox.philox4x32_10(*inp)]
    assert got == out
    assert list(philox.philox4x32_10_int(*inp)) == out


def test_vector_and_scalar_agree():
    rng = np.random.default_rng(0)
    for _ in range(50):
        a = [int(x) for x in rng.integers(0, 2 ** 32, 6)]
        assert [int(x) for x in philox.philox4x32_10(*a)] == list(philox.philox4x32_10_int(*a))
    seed = 0x1234567890ABCDEF
    for j in range(5):
        assert float(philox.uniform(seed, 5, j, 7, 9, 11)) == philox.uniform_scalar(seed, 5, j, 7, 9, 11)


def test_uniforms_open_interval_and_moments():
    idx = np.arange(200_000, dtype=np.uint64)
    ua, ub = philox.uniforms(42, philox.PURPOSE_ERR, 0, 1, idx, 0)
    u = np.concatenate([ua, ub])
    assert u.min() > 0.0 and u.max() < 1.0
    assert abs(u.mean() - 0.5) < 5 * np.sqrt(1 / 12 / u.size)
    assert stats.kstest(u, "uniform").pvalue > 1e-3


def test_normals_distribution():
    z = np.concatenate([philox.normals(7, philox.PURPOSE_DIR, it, c, 0, 40)
                        for it in range(50) for c in range(50)])
    assert abs(z.mean()) < 5 / np.sqrt(z.size)
    assert abs(z.var() - 1.0) < 5 * np.sqrt(2.0 / z.size)
    assert stats.kstest(z, "norm").pvalue > 1e-3


def test_extreme_uniform_bits():
    # all-ones and all-zeros 52-bit mantissas stay strictly inside (0, 1)
    lo = philox._u01(np.uint64(0), np.uint64(0))
    hi = philox._u01(np.uint64(0xFFFFFFFF), np.uint64(0xFFFFFFFF))
    assert lo == 2.0 ** -53 and hi == 1.0 - 2.0 ** -53
