"""Pins of the oracle's prior transform (Table 1: uniform U(a, b) and Gaussian
N(mu, sigma) priors, fixed parameters inserted) against values the
mathematics fixes, independent of the library routine the oracle calls:
textbook normal quantiles, the normal CDF written with math.erf (a round
trip), the moments of transformed uniform draws (mean mu, standard deviation
sigma, so a sigma-vs-sigma^2 or a mean/width swap fails), the uniform end
points, and the insertion of fixed parameters in parameter order."""

import math

import numpy as np
import pytest

import workloads as w
from oracle.priors import cube_to_theta, free_indices, theta_free_to_full

# Phi^-1 at a few probabilities (standard tables): Phi(1), Phi(-2), 0.975, 0.5.
KNOWN = [(0.8413447460685429, 1.0), (0.022750131948179195, -2.0), (0.975, 1.959963984540054), (0.5, 0.0),
         (0.9986501019683699, 3.0)]


def _phi(x):
    return 0.5 * (1.0 + math.erf(x / math.sqrt(2.0)))


@pytest.mark.parametrize("mu,sd", [(0.0, 0.01), (0.01, 0.02), (0.0, 1.0), (-3.0, 0.5)])
def test_gaussian_prior_known_quantiles(mu, sd):
    pri = [("N", mu, sd)]
    for c, z in KNOWN:
        th = cube_to_theta(pri, np.array([c]))
        assert th[0] == pytest.approx(mu + sd * z, rel=1e-12, abs=1e-14)


def test_gaussian_prior_round_trip_through_erf():
    pri = [("N", 0.01, 0.02)]
    for x in np.linspace(-6.0, 6.0, 49):
        c = _phi(x)
        if not 0.0 < c < 1.0:
            continue
        th = cube_to_theta(pri, np.array([c]))[0]
        z = (th - 0.01) / 0.02
        # Phi(z) reproduces c (relative error of the erf evaluation ~1e-15,
        # amplified by 1/phi(z) in z; compare in probability space)
        assert _phi(z) == pytest.approx(c, rel=1e-12, abs=1e-16)


def test_gaussian_prior_moments_of_transformed_uniforms():
    """Transformed uniform draws have mean mu and standard deviation sigma:
    the second argument of a Gaussian prior is a standard deviation (the
    reading of Table 1's m ~ N(0.01, 0.02)), not a variance."""
    rng = np.random.default_rng(0)
    c = rng.uniform(0.0, 1.0, (400000, 1))
    for mu, sd in [(0.01, 0.02), (0.0, 0.01)]:
        th = cube_to_theta([("N", mu, sd)], c)[:, 0]
        n = th.size
        assert abs(th.mean() - mu) < 5 * sd / math.sqrt(n)
        assert abs(th.std(ddof=1) / sd - 1.0) < 5 / math.sqrt(2 * n)


def test_uniform_prior_endpoints_and_midpoint():
    pri = [("U", -1.5, -0.5), ("U", 0.05, 0.255)]
    cube = np.array([[0.0, 1.0], [1.0, 0.0], [0.5, 0.5], [0.25, 0.75]])
    th = cube_to_theta(pri, cube)
    assert np.allclose(th[0], [-1.5, 0.255], rtol=0, atol=1e-15)
    assert np.allclose(th[1], [-0.5, 0.05], rtol=0, atol=1e-15)
    assert np.allclose(th[2], [-1.0, 0.1525], rtol=0, atol=1e-15)
    assert np.allclose(th[3], [-1.25, 0.05 + 0.75 * 0.205], rtol=0, atol=1e-15)


def test_fixed_parameters_take_no_cube_coordinate():
    pri = [("U", 0.0, 2.0), ("F", -1.0, 0.0), ("N", 1.0, 0.5), ("F", 0.0, 0.0), ("U", 10.0, 20.0)]
    assert free_indices(pri) == [0, 2, 4]
    cube = np.array([[0.25, 0.975, 0.5]])
    th = cube_to_theta(pri, cube)[0]
    assert np.allclose(th, [0.5, -1.0, 1.0 + 0.5 * 1.959963984540054, 0.0, 15.0], rtol=1e-13, atol=1e-15)
    full = theta_free_to_full(pri, np.array([0.5, 1.9, 15.0]))
    assert np.array_equal(full, [0.5, -1.0, 1.9, 0.0, 15.0])


def test_table1_priors_of_the_39_parameter_workload():
    """The 39-d layout's nuisance priors (Table 1): D_z ~ N(0, 0.01^2),
    m ~ N(0.01, 0.02), template amplitudes ~ N(0, 1); w0, wa uniform; the 37-d
    model fixes w0 = -1, wa = 0."""
    cfg = w.shear39()
    pri = cfg.priors()
    names = cfg.param_names
    z1 = 0.8413447460685429   # Phi(1)
    cube = np.full((1, len(free_indices(pri))), 0.5)
    free_names = [names[i] for i in free_indices(pri)]
    for nm in ("Dz_0", "m_3", "b_0", "w0", "wa"):
        cube[0, free_names.index(nm)] = z1
    th = cube_to_theta(pri, cube)[0]
    assert th[names.index("Dz_0")] == pytest.approx(0.01, rel=1e-12)
    assert th[names.index("m_3")] == pytest.approx(0.03, rel=1e-12)
    assert th[names.index("b_0")] == pytest.approx(1.0, rel=1e-12)
    assert th[names.index("w0")] == pytest.approx(-1.5 + z1, rel=1e-14)
    assert th[names.index("m_0")] == pytest.approx(0.01, rel=1e-14)
    lc = w.shear37_lcdm()
    pl = lc.priors()
    assert pl[lc.param_names.index("w0")] == ("F", -1.0, 0.0)
    assert pl[lc.param_names.index("wa")] == ("F", 0.0, 0.0)
    assert len(free_indices(pl)) == 37 and len(free_indices(pri)) == 39
