"""Seeded synthetic workloads shared by the CUDA path and the CPU oracle.

This package holds configuration (sizes, grid extents, prior boxes, fiducial
values) and seeded random draws (emulator weights, noise realisations,
covariance ingredients).  It deliberately contains none of the method's
arithmetic: no distances, windows, projections, likelihoods or sampler steps.
Both sides consume its outputs and compute everything else themselves.
"""

from .configs import (  # noqa: F401
    ShearConfig, GaussConfig, CMBConfig, SamplerConfig,
    shear5, shear39, shear37_lcdm, shear33, shear_tiny, gauss_test, cmb6, cmb_tiny,
    shear39_interp, shear37_interp, shear39_interp_linear, uneven_runs,
    SHEAR_BASE_NAMES, shear_param_names,
)
from .synth import make_shear_inputs, make_gauss_inputs, make_cmb_inputs, wishart_base  # noqa: F401
