"""CPU oracle for GPU nested slice sampling with emulator likelihoods
(arXiv:2509.13307).

TEST INFRASTRUCTURE ONLY.  This package is a plain, slow, FP64 NumPy
restatement of the method, written from the paper's equations and the
published algorithms it cites (Skilling 2006 nested sampling; Neal 2003 slice
sampling; Salmon et al. 2011 Philox).  Only the test-suite, the smoke check and
the benchmark's CPU-baseline leg may import it.  The CUDA library never calls
it, and it shares no code with the CUDA library: the only common module is the
seeded input generator package `workloads`, which holds no method arithmetic.

Modules
  philox    counter-based generator (pinned by published known-answer vectors)
  special   log-sum-exp and inverse normal CDF (scipy's ndtri)
  priors    cube -> physical prior transform (Table 1)
  shear     cosmic-shear likelihood (App. A: Eq. 3-6, the chi grid of App. A)
  cmb       CMB-like Gaussian likelihood with a dense covariance (Sec. 3.1)
  gauss     isotropic Gaussian test likelihood + closed-form evidence
  ns        nested slice sampler with batched deletion (Sec. 2.1-2.2)
  evidence  log Z / log X / H accumulation and the simulated-shrinkage error

Parity status: every function is pinned by tests under tests/ (closed forms,
invariants, brute force); exceptions are stated in the module docstrings.
"""
