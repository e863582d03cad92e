/*
 * gpuns.h -- C ABI of the GB300 (sm_103a) batched nested-slice-sampling library
 * with fused emulator -> chi(z) -> Limber -> chi^2 cosmic-shear likelihoods.
 *
 * Method: arXiv:2509.13307 (Lovick, Yallup, Piras, Spurio Mancini, Handley),
 *   Sec. 2.1  nested sampling: evidence Z = int L pi dtheta (Eq. 1), live points
 *             replaced under a hard likelihood constraint, slice sampling inside;
 *   Sec. 2.2  the k lowest live points deleted at once and k chains evolved in
 *             parallel;
 *   Eq. 2     Bayes factor B01 = Z0 / Z1 (formed by the caller from two runs);
 *   App. A    the cosmic-shear likelihood: Eq. 3 (C^eps = gg + gI + Ig + II),
 *             Eq. 4 (extended Limber with k = (ell + 1/2) / chi), Eq. 5 (shear
 *             window), Eq. 6 (NLA intrinsic-alignment window), multiplicative
 *             bias (1 + m_i)(1 + m_j), photo-z shifts n_i(z - D_z,i), a
 *             multivariate Gaussian likelihood, integrals on a chi grid uniform
 *             in scale factor from a = 1 to a_min;
 *   Table 1   uniform and Gaussian priors.
 *
 * Conventions for every entry point:
 *   - Return value: NS_OK (0) or a negative NS_E* code; ns_strerror() names it.
 *     Nothing throws or aborts across this boundary.
 *   - Pointers named *_dev are CUDA device pointers owned by the caller; every
 *     other pointer is host memory owned by the caller and only read during
 *     the call (the library copies what it keeps).
 *   - Matrices are row-major.  Floating-point arguments at the boundary are
 *     always FP64; the arithmetic precision inside is the problem's
 *     `precision`.
 *   - `stream` is a cudaStream_t passed as void* (NULL = legacy default
 *     stream).  Calls are asynchronous on that stream unless stated.
 *   - One problem or run must not be used from two streams at once: each owns
 *     scratch buffers that consecutive calls reuse.
 */
#ifndef GPUNS_H
#define GPUNS_H

#ifdef __cplusplus
extern "C" {
#endif

/* ---- status codes ------------------------------------------------------ */
#define NS_OK           0
#define NS_EINVAL      (-1)   /* invalid argument or descriptor */
#define NS_ECUDA       (-2)   /* a CUDA runtime / driver call failed */
#define NS_ENOMEM      (-3)   /* device or host allocation failed */
#define NS_ETIMEOUT    (-4)   /* a bounded device wait gave up (kernel watchdog) */
#define NS_ESLICE      (-5)   /* a slice step cap was reached (also a status bit) */
#define NS_ENONFINITE  (-6)   /* a likelihood evaluated to NaN/inf (also a status bit) */
#define NS_ENOTSUP     (-7)   /* combination not supported by the library */

/* ---- status bits accumulated by a run (ns_status.status_bits) ---------- */
#define NS_BIT_SLICE_CAP  1   /* stepping-out or shrinkage hit its cap */
#define NS_BIT_NONFINITE  2   /* some log L was NaN/inf (treated as outside) */
#define NS_BIT_TIMEOUT    4   /* a device wait hit its bound */

/* ---- enums -------------------------------------------------------------- */
enum ns_kind { NS_KIND_GAUSS = 0, NS_KIND_SHEAR = 1, NS_KIND_CMB = 2 };
/* Arithmetic of the likelihood.  FP64: every stage in double.  FP32: every
 * stage in float (emulator on CUDA cores), the constant and the final log L in
 * double.  BF16: emulator hidden/output GEMMs as tcgen05 BF16 x BF16 -> FP32
 * tensor-core MMAs, all other stages FP32.  BF16_F64CHI2: as BF16 but the
 * whitening solve and chi^2 in FP64. */
enum ns_precision { NS_PREC_FP64 = 0, NS_PREC_FP32 = 1, NS_PREC_BF16 = 2, NS_PREC_BF16_F64CHI2 = 3 };
enum ns_prior_kind { NS_PRIOR_UNIFORM = 0, NS_PRIOR_GAUSS = 1, NS_PRIOR_FIXED = 2 };
/* Hidden-layer activation: tanh, or CosmoPower's "sigmoid-linear"
 * f(x) = [g + (1 - g) sigmoid(beta x)] x with one (g, beta) per unit. */
enum ns_activation { NS_ACT_TANH = 0, NS_ACT_SIGMOID_LINEAR = 1 };
/* CMB chi^2 form (all exact in exact arithmetic; C = L L^T factorised in FP64 at
 * create):  FOLD: the linear output head is folded into the whitening,
 * W' = L^-1 diag(out_sigma) W_out and c' = L^-1 (d - out_mu - out_sigma b_out),
 * so y = c' - W' h and no per-evaluation solve remains.  LITERAL: the model
 * vector m is formed and y = L^-1 (d - m) per evaluation (FP64 only). */
enum ns_cmb_solve { NS_SOLVE_FOLD = 0, NS_SOLVE_LITERAL = 1 };

/* One prior per full parameter (Table 1).  UNIFORM: theta = a + (b - a) c;
 * GAUSS: theta = a + b Phi^-1(c) (mean a, sd b); FIXED: theta = a and the
 * parameter takes no cube coordinate.  c is the unit-cube coordinate. */
typedef struct { int kind; double a; double b; } ns_prior;

/* Emulator: an MLP of n_layers weight matrices, hidden layers act(W h + b),
 * output y = W h + b de-standardised as out_mu[o] + out_sigma * y[o].  The
 * input is x_j = (theta[inputs[j]] - in_center[j]) / in_scale[j].
 * For the shear kind the output is log10 P on the (z, k) table, z-major:
 * o = jz * n_k + ik. */
typedef struct {
    int n_layers;                 /* >= 2 */
    const int* dims;              /* n_layers + 1 sizes; dims[0] = number of inputs */
    const double* const* W;       /* W[l]: dims[l+1] x dims[l], row-major */
    const double* const* b;       /* b[l]: dims[l+1] */
    int activation;               /* ns_activation */
    const int* inputs;            /* dims[0] indices into the full parameter vector */
    const double* in_center;      /* dims[0] */
    const double* in_scale;       /* dims[0] */
    const double* out_mu;         /* dims[n_layers] */
    double out_sigma;             /* scalar output scale (used when out_sigma_vec is NULL) */
    const double* out_sigma_vec;  /* dims[n_layers] per-output scales, or NULL */
    const double* const* act_g;   /* SIGMOID_LINEAR: act_g[l], l < n_layers - 1: dims[l+1] values */
    const double* const* act_beta;/* SIGMOID_LINEAR: act_beta[l] likewise */
} ns_emulator_desc;

/* Cosmic-shear model (App. A).  Full parameter layout:
 *   0 omega_b, 1 omega_cdm, 2 h, 3 n_s, 4 ln10^10 A_s, 5 w0, 6 wa, 7 c_min,
 *   8 eta0, 9 A_IA, 10 eta_IA, 11.. D_z[n_bins], then m[n_bins], then
 *   template amplitudes b[n_tmpl]; n_params = 11 + 2 n_bins + n_tmpl.
 * Data vector element a = p * n_ell + e for bin pair p (i <= j, row-major
 * over i then j) and multipole e. */
typedef struct {
    int n_bins;
    const double* nz_mean;        /* Gaussian n_i(z) mean per bin */
    const double* nz_sigma;       /* and width */
    int n_ell;
    const double* ell;            /* multipoles */
    int n_k;                      /* table k grid: uniform in ln k on [lnk_min, lnk_max] */
    double lnk_min, lnk_max;
    int n_z;                      /* table z grid: uniform on [0, z_max] */
    double z_max;
    int n_z_emu;                  /* emulator z nodes: n_z, or fewer (uniform on [0, z_max])
                                     interpolated to n_z by Catmull-Rom in z */
    int n_chi;                    /* chi grid: uniform in a on [a_min, 1], node 0 at a = 1 */
    double a_min;
    double ia_pivot;              /* A(z) = A_IA ((1 + z) / ia_pivot)^eta_IA */
    double c1rho;                 /* C_1 rho_cr (Eq. 6) */
    int n_tmpl;
    const double* tmpl;           /* n_data x n_tmpl noise templates (may be NULL if n_tmpl = 0) */
    int z_interp;                 /* coarse emulator z -> table z (n_z_emu < n_z): 0 Catmull-Rom
                                     (4 taps), 1 linear between the bracketing coarse nodes (the
                                     paper's interpolated P(k), App. B) */
} ns_shear_desc;

/* CMB problem kind (Sec. 3.1).  The model is the emulator output itself (TT,
 * TE, EE stacked, dims[n_layers] values), inputs = the full parameter vector;
 * the emulator's last layer is linear.  Two likelihood forms:
 *   NS_CMB_GAUSS (dense covariance): log L = -1/2 |L^-1 (d - m)|^2 + c0 with
 *     d and cov of length D = dims[n_layers]; `solve` as above.
 *   NS_CMB_TT_CV (the paper's cosmic-variance-limited TT analysis, Sec. 3.1):
 *     for each of the first n_tt outputs (multipoles ell[i]), k = 2 ell + 1 and
 *     k d_ell / C_ell(theta) follows a chi-squared law with k degrees of
 *     freedom; log L = sum_ell [ln f_chi2(k d / C; k) + ln(k / C)], i.e. the
 *     density of d_ell given C_ell.  data = the n_tt observed TT values
 *     (n_data = n_tt), cov = NULL.
 * Precisions FP64, FP32 and BF16 (hidden layers on tensor cores, head and the
 * likelihood sums in FP32, constants and the final sum in FP64); LITERAL
 * needs FP64. */
enum ns_cmb_form { NS_CMB_GAUSS = 0, NS_CMB_TT_CV = 1 };
typedef struct {
    int solve;                    /* ns_cmb_solve (NS_CMB_GAUSS only) */
    int form;                     /* ns_cmb_form */
    int n_tt;                     /* NS_CMB_TT_CV: TT multipoles = the first n_tt emulator outputs */
    const double* ell;            /* NS_CMB_TT_CV: their multipoles (n_tt values) */
} ns_cmb_desc;

/* Isotropic Gaussian test likelihood on the cube: log L = -1/2 |(x - mu)/sigma|^2 - d ln(sigma sqrt(2 pi)). */
typedef struct { double mu; double sigma; } ns_gauss_desc;

typedef struct {
    int kind;                     /* ns_kind */
    int precision;                /* ns_precision */
    int n_params;                 /* length of the full parameter vector */
    const ns_prior* priors;       /* n_params */
    int n_data;                   /* D (shear, CMB); ignored for GAUSS */
    const double* data;           /* D */
    const double* cov;            /* D x D symmetric positive definite; factorised in FP64.
                                     data and cov may both be NULL: a model-only problem whose
                                     loglike calls fail with NS_EINVAL (the CMB TT_CV form takes
                                     data and no covariance) */
    ns_emulator_desc emu;
    ns_shear_desc shear;
    ns_gauss_desc gauss;
    int max_batch;                /* largest batch B any call will pass (>= 1) */
    ns_cmb_desc cmb;
    int hidden_tile;              /* BF16 emulator layers: 0 = per-layer tcgen05 GEMMs with N-tiles
                                     chosen by the tile autotuner at creation; 16, 32, 64 or 128 (at
                                     most the layer's width) = per-layer GEMMs with that N-tile;
                                     -1 = the input and hidden layers as one clustered kernel
                                     (activations kept in shared memory and exchanged between the
                                     cluster's CTAs; tanh, every hidden width 512 or 1024, at most 4
                                     hidden layers, at most 32 inputs, shear kind, else NS_ENOTSUP).
                                     Results are bit-identical in every mode. */
} ns_problem_desc;

typedef struct ns_problem ns_problem;
typedef struct ns_run ns_run;
typedef struct ns_multi ns_multi;

/* Nested-sampling settings (Sec. 2.1-2.2 and the recorded readings of the
 * slice-sampler internals). */
typedef struct {
    int n_live;                   /* n */
    int n_delete;                 /* k: deleted per iteration, chains evolved in parallel */
    int repeats;                  /* slice moves per chain; <= 0 means 5 d */
    double tol;                   /* stop when ln(Z_dead + Z_live) - ln Z_dead < tol */
    unsigned long long seed;      /* Philox4x32-10 key */
    double width;                 /* initial slice width along a unit-Mahalanobis direction */
    int step_cap;                 /* cap on stepping-out steps and on shrinkage steps */
    double ridge;                 /* added to the live-covariance diagonal */
    int rounds_per_sync;          /* likelihood rounds launched between host checks (<= 0: 16);
                                     rounded up to an even number */
    int chain_groups;             /* 1 or 2 groups of chains whose likelihood rounds run on two
                                     streams and overlap on the GPU (results are identical);
                                     <= 0: 1 */
    int n_shards;                 /* > 1: one nested-sampling run split over n_shards devices,
                                     this run object evolving shard `shard` of the k chains
                                     (ns_shard_*); 0 or 1: an ordinary run */
    int shard;                    /* shard index in [0, n_shards) */
} ns_config;

typedef struct {
    long long iterations;         /* NS iterations completed by this run */
    long long evaluations;        /* likelihood evaluations (init included) */
    long long rounds;             /* batched likelihood rounds launched */
    int converged;                /* termination criterion met */
    int status_bits;              /* NS_BIT_* */
    double logZ;                  /* dead-point evidence so far */
    double logX;                  /* log enclosed prior mass */
    double lstar;                 /* last deletion threshold */
    long long nonfinite;          /* likelihood evaluations that returned NaN / inf (each treated
                                     as outside the constraint; sets NS_BIT_NONFINITE) */
} ns_status;

/* ---- entry points ------------------------------------------------------- */

/* Static description of a status code (never NULL). */
const char* ns_strerror(int code);

/* Build a problem on the current CUDA device: copies every host array, converts
 * weights to the problem precision, factorises cov = L L^T in FP64 (on the host
 * for D <= 1024, else by blocked FP64 kernels on the device), forms L^-1 (and,
 * for the CMB fold, W' and c') and the constant c0 = -sum ln L_aa - D/2 ln 2 pi.
 * Errors: NS_EINVAL (bad sizes, non-SPD covariance, unknown enums),
 * NS_ENOMEM, NS_ECUDA, NS_ENOTSUP (e.g. BF16 with shapes the tensor-core
 * path cannot tile). */
int ns_problem_create(const ns_problem_desc* desc, ns_problem** out);
int ns_problem_free(ns_problem* p);

/* Number of free (non-FIXED) parameters d: the dimension of the unit cube the
 * sampler explores (Sec. 2.5: 39 for w0-wa, 37 for LCDM). */
int ns_problem_dim(const ns_problem* p, int* d);

/* Prior transform of Table 1 (Sec. 2.5 priors; every prior is uniform in the
 * unit cube, where the sampler works): cube_dev (B x d) in (0,1) -> theta_dev
 * (B x d) physical free parameters, uniform a + (b - a) c, Gaussian
 * a + b Phi^-1(c).  Phi^-1 is the sampler's: FP64 for FP64 problems, FP32 on
 * min(c, 1 - c) for reduced-precision problems (finite on all of (0, 1)).
 * B <= max_batch, else NS_EINVAL. */
int ns_prior_transform(const ns_problem* p, const double* cube_dev, int B,
                       double* theta_dev, void* stream);

/* Batched log-likelihood at physical free parameters theta_dev (B x d):
 * logL_dev[b] = log L(theta_b).
 *   Shear kind: the Gaussian likelihood of App. A, log L = -1/2 (d - m)^T
 *     C^-1 (d - m) - 1/2 ln det(2 pi C), with the data vector
 *     m = (1 + m_i)(1 + m_j) C_ij(ell) + T b, C_ij(ell) the extended Limber
 *     integral of Eq. 3-4 (k = (ell + 1/2) / chi) over the windows of Eq. 5
 *     (lensing) and Eq. 6 (intrinsic alignment) on the a-uniform chi grid of
 *     App. A, with P(k, z) from the emulator of Sec. 2.5 and the photo-z
 *     shifts n_i(z - D_z,i).
 *   CMB kind: Sec. 2.4 (cosmic-variance TT form) or a dense Gaussian.
 *   Gaussian test kind: the closed form below.
 * theta_dev and logL_dev are caller-owned device memory (row-major FP64).
 * B <= max_batch (else NS_EINVAL); B = 0 is a no-op.  NS_EINVAL for a
 * model-only problem.  Non-finite results are returned as they are. */
int loglike_batch(const ns_problem* p, const double* theta_dev, int B,
                  double* logL_dev, void* stream);

/* Model data vector m(theta) (B x D, FP64 out), before the residual: the shear
 * spectra with biases and templates, or the CMB emulator output.  Used to
 * build mock data.  NS_EINVAL for the GAUSS kind. */
int ns_model_batch(const ns_problem* p, const double* theta_dev, int B,
                   double* model_dev, void* stream);

/* Emulator output (B x dims[n_layers], FP64 out) at physical free parameters:
 * for the shear kind log10 P on the emulator's (z, k) grid, z-major, for the
 * CMB kind the spectra; computed in the problem precision (BF16: tcgen05 GEMMs
 * with FP32 accumulation).
 * NS_EINVAL for the GAUSS kind. */
int ns_emulator_batch(const ns_problem* p, const double* theta_dev, int B,
                      double* out_dev, void* stream);

/* BF16 problems: the N-tile width of every tensor-core layer (0 for layers on
 * CUDA cores; 128 for the layers of the fused stack, whose CTAs own 128
 * features of a 64-row tile) and, for autotuned hidden layers, the time per
 * launch [ms] the tile autotuner measured at creation on min(max_batch, 384)
 * rows (0 otherwise); ms may be NULL.  n >= the number of emulator layers. */
int ns_problem_tiles(const ns_problem* p, int* tile_n, float* ms, int n);

/* BF16 problems: *cluster_size = the thread-block cluster size of the fused
 * input + hidden-layer kernel (its CTAs own 128 features each of a 64-row
 * tile), or 0 when the layers run as separate GEMMs. */
int ns_problem_fused(const ns_problem* p, int* cluster_size);

/* Device status bits of the problem's batch calls (NS_BIT_TIMEOUT: a bounded
 * device wait inside a likelihood kernel gave up; the affected rows are NaN).
 * Synchronises the device first; clear != 0 resets the bits.  Runs check the
 * same bits at every host synchronisation and stop with NS_ETIMEOUT. */
int ns_problem_status(ns_problem* p, int* bits, int clear);

/* Log-likelihood (as loglike_batch) and its gradient d log L / d theta
 * (grad_dev, B x d, caller-owned device memory) by a hand-written reverse
 * pass through the stages of App. A (chi^2, data vector, Limber Eq. 3-4,
 * windows Eq. 5-6, distances and growth, the emulator of Sec. 2.5 and the
 * Table 1 prior's physical parameters); the paper's pipeline is
 * auto-differentiable (Sec. 2.2, Sec. 4.2) and its HMC comparison runs use
 * these gradients (Sec. 3.2).  Shear kind; closed form for the Gaussian test
 * kind; NS_ENOTSUP for the CMB kind.  B <= max_batch, else NS_EINVAL. */
int loglike_grad_batch(const ns_problem* p, const double* theta_dev, int B,
                       double* logL_dev, double* grad_dev, void* stream);

/* No-U-Turn sampler (Hoffman & Gelman 2014, slice variable, dual averaging) on
 * the problem's posterior, for the HMC comparison runs of Sec. 3.2.  Target:
 * unconstrained z in R^d with cube coordinate c = 1/(1 + e^-z), theta = the
 * prior transform of c, log p(z) = log L(theta) + sum ln(c (1 - c)).  The
 * chains advance in lockstep: each leapfrog round is one loglike_grad_batch
 * call over the chains still building their subtree; the control logic runs
 * on the host in FP64.  Random numbers: Philox4x32-10, counter
 * (purpose | j << 8, iteration, chain, extra) with purposes 7 momentum (j =
 * dimension pair, Box-Muller), 8 slice, 9 direction (j = depth), 10 merge
 * (j = depth), 11 reservoir (j = depth, extra = leaf index).
 * Warm-up: dual averaging (gamma 0.05, t0 10, kappa 0.75, mu = ln(10 eps0))
 * towards target_accept; with adapt_mass the inverse mass becomes the
 * regularised variance of z over warm-up iterations [W/4, 3W/4) and dual
 * averaging restarts there; sampling uses the averaged step size.
 * z0 (host, n_chains x d): starting points.  samples (host, n_chains x
 * n_samples x d): z after each kept iteration (map to theta with
 * ns_prior_transform of the logistic); logp (host, may be NULL): log p(z).
 * step_size (host, n_chains, may be NULL): final step sizes.  Synchronous.
 * Shear and Gaussian-test kinds; n_chains <= max_batch. */
typedef struct {
    int n_chains;
    int n_warmup;
    int n_samples;
    unsigned long long seed;
    double target_accept;         /* delta, e.g. 0.8 */
    int max_depth;                /* trajectory doublings (1 .. 20), e.g. 10 */
    double init_step;             /* eps0 > 0 */
    int adapt_mass;               /* 1: diagonal inverse mass from the warm-up window */
} ns_nuts_config;

typedef struct {
    long long gradient_evals;     /* leapfrog steps summed over chains */
    long long batched_calls;      /* lockstep rounds (batched gradient calls) */
    int divergences;              /* divergent transitions among the kept iterations */
    double mean_depth;            /* mean trajectory doublings of the kept iterations */
    double mean_accept;           /* mean acceptance statistic of the kept iterations */
} ns_nuts_stats;

int ns_nuts_run(const ns_problem* p, const ns_nuts_config* cfg, const double* z0, double* samples,
                double* logp, double* step_size, ns_nuts_stats* stats, void* stream);

/* Start a nested-sampling run (Sec. 2.1): draws n live points from the prior,
 * i.e. uniformly in the unit cube (Philox counter (INIT | chunk << 8, 0,
 * point, 0)), evaluates them, zeroes the evidence accumulators (Z = 0,
 * X = 1).  *out is owned by the caller until ns_free.  The run keeps the problem pointer: free the run first.
 * Errors: NS_EINVAL (n_delete not in [1, n_live - 1], n_delete > max_batch,
 * n_live > 4096, d > 64). */
int ns_init(const ns_problem* p, const ns_config* cfg, void* stream, ns_run** out);

/* Run up to n_iters nested-sampling iterations (Sec. 2.1-2.2; fewer if the
 * termination criterion is met) and fill *st (may be NULL).  An iteration
 * deletes the k lowest live points (L* = the k-th lowest log L), books them
 * into Z (Eq. 1) and X with n, n-1, ..., n-k+1 live points, and replaces them
 * by k slice-sampling chains (Neal 2003, the NSS scheme the paper adopts) that
 * evolve in parallel under the hard constraint log L > L*.  n_iters = 0 only
 * fills *st.  Errors: NS_ETIMEOUT (a bounded device wait gave up, or the round
 * bound was reached), NS_ECUDA.  Synchronises the run's stream. */
int ns_step(ns_run* r, int n_iters, ns_status* st);

/* Final evidence (Eq. 1, the dead points weighted by the expected prior-volume
 * shrinkage) with the live points added (ascending log L with n, n-1, ...
 * 1 live points) without changing the run: log Z, its error (standard
 * deviation over n_replays simulated shrinkage sequences, Philox counters
 * (ERR, replay, dead index, 0); n_replays <= 0 means 200), log X, the
 * information H and the number of dead points including the live ones.
 * Any output pointer may be NULL.  Synchronises the run's stream. */
int ns_evidence(const ns_run* r, int n_replays, double* logZ, double* logZ_err,
                double* logX, double* H, long long* n_dead);
/* (The simulated-shrinkage error assumes, as the paper's Sec. 4.2 notes, that
 * each new point is drawn uniformly within the constraint; the slice chains
 * approximate that draw.  Errors: NS_EINVAL for a NULL run, NS_ENOMEM,
 * NS_ECUDA.) */

/* Evidence of a dead-point sequence that the caller holds on the device, for
 * callers that cannot allocate device memory when they need the number: a host
 * framework that reserves the device memory up front for its own caching pool
 * (a library cudaMalloc then fails or fragments that pool), or a control loop
 * that must not call cudaMalloc / cudaFree because they can synchronise the
 * device.  It allocates nothing: the per-replay values live in a library-owned
 * array of 4096 doubles that every GPU loading the library keeps until the
 * process exits.  The paper has no counterpart; this is an interface
 * convenience.
 *   logL_dev  (n) log L of the dead points in deletion order, the final live
 *             points appended in ascending order;
 *   nlive_dev (n) live-point count booked for each (n_live - j within a batch;
 *             n_live, n_live - 1, ..., 1 for the appended live points);
 *   out_dev   (3) ln Z by the expected shrinkage, its simulated-shrinkage
 *             standard deviation (ddof 1) over n_replays Philox replays
 *             (counters (ERR, replay, index, 0) with key `seed`, so the same
 *             sequence and seed give ns_evidence's error), and the final ln X.
 * n_replays <= 0 means 200; 2 <= n_replays <= 4096 else NS_EINVAL.  Every live
 * count must be >= 1; a smaller one makes all three outputs NaN.  The first
 * call on a device looks up the array's device address (cudaGetSymbolAddress)
 * with that device current: make that first call before any stream capture.
 * The address is kept for the process; calls after a cudaDeviceReset of that
 * device are not supported.  All calls on a device share the array, so calls
 * that overlap on the GPU race; each call writes every slot it reads, so
 * nothing needs clearing. */
int ns_evidence_noalloc(const double* logL_dev, const int* nlive_dev, long long n,
                        unsigned long long seed, int n_replays, double* out_dev, void* stream);

/* One run split over several devices (the multi-device direction the paper
 * leaves to future work, Sec. 4.1 and Sec. 5; the k chains of an iteration are
 * independent, Sec. 2.2).  Every device holds an ns_run of the same problem and
 * config (seed included) with n_shards = G and its own shard index s; the live
 * set, deletion, evidence update, covariance factor and chain starts are
 * computed redundantly and identically on every device, and shard s evolves
 * the contiguous chains [floor(k s / G), floor(k (s + 1) / G)).  Per iteration:
 *   ns_shard_evolve   deletion, evidence update, covariance, directions and
 *                     starts, then the likelihood rounds of this shard's
 *                     chains (synchronises the run's stream); does nothing
 *                     once the run has converged (st->converged = 1);
 *   ns_shard_export   this shard's final chain states into finals_dev
 *                     (caller-owned device memory, rows = the shard's chain
 *                     count, row = x[0..d), log L, evaluation count; FP64),
 *                     asynchronously on the run's stream;
 *   (the caller all-gathers the shards' rows in shard order, e.g. with NCCL;
 *    the only exchange of the iteration: k (d + 2) doubles in total)
 *   ns_shard_insert   all k rows in chain order (caller-owned device memory):
 *                     the final points replace the deleted slots and the
 *                     termination test is updated (synchronises).
 * Each shard then holds exactly the single-device run's state (the chains draw
 * from Philox counters keyed by chain index, and a likelihood value does not
 * depend on the batch it is evaluated in), except that status bits and the
 * non-finite count are the shard's own.  ns_step with n_iters > 0 returns
 * NS_EINVAL on a shard; the ns_shard_* calls out of order return NS_EINVAL. */
int ns_shard_evolve(ns_run* r, ns_status* st);
int ns_shard_export(const ns_run* r, double* finals_dev);
int ns_shard_insert(ns_run* r, const double* all_finals_dev, ns_status* st);
/* The chain range [*chain_begin, *chain_end) this run evolves (0, k unless sharded). */
int ns_shard_range(const ns_run* r, int* chain_begin, int* chain_end);

/* Copy out the live set (x: n x d cube coordinates, logL: n); either may be NULL. */
int ns_live_points(const ns_run* r, double* x, double* logL);

/* Copy out up to max_out dead points in deletion order (x: cube coordinates,
 * logL, and the live-point count booked for each).  *n_out = number copied. */
int ns_dead_points(const ns_run* r, long long max_out, double* x, double* logL,
                   int* n_live_at_death, long long* n_out);

/* Record of the last completed iteration: L*, deleted live slots (k, ascending
 * (log L, slot)), start slots (k), evaluations per chain (k).  Any may be NULL. */
int ns_last_iteration(const ns_run* r, double* lstar, int* deleted, int* starts, int* evals);

/* Packed runs: n_runs independent nested-sampling runs (Sec. 2.1-2.2 each)
 * whose problems share one likelihood model (same kind, precision, emulator,
 * data and covariance: problems[0]'s model is used for every likelihood call)
 * but may differ in their priors -- hence in their dimension, e.g. the 37-d
 * LCDM and 39-d w0-wa models of one data set -- and in cfgs[i] (n_live,
 * n_delete, seed, ...).  Every round packs the proposals of all runs' chains
 * into one batch, tagged with the run index for the prior transform, and
 * scores it with one likelihood launch; each run keeps its own iteration
 * cycle, started and finished by the host between graph launches.
 * Errors: NS_EINVAL for mismatched problems or n_runs outside [1, 64]. */
int ns_multi_init(const ns_problem* const* problems, int n_runs, const ns_config* cfgs, void* stream,
                  ns_multi** out);

/* Each run not yet converged makes up to n_iters more iterations; st (may be
 * NULL) receives n_runs statuses.  Synchronises the stream. */
int ns_multi_step(ns_multi* m, int n_iters, ns_status* st);

/* Borrow run i (for ns_evidence, ns_live_points, ns_dead_points, ...); it
 * stays owned by m: do not ns_free it. */
int ns_multi_run(const ns_multi* m, int i, ns_run** out);

int ns_multi_free(ns_multi* m);

/* Stage timing for roofline reporting: with stage != 0, every graph launch of
 * likelihood rounds records CUDA events on its stream around that stage in its
 * first round (1 = shear Limber stage: P lookup, Limber sums, data vector,
 * including any wait for the windows stage; 2 = emulator output GEMM;
 * 3 = whitening / chi^2; 4 = first hidden emulator GEMM; 5 = shear windows
 * stage: distances, growth, windows, on its own stream beside the emulator)
 * and the stage's batch size.  0 turns it off.
 * Resets the accumulators. */
int ns_profile_stage(ns_run* r, int stage);

/* Accumulated stage time [ms], number of timed launches and rows they processed. */
int ns_profile_read(const ns_run* r, double* total_ms, long long* launches, long long* rows);

int ns_free(ns_run* r);

#ifdef __cplusplus
}
#endif
#endif /* GPUNS_H */
