// Internal interfaces of the likelihood stages (not part of the C ABI).
#pragma once

#include <cuda.h>
#include <vector>

#include "common.cuh"

namespace gpuns {

// Device-side description of the shear model (App. A), built at problem creation.
struct ShearParams {
    int n_params, nb, n_pairs, n_ell, n_k, n_z, N, D, n_tmpl;
    double lnk_min, lnk_max, dlnk, ia_pivot, c1rho;
    double dz;            // table z spacing
    const float* a_f;     // FP32 copies of the node constants
    const float* lna_f;
    const float* z_f;
    const float* wa_f;
    const int* zrp;       // N   padded-table row of each node's first z-tap
    const float* zw4f;    // 4N  doubled Catmull-Rom z-weights (unfolded)
    const double* zw4d;
    const double* a;      // N   scale factor at chi nodes (node 0: a = 1)
    const double* lna;    // N
    const double* z;      // N
    const double* wa;     // N   trapezoid weights in a
    const int* zrow;      // 4N  z-taps of the P table at each node (ghosts folded)
    const double* zw;     // 4N
    const double* lnell;  // n_ell  ln(ell + 1/2)
    const double* nz_mean;
    const double* nz_sigma;
    const int* pi;        // n_pairs
    const int* pj;
    const double* data;   // D
    const double* tmpl;   // D x n_tmpl
    // FP32 copies read by the float kernels (GB300 runs FP64, conversions
    // included, at a small fraction of its FP32 rate, so float kernels take no
    // per-thread double -> float conversions)
    float lnk_min_f, lnk_max_f, inv_dlnk_f, ia_pivot_f, c1rho_f;
    const float* lnell_f;
    const float* nz_mean_f;
    const float* nz_sigma_f;
    const float* data_f;
    const float* tmpl_f;
};

struct Workspace {
    int cap = 0;
    int* d_nrows = nullptr;       // device row count used by every stage
    int* d_err = nullptr;         // device status bits (NS_BIT_TIMEOUT when a bounded wait gave up)
    int* h_err = nullptr;         // pinned mirror of d_err
    double* theta_full = nullptr; // cap x P
    void* act[2] = {nullptr, nullptr};
    void* table = nullptr;        // cap x n_out (emulator output)
    void* table_fine = nullptr;   // cap x n_z*n_k (coarse-z emulators)
    void* resid = nullptr;        // cap x D residuals
    void* win = nullptr;          // cap x (nb + 1) x pitch: ln chi and windows (pitch = N rounded up to 4)
    double* logL = nullptr;       // cap
    // tcgen05 tensor maps (BF16 precision): A operand of layer l >= 1 and its output
    std::vector<CUtensorMap> tmA;
    CUtensorMap tmX_out{};        // the last layer's activations in kSwapRows-row boxes
    CUtensorMap tmF_out{};        // fused emulator stack: its output activations in 64-row boxes of two k-blocks
    std::vector<void*> owned;
    // second stream for the emulator-independent windows stage; fork/join events
    cudaStream_t side = nullptr;
    cudaEvent_t ev_fork = nullptr, ev_join = nullptr;
};

}  // namespace gpuns

struct ns_problem {
    int kind = 0, precision = 0, P = 0, d = 0, D = 0, max_batch = 0;
    std::vector<ns_prior> priors;
    int* d_pkind = nullptr;
    double* d_pa = nullptr;
    double* d_pb = nullptr;
    int* d_free_of_full = nullptr;   // P: free index or -1
    // gauss
    double g_mu = 0.5, g_sigma = 0.05;
    // emulator
    int n_layers = 0;
    std::vector<int> dims;
    std::vector<void*> d_W;          // per layer, compute dtype (layer 0: FP64 or FP32)
    std::vector<void*> d_b;          // per layer, FP64 (FP64 mode) else FP32
    std::vector<CUtensorMap> tmB;    // BF16: weight tensor maps for layers >= 1
    std::vector<int> tile_n;         // BF16: N tile per layer (hidden layers autotuned at creation)
    std::vector<float> tile_ms;      // BF16: measured time per launch of the chosen hidden tiles
    int fused_cs = 0;                // BF16: > 0 when the input and hidden layers run as one clustered kernel
                                     // (cluster of fused_cs CTAs, hidden width 128 fused_cs)
    std::vector<CUtensorMap> tmF;    // its weight maps: boxes of 128 rows x two k-blocks
    int* d_inputs = nullptr;
    double* d_in_center = nullptr;
    double* d_in_scale = nullptr;
    double* d_in_inv_scale = nullptr;  // 1 / in_scale (reduced-precision input layer)
    void* d_out_mu = nullptr;        // FP64 or FP32
    double out_sigma = 1.0;
    int hidden_max = 0;
    // shear
    gpuns::ShearParams sp{};
    int n_z_emu = 0;
    int* d_zi_row = nullptr;         // n_z x 4 coarse -> fine z taps
    double* d_zi_w = nullptr;
    // chi2
    double c0 = 0.0;
    double* d_LinvT64 = nullptr;     // D x D: LinvT[b*D + a] = (L^-1)[a][b]
    float* d_LinvT32 = nullptr;
    bool has_lik = true;             // false for a model-only problem (no data / covariance)
    // activations (per hidden layer l < n_layers - 1, compute dtype; FP32 for BF16)
    int act = 0;
    std::vector<void*> d_act_g, d_act_beta;
    void* d_out_sig = nullptr;       // per-output scales (compute dtype) or null: scalar out_sigma
    // CMB
    int cmb_solve = 0;
    void* d_Wfold = nullptr;         // D x H: W' = L^-1 diag(sigma) W_out (compute dtype)
    void* d_cfold = nullptr;         // D: c' = L^-1 (d - mu - sigma b_out)
    void* d_zeroD = nullptr;         // D zeros: bias of the folded head
    double* d_lit_mu = nullptr;      // LITERAL: d - mu
    double* d_lit_sig = nullptr;     // LITERAL: -sigma
    int cmb_form = 0;                // ns_cmb_form
    int n_tt = 0;                    // TT_CV: multipoles (the first n_tt outputs)
    void* d_tt_obs = nullptr;        // TT_CV: observed d_ell (compute dtype)
    void* d_tt_halfk = nullptr;      // TT_CV: k/2 = ell + 1/2 (compute dtype)
    std::vector<void*> owned;
    gpuns::Workspace ws;             // scratch of loglike_batch / ns_model_batch
};

namespace gpuns {

int workspace_create(const ns_problem* p, int cap, Workspace* ws);
// Queue a copy of the device status bits into the pinned mirror on `st`; after
// the stream has synchronised, workspace_err_bits returns them.
int workspace_err_fetch(Workspace* ws, cudaStream_t st);
inline int workspace_err_bits(const Workspace* ws) { return ws->h_err ? *ws->h_err : 0; }
void workspace_free(Workspace* ws);

// Full likelihood pipeline on rows [0, *d_nrows) of ws->theta_full; grid_rows
// bounds the row count for grid sizing.  Writes logL_out (FP64) or, when
// model_out != nullptr, the shear model vectors (FP64, rows x D) instead.
// Optional probe around one likelihood stage: events recorded on the launch
// stream before/after it and the stage's row count copied to pinned memory.
enum ProbeStage {
    PROBE_NONE = 0, PROBE_PROJECTION = 1, PROBE_EMU_OUT = 2, PROBE_CHI2 = 3, PROBE_EMU_HIDDEN = 4, PROBE_WINDOWS = 5
};
struct StageProbe {
    int stage = PROBE_NONE;
    cudaEvent_t ev0 = nullptr, ev1 = nullptr;
    int* h_rows = nullptr;   // pinned
};

int run_likelihood(const ns_problem* p, Workspace* ws, int grid_rows,
                   double* logL_out, double* model_out, cudaStream_t st, const StageProbe* probe = nullptr);

// Emulator stage only; writes the raw emulator output as FP64 (rows x n_out).
int run_emulator_only(const ns_problem* p, Workspace* ws, int grid_rows, double* out, cudaStream_t st);

// Prior transform into the workspace: cube (rows x d) -> theta_full.
int launch_cube_to_theta(const ns_problem* p, Workspace* ws, const double* cube, int grid_rows,
                         cudaStream_t st);

// Shear projection (projection.cu), two stages.  Windows: per row ln chi and
// the lensing/IA windows into `win` (rows x (nb + 1) x N); independent of the
// emulator, so it may run on a second stream beside it.  Limber: P lookup,
// Limber sums and the data vector; writes the residual d - m per row, or the
// model vectors when model_out != nullptr.  FAST selects SFU transcendentals.
template <typename T, bool FAST>
int launch_windows(const ShearParams& sp, const double* theta_full, T* win, const int* nrows, int grid_rows,
                   cudaStream_t st);
template <typename T, bool FAST>
int launch_limber(const ShearParams& sp, const double* theta_full, const T* table, const T* win, T* resid,
                  double* model_out, const int* nrows, int grid_rows, int* err, cudaStream_t st);
// Whether both projection stages fit the shared memory of one CTA (elt = 4 or 8).
bool projection_fits(const ShearParams& sp, int elt);
// Whitened chi^2 and log L = c0 - chi^2 / 2 (projection.cu).  rows_ready: the
// row count is final before the preceding kernel completes (the shear
// likelihood's fork / join events), so the kernel may read it, and request
// the constant L^-T, before its dependency wait.
template <typename TR, typename TA>
int launch_chi2(const TR* resid, int D, const TA* LinvT, double c0, double* logL, const int* nrows, int grid_rows,
                cudaStream_t st, bool rows_ready = false);

// Adjoint of the shear projection (adjoint.cu).
int adjoint_scratch_elems(const ShearParams& sp);
template <typename T>
int launch_projection_adj(const ShearParams& sp, const double* theta_full, const T* table, const T* LinvT, double c0,
                          T* scratch, T* gtab, double* gfull, double* logL, const int* nrows, int grid_rows,
                          cudaStream_t st);
int launch_free_to_full(const ns_problem* p, const double* theta, int B, double* theta_full, cudaStream_t st);
int launch_zinterp_generic(const ns_problem* p, const void* coarse, void* fine, const int* nrows, int grid_rows,
                           int elt, cudaStream_t st);
int launch_free_to_full_ext(const ns_problem* p, const double* theta, int B, double* theta_full, cudaStream_t st);

// BF16 tcgen05 GEMM: C[M x N] = epi(A[M x K] * W[N x K]^T + bias), M = *d_nrows.
// epi 0: tanh -> bf16 C (ldc = N); epi 1: mu + sigma * v -> fp32 C.
// Epilogues of the tensor-core GEMM: hidden tanh -> bf16; output
// mu + sigma (acc + b) -> FP32; hidden sigmoid-linear -> bf16 with per-unit
// g (passed as out_mu) and beta (act_beta).
enum { TC_EPI_TANH = 0, TC_EPI_OUT = 1, TC_EPI_SIGLIN = 2 };
int launch_gemm_tc(const CUtensorMap* tmA, const CUtensorMap* tmB, int tile_n,
                   const float* bias, const float* out_mu, float out_sigma,
                   void* C, const int* d_nrows, int grid_rows, int N, int K, int epi,
                   const float* act_beta, int* d_err, cudaStream_t st);
// k-blocks of 64 per ring slot of launch_gemm_tc for a reduction length K; its
// tmA and tmB must be made with kps = gemm_tc_kps(K).
int gemm_tc_kps(int K);
// bf16 tensor map over a row-major rows x K matrix: kps = 1 a 2-D map with
// box_rows x 64 boxes; kps > 1 a 3-D view whose box is kps such tiles.
int make_tensor_map_bf16(CUtensorMap* tm, const void* base, int rows, int K, int box_rows, int kps = 1);
// Split-BF16 tcgen05 GEMM (adjoint): C = epi((A_hi + A_lo) W^T + ...) with A
// given as a bf16 (hi, lo) pair whose sum is the FP32 operand; tmAhi / tmAlo box
// 128 rows, tmB boxes tile_n (64, 128, 256) rows of W (N x K).  Epilogues:
// SPL_TANH (C, C_lo) = split(tanh(acc + b)); SPL_OUT C (FP32) = mu + sigma (acc + b);
// SPL_DTANH (C, C_lo) = split(acc (1 - h^2)), h = aux_hi + aux_lo (rows x N);
// SPL_DTANH32 the same into FP32 C.  Row pitch of every output and aux: N.
enum { SPL_TANH = 0, SPL_OUT = 1, SPL_DTANH = 2, SPL_DTANH32 = 3 };
int launch_gemm_split(const CUtensorMap* tmAhi, const CUtensorMap* tmAlo, const CUtensorMap* tmB, int tile_n,
                      const float* bias, const float* out_mu, float out_sigma, void* C, __nv_bfloat16* C_lo,
                      const __nv_bfloat16* aux_hi, const __nv_bfloat16* aux_lo, const int* d_nrows, int grid_rows,
                      int N, int K, int epi, int* d_err, cudaStream_t st);
// Output layer with swapped operands (rows of W as the MMA's M, activation rows
// as its N, kSwapRows per CTA): tmW boxes 128 rows of W, tmX boxes kSwapRows
// activation rows; FP32 out = mu + sigma (acc + b), row-major rows x N.
constexpr int kSwapRows = 256;
// Fused emulator stack (gemm_tc.cu): the input layer and every hidden layer of
// a BF16 tanh emulator whose hidden widths all equal 128 p->fused_cs, one
// thread-block cluster per 64-row tile; writes the last hidden layer's
// activations through ws->tmF_out.
constexpr int kFusedMaxHidden = 4;
int launch_emu_fused(const ns_problem* p, const Workspace* ws, int grid_rows, cudaStream_t st);
int launch_gemm_tc_out_swap(const CUtensorMap* tmW, const CUtensorMap* tmX, const float* bias, const float* out_mu,
                            float out_sigma, float* C, const int* d_nrows, int grid_rows, int N, int K, int* d_err,
                            cudaStream_t st);
// Dense FP64 set-up kernels (dense_linalg.cu): C (device, overwritten by L) ->
// L^-1 (new device buffer) and sum ln L_aa; NS_EINVAL if C is not SPD.
int device_cholesky_inverse(double* dC, int D, double** Xout, double* sum_log_diag, cudaStream_t st);
int device_transpose(const double* dA, double* dT, int D, cudaStream_t st);
// C = A W^T on the device in FP64 (likelihood.cu); nrows_dev holds M; zeros_n: N zeros.
int gemm_f64_plain(const double* A, const double* W, double* C, const int* nrows_dev, int M, int N, int K,
                   const double* zeros_n, cudaStream_t st);
int gemm_tc_supported(int N, int K);

}  // namespace gpuns
