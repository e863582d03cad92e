// Likelihood stages on CUDA cores (FP64 / FP32) and the pipeline driver.
//
//   prior transform   Table 1 (uniform, Gaussian via Phi^-1, fixed)
//   emulator          MLP stand-in for CosmoPower (Sec. 2.5): input layer on
//                     CUDA cores, hidden/output layers as GEMMs (SIMT here,
//                     tcgen05 tensor cores for BF16 in gemm_tc.cu)
//   projection.cu     App. A projection (distances, windows, P lookup, Limber,
//                     data vector) and the whitened chi^2.
#include <algorithm>

#include "likelihood.cuh"

namespace gpuns {

__global__ void k_set_int(int* p, int v) {
    pdl_begin();
    *p = v;
}

__constant__ double c_glx[4] = {-0.86113631159405257522, -0.33998104358485626480,
                                 0.33998104358485626480, 0.86113631159405257522};
__constant__ double c_glw[4] = {0.34785484513745385737, 0.65214515486254614263,
                                 0.65214515486254614263, 0.34785484513745385737};

// ------------------------------------------------------------ prior transform
__global__ void k_cube_to_theta(const double* __restrict__ cube, int d, int P,
                                const int* __restrict__ kind, const double* __restrict__ pa,
                                const double* __restrict__ pb, const int* __restrict__ free_of_full,
                                double* __restrict__ theta_full, const int* __restrict__ nrows) {
    pdl_begin();
    const int row = blockIdx.x;
    if (row >= *nrows) return;
    for (int i = threadIdx.x; i < P; i += blockDim.x) {
        const int f = free_of_full[i];
        double v;
        if (f < 0) {
            v = pa[i];
        } else {
            const double c = cube[(size_t)row * d + f];
            if (kind[i] == NS_PRIOR_UNIFORM) v = pa[i] + (pb[i] - pa[i]) * c;
            else v = pa[i] + pb[i] * normcdfinv(c);
        }
        theta_full[(size_t)row * P + i] = v;
    }
}

__global__ void k_cube_to_free(const double* __restrict__ cube, int d, int P,
                               const int* __restrict__ kind, const double* __restrict__ pa,
                               const double* __restrict__ pb, const int* __restrict__ free_of_full,
                               double* __restrict__ theta, int B, int f32) {
    const int row = blockIdx.x;
    if (row >= B) return;
    for (int i = threadIdx.x; i < P; i += blockDim.x) {
        const int f = free_of_full[i];
        if (f < 0) continue;
        const double c = cube[(size_t)row * d + f];
        theta[(size_t)row * d + f] = (kind[i] == NS_PRIOR_UNIFORM) ? pa[i] + (pb[i] - pa[i]) * c
                                                                   : pa[i] + pb[i] * gauss_quantile(c, f32 != 0);
    }
}

__global__ void k_free_to_full(const double* __restrict__ theta, int d, int P,
                               const double* __restrict__ pa, const int* __restrict__ free_of_full,
                               double* __restrict__ theta_full, int B) {
    const int row = blockIdx.x;
    if (row >= B) return;
    for (int i = threadIdx.x; i < P; i += blockDim.x) {
        const int f = free_of_full[i];
        theta_full[(size_t)row * P + i] = (f < 0) ? pa[i] : theta[(size_t)row * d + f];
    }
}

// ------------------------------------------------------------ gauss test
__global__ void k_gauss_loglike(const double* __restrict__ theta_full, int P, double mu, double sigma,
                                double* __restrict__ logL, const int* __restrict__ nrows) {
    const int row = blockIdx.x * blockDim.x + threadIdx.x;
    if (row >= *nrows) return;
    double s = 0.0;
    for (int i = 0; i < P; ++i) {
        const double r = (theta_full[(size_t)row * P + i] - mu) / sigma;
        s += r * r;
    }
    logL[row] = -0.5 * s - P * log(sigma * 2.5066282746310005024);
}

// ------------------------------------------------------------ emulator
// Hidden-layer activation: tanh, or CosmoPower's sigmoid-linear
// f(x) = [g + (1 - g) sigmoid(beta x)] x with one (g, beta) per unit.
template <typename T> __device__ inline T act_tanh(T x);
template <> __device__ inline double act_tanh<double>(double x) { return tanh(x); }
template <> __device__ inline float act_tanh<float>(float x) { return tanhf(x); }
template <typename T> __device__ inline T ex_acc(T x);
template <> __device__ inline double ex_acc<double>(double x) { return exp(x); }
template <> __device__ inline float ex_acc<float>(float x) { return expf(x); }

template <typename T>
struct ActDev {
    int kind;
    const T* g;
    const T* beta;
};

template <typename T>
__device__ __forceinline__ T act_apply(const ActDev<T>& a, int n, T x) {
    if (a.kind == NS_ACT_TANH) return act_tanh<T>(x);
    const T g = a.g[n];
    return (g + (T(1) - g) / (T(1) + ex_acc<T>(-a.beta[n] * x))) * x;
}

template <typename TO, typename T> __device__ inline TO cvt_out(T v) { return (TO)v; }
template <> __device__ inline __nv_bfloat16 cvt_out<__nv_bfloat16, float>(float v) { return __float2bfloat16_rn(v); }

template <typename T> __device__ inline T cvt_in(T v) { return v; }
__device__ inline float cvt_in(__nv_bfloat16 v) { return __bfloat162float(v); }

// Input layer: h = act(W0 x + b0), x = (theta[inputs] - center) / scale.  A
// CTA takes kInRows consecutive rows; thread t owns units t, t + blockDim, ...
// and keeps a unit's bias and K0 (<= KMAX) weights in registers over the CTA's
// rows, so the weights are read once per CTA and the launch has
// ceil(rows / kInRows) CTAs rather than one per (row, 256 units).
constexpr int kInRows = 2;
template <typename T, typename TO, int KMAX>
__global__ void __launch_bounds__(256)
k_emu_input(const double* __restrict__ theta_full, int P, const int* __restrict__ inputs,
            const double* __restrict__ center, const double* __restrict__ scale,
            const double* __restrict__ inv_scale, int K0,
            const T* __restrict__ W0, const T* __restrict__ b0, ActDev<T> act, int N,
            TO* __restrict__ out, const int* __restrict__ nrows) {
    // the weights of a thread's first UP units are problem constants: in
    // registers before the dependency wait
    constexpr int UP = KMAX <= 8 ? 4 : 1;
    T wp[UP][KMAX], bp[UP];
#pragma unroll
    for (int u = 0; u < UP; ++u) {
        const int n = threadIdx.x + u * blockDim.x;
#pragma unroll
        for (int j = 0; j < KMAX; ++j) wp[u][j] = (n < N && j < K0) ? W0[(size_t)n * K0 + j] : T(0);
        bp[u] = n < N ? b0[n] : T(0);
    }
    pdl_begin();
    const int M = *nrows;
    const int r0 = blockIdx.x * kInRows;
    if (r0 >= M) return;
    const int nr = min(kInRows, M - r0);
    __shared__ T x[kInRows][KMAX];
    for (int i = threadIdx.x; i < nr * K0; i += blockDim.x) {
        const int r = i / K0, j = i - r * K0;
        // FP64 standardisation; reduced-precision emulators multiply by the
        // reciprocal scale (an FP64 divide is a long sequence on GB300's FP64 pipe)
        const double v = theta_full[(size_t)(r0 + r) * P + inputs[j]] - center[j];
        x[r][j] = sizeof(T) == 8 ? (T)(v / scale[j]) : (T)(v * inv_scale[j]);
    }
    __syncthreads();
    auto unit = [&](int n, const T (&w)[KMAX], T bn) {
        for (int r = 0; r < nr; ++r) {
            T acc = bn;
#pragma unroll
            for (int j = 0; j < KMAX; ++j)
                if (j < K0) acc = fma(w[j], x[r][j], acc);
            out[(size_t)(r0 + r) * N + n] = cvt_out<TO, T>(act_apply<T>(act, n, acc));
        }
    };
#pragma unroll
    for (int u = 0; u < UP; ++u) {
        const int n = threadIdx.x + u * blockDim.x;
        if (n < N) unit(n, wp[u], bp[u]);
    }
    for (int n = threadIdx.x + UP * blockDim.x; n < N; n += blockDim.x) {
        T w[KMAX];
#pragma unroll
        for (int j = 0; j < KMAX; ++j) w[j] = j < K0 ? W0[(size_t)n * K0 + j] : T(0);
        unit(n, w, b0[n]);
    }
}

// C[M x N] = epi(A[M x K] W[N x K]^T + b).  Threads own an interleaved
// TM x TN sub-tile (rows ty + i*BM/TM, cols tx + j*BN/TN) so shared-memory
// reads and global stores are conflict-free / coalesced.  A may be stored in
// a narrower type (bf16 activations) and is widened on load.
//   EPI_ACT: act(acc + b);  EPI_OUT: mu + s (acc + b), s = sig_vec[n] or sigma.
enum { EPI_ACT = 0, EPI_OUT = 1 };

template <typename T, typename TA, int BM, int BN, int BK, int TM, int TN, int EPI>
__global__ void __launch_bounds__((BM / TM) * (BN / TN))
k_gemm_simt(const TA* __restrict__ A, const T* __restrict__ W, const T* __restrict__ bias, ActDev<T> act,
            const T* __restrict__ out_mu, const T* __restrict__ sig_vec, T out_sigma, T* __restrict__ C,
            const int* __restrict__ nrows, int N, int K) {
    constexpr int TX = BN / TN, TY = BM / TM, NT = TX * TY;
    const int M = *nrows;
    const int m0 = blockIdx.y * BM, n0 = blockIdx.x * BN;
    if (m0 >= M) return;
    __shared__ T As[BK][BM + 1];
    __shared__ T Bs[BK][BN + 1];
    const int tid = threadIdx.x, tx = tid % TX, ty = tid / TX;
    T acc[TM][TN];
#pragma unroll
    for (int i = 0; i < TM; ++i)
#pragma unroll
        for (int j = 0; j < TN; ++j) acc[i][j] = T(0);
    for (int k0 = 0; k0 < K; k0 += BK) {
        for (int i = tid; i < BM * BK; i += NT) {
            const int r = i / BK, c = i % BK;
            const int gm = m0 + r, gk = k0 + c;
            As[c][r] = (gm < M && gk < K) ? (T)cvt_in(A[(size_t)gm * K + gk]) : T(0);
        }
        for (int i = tid; i < BN * BK; i += NT) {
            const int r = i / BK, c = i % BK;
            const int gn = n0 + r, gk = k0 + c;
            Bs[c][r] = (gn < N && gk < K) ? W[(size_t)gn * K + gk] : T(0);
        }
        __syncthreads();
#pragma unroll
        for (int kk = 0; kk < BK; ++kk) {
            T a[TM], b[TN];
#pragma unroll
            for (int i = 0; i < TM; ++i) a[i] = As[kk][ty + i * TY];
#pragma unroll
            for (int j = 0; j < TN; ++j) b[j] = Bs[kk][tx + j * TX];
#pragma unroll
            for (int i = 0; i < TM; ++i)
#pragma unroll
                for (int j = 0; j < TN; ++j) acc[i][j] = fma(a[i], b[j], acc[i][j]);
        }
        __syncthreads();
    }
#pragma unroll
    for (int i = 0; i < TM; ++i) {
        const int gm = m0 + ty + i * TY;
        if (gm >= M) continue;
#pragma unroll
        for (int j = 0; j < TN; ++j) {
            const int gn = n0 + tx + j * TX;
            if (gn >= N) continue;
            T v = acc[i][j] + (bias ? bias[gn] : T(0));
            if (EPI == EPI_ACT) v = act_apply<T>(act, gn, v);
            else v = out_mu[gn] + (sig_vec ? sig_vec[gn] : out_sigma) * v;
            C[(size_t)gm * N + gn] = v;
        }
    }
}

// Coarse-z emulator table -> n_z table: out[jz][ik] = sum_q w[jz][q] in[row[jz][q]][ik]
// (Catmull-Rom in z with folded ghosts).
template <typename T>
__global__ void k_zinterp(const T* __restrict__ coarse, int nzc, const int* __restrict__ zr,
                          const double* __restrict__ zwt, T* __restrict__ fine, int nz, int nk,
                          const int* __restrict__ nrows) {
    const int row = blockIdx.y;
    if (row >= *nrows) return;
    const T* c = coarse + (size_t)row * nzc * nk;
    T* f = fine + (size_t)row * nz * nk;
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < nz * nk; i += gridDim.x * blockDim.x) {
        const int jz = i / nk, ik = i % nk;
        T v = T(0);
#pragma unroll
        for (int q = 0; q < 4; ++q) v += (T)zwt[jz * 4 + q] * c[zr[jz * 4 + q] * nk + ik];
        f[i] = v;
    }
}

template <typename T, typename TA>
struct SimtTile;
template <typename TA> struct SimtTile<double, TA> { static constexpr int BM = 64, BN = 64, BK = 8, TM = 4, TN = 4; };
template <typename TA> struct SimtTile<float, TA> { static constexpr int BM = 128, BN = 128, BK = 8, TM = 8, TN = 8; };

template <typename T, typename TA>
int launch_gemm_simt(const TA* A, const T* W, const T* bias, ActDev<T> act, const T* mu, const T* sig_vec, T sigma,
                     T* C, const int* nrows, int grid_rows, int N, int K, int epi, cudaStream_t st) {
    using S = SimtTile<T, TA>;
    constexpr int NT = (S::BM / S::TM) * (S::BN / S::TN);
    dim3 grid((N + S::BN - 1) / S::BN, (grid_rows + S::BM - 1) / S::BM);
    if (epi == EPI_ACT)
        k_gemm_simt<T, TA, S::BM, S::BN, S::BK, S::TM, S::TN, EPI_ACT><<<grid, NT, 0, st>>>(
            A, W, bias, act, mu, sig_vec, sigma, C, nrows, N, K);
    else
        k_gemm_simt<T, TA, S::BM, S::BN, S::BK, S::TM, S::TN, EPI_OUT><<<grid, NT, 0, st>>>(
            A, W, bias, act, mu, sig_vec, sigma, C, nrows, N, K);
    NS_CUDA_TRY(cudaGetLastError());
    return NS_OK;
}

// Plain FP64 GEMM C = A W^T (M x N, K inner) on the device, for set-up work
// (the CMB whitening fold); nrows_dev holds M.
int gemm_f64_plain(const double* A, const double* W, double* C, const int* nrows_dev, int M, int N, int K,
                   const double* zeros_n, cudaStream_t st) {
    return launch_gemm_simt<double, double>(A, W, zeros_n, ActDev<double>{0, nullptr, nullptr}, zeros_n, nullptr,
                                            1.0, C, nrows_dev, M, N, K, EPI_OUT, st);
}

int launch_cube_to_theta(const ns_problem* p, Workspace* ws, const double* cube, int grid_rows,
                         cudaStream_t st) {
    if (grid_rows <= 0) return NS_OK;
    NS_CUDA_TRY(launch_pdl(k_cube_to_theta, dim3(grid_rows), dim3(64), 0, st, cube, p->d, p->P,
                           (const int*)p->d_pkind, (const double*)p->d_pa, (const double*)p->d_pb,
                           (const int*)p->d_free_of_full, ws->theta_full, (const int*)ws->d_nrows));
    return NS_OK;
}

template <typename T>
static ActDev<T> layer_act(const ns_problem* p, int l) {
    ActDev<T> a{p->act, nullptr, nullptr};
    if (p->act == NS_ACT_SIGMOID_LINEAR) {
        a.g = (const T*)p->d_act_g[l];
        a.beta = (const T*)p->d_act_beta[l];
    }
    return a;
}

template <typename T, typename TO>
static int launch_emu_input(const ns_problem* p, const Workspace* ws, int grid_rows, TO* out, bool pdl,
                            cudaStream_t st) {
    const int K0 = p->dims[0], H1 = p->dims[1];
    const dim3 g((grid_rows + kInRows - 1) / kInRows);
    auto kern = K0 <= 8 ? k_emu_input<T, TO, 8> : k_emu_input<T, TO, 32>;
    if (pdl) {
        NS_CUDA_TRY(launch_pdl(kern, g, dim3(256), 0, st, (const double*)ws->theta_full, p->P,
                               (const int*)p->d_inputs, (const double*)p->d_in_center, (const double*)p->d_in_scale,
                               (const double*)p->d_in_inv_scale, K0, (const T*)p->d_W[0], (const T*)p->d_b[0],
                               layer_act<T>(p, 0), H1, out, (const int*)ws->d_nrows));
    } else {
        kern<<<g, 256, 0, st>>>(ws->theta_full, p->P, p->d_inputs, p->d_in_center, p->d_in_scale,
                                p->d_in_inv_scale, K0, (const T*)p->d_W[0], (const T*)p->d_b[0], layer_act<T>(p, 0),
                                H1, out, ws->d_nrows);
        NS_CUDA_TRY(cudaGetLastError());
    }
    return NS_OK;
}

// The emulator's last layer: W h + b, de-standardised as mu + s * (.), written to out.
struct Head {
    const void* W;
    const void* bias;
    const void* mu;
    const void* sig_vec;
    double sigma;
    void* out;
    int n_out = 0;           // outputs computed (the first rows of W); 0: all
};

static Head model_head(const ns_problem* p, void* out) {
    const int L = p->n_layers;
    return Head{p->d_W[L - 1], p->d_b[L - 1], p->d_out_mu, p->d_out_sig, p->out_sigma, out};
}

template <typename T>
static int run_emulator_simt(const ns_problem* p, Workspace* ws, int grid_rows, cudaStream_t st, const Head& hd) {
    const int L = p->n_layers;
    NS_TRY((launch_emu_input<T, T>(p, ws, grid_rows, (T*)ws->act[0], false, st)));
    int cur = 0;
    for (int l = 1; l < L; ++l) {
        const int K = p->dims[l], N = p->dims[l + 1];
        if (l == L - 1) {
            NS_TRY((launch_gemm_simt<T, T>((const T*)ws->act[cur], (const T*)hd.W, (const T*)hd.bias, ActDev<T>{0, nullptr, nullptr},
                                           (const T*)hd.mu, (const T*)hd.sig_vec, (T)hd.sigma, (T*)hd.out,
                                           ws->d_nrows, grid_rows, hd.n_out ? hd.n_out : N, K, EPI_OUT, st)));
        } else {
            NS_TRY((launch_gemm_simt<T, T>((const T*)ws->act[cur], (const T*)p->d_W[l], (const T*)p->d_b[l],
                                           layer_act<T>(p, l), nullptr, nullptr, T(0), (T*)ws->act[cur ^ 1],
                                           ws->d_nrows, grid_rows, N, K, EPI_ACT, st)));
        }
        cur ^= 1;
    }
    return NS_OK;
}

static int probe_begin(const StageProbe* pr, int stage, Workspace* ws, cudaStream_t st) {
    if (!pr || pr->stage != stage) return NS_OK;
    NS_CUDA_TRY(cudaMemcpyAsync(pr->h_rows, ws->d_nrows, sizeof(int), cudaMemcpyDeviceToHost, st));
    NS_CUDA_TRY(cudaEventRecordWithFlags(pr->ev0, st, cudaEventRecordExternal));
    return NS_OK;
}
static int probe_end(const StageProbe* pr, int stage, cudaStream_t st) {
    if (!pr || pr->stage != stage) return NS_OK;
    NS_CUDA_TRY(cudaEventRecordWithFlags(pr->ev1, st, cudaEventRecordExternal));
    return NS_OK;
}

// BF16: input layer on CUDA cores, hidden layers as tcgen05 GEMMs with the
// activation in the epilogue.  The last layer: for the shear kind a tcgen05
// GEMM with the de-standardising epilogue into the FP32 table; for the CMB
// kind `hd` on CUDA cores in FP32 (the folded head needs FP32 weights).
static int run_emulator_bf16(const ns_problem* p, Workspace* ws, int grid_rows, cudaStream_t st,
                             const StageProbe* probe, const Head* hd) {
    const int L = p->n_layers;
    int cur = 0, l1 = 1;
    if (p->fused_cs) {
        // input and hidden layers in one clustered kernel; its output is the
        // buffer the per-layer path would leave the last hidden layer in
        NS_TRY(probe_begin(probe, PROBE_EMU_HIDDEN, ws, st));
        NS_TRY(launch_emu_fused(p, ws, grid_rows, st));
        NS_TRY(probe_end(probe, PROBE_EMU_HIDDEN, st));
        cur = (L - 2) & 1;
        l1 = L - 1;
    } else {
        NS_TRY((launch_emu_input<float, __nv_bfloat16>(p, ws, grid_rows, (__nv_bfloat16*)ws->act[0], true, st)));
    }
    for (int l = l1; l < L; ++l) {
        const int K = p->dims[l], N = p->dims[l + 1];
        const bool last = (l == L - 1);
        const int stage = last ? PROBE_EMU_OUT : (l == 1 ? PROBE_EMU_HIDDEN : PROBE_NONE);
        NS_TRY(probe_begin(probe, stage, ws, st));
        if (last && hd) {
            NS_TRY((launch_gemm_simt<float, __nv_bfloat16>(
                (const __nv_bfloat16*)ws->act[cur], (const float*)hd->W, (const float*)hd->bias,
                ActDev<float>{0, nullptr, nullptr}, (const float*)hd->mu, (const float*)hd->sig_vec,
                (float)hd->sigma, (float*)hd->out, ws->d_nrows, grid_rows, hd->n_out ? hd->n_out : N, K, EPI_OUT,
                st)));
        } else if (last && p->tile_n[l] == 128) {
            // the output layer with few rows: features as the MMA's M (one wave of CTAs)
            NS_TRY(launch_gemm_tc_out_swap(&p->tmB[l], &ws->tmX_out, (const float*)p->d_b[l],
                                           (const float*)p->d_out_mu, (float)p->out_sigma, (float*)ws->table,
                                           ws->d_nrows, grid_rows, N, K, ws->d_err, st));
        } else {
            const ActDev<float> a = layer_act<float>(p, l);
            const int epi = last ? TC_EPI_OUT : (p->act == NS_ACT_SIGMOID_LINEAR ? TC_EPI_SIGLIN : TC_EPI_TANH);
            NS_TRY(launch_gemm_tc(&ws->tmA[l], &p->tmB[l], p->tile_n[l], (const float*)p->d_b[l],
                                  last ? (const float*)p->d_out_mu : a.g, last ? (float)p->out_sigma : 0.f,
                                  last ? ws->table : ws->act[cur ^ 1], ws->d_nrows, grid_rows, N, K, epi,
                                  last ? nullptr : a.beta, ws->d_err, st));
        }
        NS_TRY(probe_end(probe, stage, st));
        cur ^= 1;
    }
    return NS_OK;
}

template <typename T>
__global__ void k_to_double(const T* __restrict__ in, double* __restrict__ out, int n_per_row,
                            const int* __restrict__ nrows) {
    const int row = blockIdx.y;
    if (row >= *nrows) return;
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < n_per_row; i += gridDim.x * blockDim.x)
        out[(size_t)row * n_per_row + i] = (double)in[(size_t)row * n_per_row + i];
}

// chi^2 = sum_a y_a^2 per row (fixed-order block tree, partials widened to
// FP64), log L = c0 - chi^2 / 2 in FP64.
template <typename T>
__global__ void __launch_bounds__(256) k_rowsq(const T* __restrict__ y, int D, double c0, double* __restrict__ logL,
                                               const int* __restrict__ nrows) {
    const int row = blockIdx.x;
    if (row >= *nrows) return;
    __shared__ double part[256];
    const T* yr = y + (size_t)row * D;
    T s = T(0);
    for (int a = threadIdx.x; a < D; a += 256) s = fma(yr[a], yr[a], s);
    part[threadIdx.x] = (double)s;
    __syncthreads();
    for (int o = 128; o > 0; o >>= 1) {
        if (threadIdx.x < o) part[threadIdx.x] += part[threadIdx.x + o];
        __syncthreads();
    }
    if (threadIdx.x == 0) logL[row] = c0 - 0.5 * part[0];
}

// Cosmic-variance TT log L per row: c0 - sum_ell (k/2) g(C_ell / d_ell) with
// g(r) = ln r + 1/r - 1 = log1p(u) - u / (1 + u), u = r - 1 (no cancellation
// near the peak); partial sums widened to FP64 in a fixed-order block tree.
template <typename T>
__global__ void __launch_bounds__(256) k_cmb_tt(const T* __restrict__ C, int n_tt, int ld, const T* __restrict__ dobs,
                                                const T* __restrict__ halfk, double c0, double* __restrict__ logL,
                                                const int* __restrict__ nrows) {
    const int row = blockIdx.x;
    if (row >= *nrows) return;
    __shared__ double part[256];
    const T* c = C + (size_t)row * ld;
    T s = T(0);
    for (int i = threadIdx.x; i < n_tt; i += 256) {
        const T u = c[i] / dobs[i] - T(1);
        s += halfk[i] * (log1p(u) - u / (T(1) + u));
    }
    part[threadIdx.x] = (double)s;
    __syncthreads();
    for (int o = 128; o > 0; o >>= 1) {
        if (threadIdx.x < o) part[threadIdx.x] += part[threadIdx.x + o];
        __syncthreads();
    }
    if (threadIdx.x == 0) logL[row] = c0 - part[0];
}

int run_emulator_only(const ns_problem* p, Workspace* ws, int grid_rows, double* out, cudaStream_t st) {
    if (grid_rows <= 0) return NS_OK;
    const int n_out = p->dims.back();
    dim3 g((n_out + 255) / 256, grid_rows);
    const Head hd = model_head(p, ws->table);
    if (p->precision == NS_PREC_FP64) {
        NS_TRY(run_emulator_simt<double>(p, ws, grid_rows, st, hd));
        k_to_double<double><<<g, 256, 0, st>>>((const double*)ws->table, out, n_out, ws->d_nrows);
    } else {
        if (p->precision == NS_PREC_FP32) NS_TRY(run_emulator_simt<float>(p, ws, grid_rows, st, hd));
        else NS_TRY(run_emulator_bf16(p, ws, grid_rows, st, nullptr, p->kind == NS_KIND_CMB ? &hd : nullptr));
        k_to_double<float><<<g, 256, 0, st>>>((const float*)ws->table, out, n_out, ws->d_nrows);
    }
    NS_CUDA_TRY(cudaGetLastError());
    return NS_OK;
}

// CMB kind (Sec. 3.1 problem, dense covariance): FOLD runs the hidden layers
// and the folded head y = c' - W' h, then chi^2 = |y|^2; LITERAL (FP64) forms
// r = (d - mu) - sigma (W h + b) with the same head kernel and whitens it by
// L^-1; model_out gets the de-standardised emulator output.
static int run_cmb(const ns_problem* p, Workspace* ws, int grid_rows, double* logL_out, double* model_out,
                   cudaStream_t st, const StageProbe* probe) {
    const int D = p->D;
    if (model_out) return run_emulator_only(p, ws, grid_rows, model_out, st);
    const bool f64 = p->precision == NS_PREC_FP64;
    if (p->cmb_form == NS_CMB_TT_CV) {
        // the TT block of the head only (the first n_tt outputs), then the sums
        Head hd = model_head(p, ws->table);
        hd.n_out = p->n_tt;
        if (f64) NS_TRY(run_emulator_simt<double>(p, ws, grid_rows, st, hd));
        else if (p->precision == NS_PREC_FP32) NS_TRY(run_emulator_simt<float>(p, ws, grid_rows, st, hd));
        else NS_TRY(run_emulator_bf16(p, ws, grid_rows, st, probe, &hd));
        NS_TRY(probe_begin(probe, PROBE_CHI2, ws, st));
        if (f64)
            k_cmb_tt<double><<<grid_rows, 256, 0, st>>>((const double*)ws->table, p->n_tt, p->n_tt,
                                                        (const double*)p->d_tt_obs, (const double*)p->d_tt_halfk,
                                                        p->c0, logL_out, ws->d_nrows);
        else
            k_cmb_tt<float><<<grid_rows, 256, 0, st>>>((const float*)ws->table, p->n_tt, p->n_tt,
                                                       (const float*)p->d_tt_obs, (const float*)p->d_tt_halfk,
                                                       p->c0, logL_out, ws->d_nrows);
        NS_CUDA_TRY(cudaGetLastError());
        return probe_end(probe, PROBE_CHI2, st);
    }
    if (p->cmb_solve == NS_SOLVE_LITERAL) {
        const int L = p->n_layers;
        const Head hd{p->d_W[L - 1], p->d_b[L - 1], p->d_lit_mu, p->d_lit_sig, 0.0, ws->resid};
        NS_TRY(run_emulator_simt<double>(p, ws, grid_rows, st, hd));
        NS_TRY(probe_begin(probe, PROBE_CHI2, ws, st));
        NS_TRY((launch_chi2<double, double>((const double*)ws->resid, D, p->d_LinvT64, p->c0, logL_out,
                                            ws->d_nrows, grid_rows, st)));
        return probe_end(probe, PROBE_CHI2, st);
    }
    const Head hd{p->d_Wfold, p->d_zeroD, p->d_cfold, nullptr, -1.0, ws->table};
    if (f64) NS_TRY(run_emulator_simt<double>(p, ws, grid_rows, st, hd));
    else if (p->precision == NS_PREC_FP32) NS_TRY(run_emulator_simt<float>(p, ws, grid_rows, st, hd));
    else NS_TRY(run_emulator_bf16(p, ws, grid_rows, st, probe, &hd));
    NS_TRY(probe_begin(probe, PROBE_CHI2, ws, st));
    if (f64) k_rowsq<double><<<grid_rows, 256, 0, st>>>((const double*)ws->table, D, p->c0, logL_out, ws->d_nrows);
    else k_rowsq<float><<<grid_rows, 256, 0, st>>>((const float*)ws->table, D, p->c0, logL_out, ws->d_nrows);
    NS_CUDA_TRY(cudaGetLastError());
    return probe_end(probe, PROBE_CHI2, st);
}

int run_likelihood(const ns_problem* p, Workspace* ws, int grid_rows, double* logL_out, double* model_out,
                   cudaStream_t st, const StageProbe* probe) {
    if (grid_rows <= 0) return NS_OK;
    if (p->kind == NS_KIND_GAUSS) {
        k_gauss_loglike<<<(grid_rows + 127) / 128, 128, 0, st>>>(ws->theta_full, p->P, p->g_mu, p->g_sigma,
                                                                 logL_out, ws->d_nrows);
        NS_CUDA_TRY(cudaGetLastError());
        return NS_OK;
    }
    if (p->kind == NS_KIND_CMB) return run_cmb(p, ws, grid_rows, logL_out, model_out, st, probe);
    const ShearParams& sp = p->sp;
    const bool coarse = p->n_z_emu != sp.n_z;
    const bool f64 = p->precision == NS_PREC_FP64;
    // fork: the windows stage needs only theta, so it runs on the side stream
    // while the emulator runs on `st`; the Limber stage joins both.
    NS_CUDA_TRY(cudaEventRecord(ws->ev_fork, st));
    NS_CUDA_TRY(cudaStreamWaitEvent(ws->side, ws->ev_fork, 0));
    NS_TRY(probe_begin(probe, PROBE_WINDOWS, ws, ws->side));
    if (f64) NS_TRY(launch_windows<double, false>(sp, ws->theta_full, (double*)ws->win, ws->d_nrows, grid_rows, ws->side));
    else if (p->precision == NS_PREC_FP32)
        NS_TRY(launch_windows<float, false>(sp, ws->theta_full, (float*)ws->win, ws->d_nrows, grid_rows, ws->side));
    else NS_TRY(launch_windows<float, true>(sp, ws->theta_full, (float*)ws->win, ws->d_nrows, grid_rows, ws->side));
    NS_TRY(probe_end(probe, PROBE_WINDOWS, ws->side));
    NS_CUDA_TRY(cudaEventRecord(ws->ev_join, ws->side));
    if (f64) {
        NS_TRY(run_emulator_simt<double>(p, ws, grid_rows, st, model_head(p, ws->table)));
        const double* tab = (const double*)ws->table;
        if (coarse) {
            dim3 g((sp.n_z * sp.n_k + 255) / 256, grid_rows);
            k_zinterp<double><<<g, 256, 0, st>>>(tab, p->n_z_emu, p->d_zi_row, p->d_zi_w,
                                                 (double*)ws->table_fine, sp.n_z, sp.n_k, ws->d_nrows);
            NS_CUDA_TRY(cudaGetLastError());
            tab = (const double*)ws->table_fine;
        }
        NS_CUDA_TRY(cudaStreamWaitEvent(st, ws->ev_join, 0));
        NS_TRY(launch_limber<double, false>(sp, ws->theta_full, tab, (const double*)ws->win, (double*)ws->resid,
                                            model_out, ws->d_nrows, grid_rows, ws->d_err, st));
        if (model_out) return NS_OK;
        return launch_chi2<double, double>((const double*)ws->resid, sp.D, p->d_LinvT64, p->c0, logL_out,
                                           ws->d_nrows, grid_rows, st, true);
    }
    // FP32 stages (FP32 / BF16 / BF16_F64CHI2)
    if (p->precision == NS_PREC_FP32) NS_TRY(run_emulator_simt<float>(p, ws, grid_rows, st, model_head(p, ws->table)));
    else NS_TRY(run_emulator_bf16(p, ws, grid_rows, st, probe, nullptr));
    const float* tab = (const float*)ws->table;
    if (coarse) {
        dim3 g((sp.n_z * sp.n_k + 255) / 256, grid_rows);
        k_zinterp<float><<<g, 256, 0, st>>>(tab, p->n_z_emu, p->d_zi_row, p->d_zi_w, (float*)ws->table_fine,
                                            sp.n_z, sp.n_k, ws->d_nrows);
        NS_CUDA_TRY(cudaGetLastError());
        tab = (const float*)ws->table_fine;
    }
    NS_CUDA_TRY(cudaStreamWaitEvent(st, ws->ev_join, 0));
    NS_TRY(probe_begin(probe, PROBE_PROJECTION, ws, st));
    if (p->precision == NS_PREC_FP32)
        NS_TRY(launch_limber<float, false>(sp, ws->theta_full, tab, (const float*)ws->win, (float*)ws->resid,
                                           model_out, ws->d_nrows, grid_rows, ws->d_err, st));
    else
        NS_TRY(launch_limber<float, true>(sp, ws->theta_full, tab, (const float*)ws->win, (float*)ws->resid,
                                          model_out, ws->d_nrows, grid_rows, ws->d_err, st));
    NS_TRY(probe_end(probe, PROBE_PROJECTION, st));
    if (model_out) return NS_OK;
    NS_TRY(probe_begin(probe, PROBE_CHI2, ws, st));
    if (p->precision == NS_PREC_BF16_F64CHI2)
        NS_TRY(launch_chi2<float, double>((const float*)ws->resid, sp.D, p->d_LinvT64, p->c0, logL_out,
                                          ws->d_nrows, grid_rows, st, true));
    else
        NS_TRY(launch_chi2<float, float>((const float*)ws->resid, sp.D, p->d_LinvT32, p->c0, logL_out,
                                         ws->d_nrows, grid_rows, st, true));
    return probe_end(probe, PROBE_CHI2, st);
}

}  // namespace gpuns

// host helpers used by the C API in problem.cu
namespace gpuns {
int launch_cube_to_free(const ns_problem* p, const double* cube, int B, double* theta, cudaStream_t st) {
    // the sampler's prior transform: FP32 quantile for reduced-precision problems
    k_cube_to_free<<<B, 64, 0, st>>>(cube, p->d, p->P, p->d_pkind, p->d_pa, p->d_pb, p->d_free_of_full, theta, B,
                                     p->precision != NS_PREC_FP64 ? 1 : 0);
    NS_CUDA_TRY(cudaGetLastError());
    return NS_OK;
}
int launch_free_to_full(const ns_problem* p, const double* theta, int B, double* theta_full, cudaStream_t st) {
    k_free_to_full<<<B, 64, 0, st>>>(theta, p->d, p->P, p->d_pa, p->d_free_of_full, theta_full, B);
    NS_CUDA_TRY(cudaGetLastError());
    return NS_OK;
}
}  // namespace gpuns

namespace gpuns {
int launch_zinterp_generic(const ns_problem* p, const void* coarse, void* fine, const int* nrows, int grid_rows, int elt,
                           cudaStream_t st) {
    const ShearParams& sp = p->sp;
    dim3 g((sp.n_z * sp.n_k + 255) / 256, grid_rows);
    if (elt == 8)
        k_zinterp<double><<<g, 256, 0, st>>>((const double*)coarse, p->n_z_emu, p->d_zi_row, p->d_zi_w, (double*)fine,
                                             sp.n_z, sp.n_k, nrows);
    else
        k_zinterp<float><<<g, 256, 0, st>>>((const float*)coarse, p->n_z_emu, p->d_zi_row, p->d_zi_w, (float*)fine,
                                            sp.n_z, sp.n_k, nrows);
    NS_CUDA_TRY(cudaGetLastError());
    return NS_OK;
}
int launch_free_to_full_ext(const ns_problem* p, const double* theta, int B, double* theta_full, cudaStream_t st) {
    return launch_free_to_full(p, theta, B, theta_full, st);
}
}  // namespace gpuns
