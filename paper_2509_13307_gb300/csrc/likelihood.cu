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

__global__ void k_set_int(int* p, int v) { *p = v; }

__constant__ double c_glx[4] = {-0.86113631159405257522, -0.33998104358485626480,
                                 0.33998104358485626480, 0.86113631159405257522};
__constant__ double c_glw[4] = {0.34785484513745385737, 0.65214515486254614263,
                                 0.65214515486254614263, 0.34785484513745385737};

// ------------------------------------------------------------ prior transform
__global__ void k_cube_to_theta(const double* __restrict__ cube, int d, int P,
                                const int* __restrict__ kind, const double* __restrict__ pa,
                                const double* __restrict__ pb, const int* __restrict__ free_of_full,
                                double* __restrict__ theta_full, const int* __restrict__ nrows) {
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
                               double* __restrict__ theta, int B) {
    const int row = blockIdx.x;
    if (row >= B) return;
    for (int i = threadIdx.x; i < P; i += blockDim.x) {
        const int f = free_of_full[i];
        if (f < 0) continue;
        const double c = cube[(size_t)row * d + f];
        theta[(size_t)row * d + f] = (kind[i] == NS_PRIOR_UNIFORM) ? pa[i] + (pb[i] - pa[i]) * c
                                                                   : pa[i] + pb[i] * normcdfinv(c);
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
template <typename T> __device__ inline T act_tanh(T x);
template <> __device__ inline double act_tanh<double>(double x) { return tanh(x); }
template <> __device__ inline float act_tanh<float>(float x) { return tanhf(x); }

template <typename TO> __device__ inline TO to_out(float v);
template <> __device__ inline float to_out<float>(float v) { return v; }
template <> __device__ inline __nv_bfloat16 to_out<__nv_bfloat16>(float v) { return __float2bfloat16_rn(v); }

// Input layer: h = tanh(W0 x + b0), x = (theta[inputs] - center) / scale.
template <typename T, typename TO>
__global__ void k_emu_input(const double* __restrict__ theta_full, int P, const int* __restrict__ inputs,
                            const double* __restrict__ center, const double* __restrict__ scale, int K0,
                            const T* __restrict__ W0, const T* __restrict__ b0, int N,
                            TO* __restrict__ out, const int* __restrict__ nrows) {
    const int row = blockIdx.y;
    if (row >= *nrows) return;
    __shared__ T x[32];
    if (threadIdx.x < K0) {
        const int j = threadIdx.x;
        x[j] = (T)((theta_full[(size_t)row * P + inputs[j]] - center[j]) / scale[j]);
    }
    __syncthreads();
    const int n = blockIdx.x * blockDim.x + threadIdx.x;
    if (n >= N) return;
    T acc = b0[n];
    for (int j = 0; j < K0; ++j) acc += W0[(size_t)n * K0 + j] * x[j];
    out[(size_t)row * N + n] = (TO)act_tanh<T>(acc);
}
template <>
__global__ void k_emu_input<float, __nv_bfloat16>(const double* __restrict__ theta_full, int P,
        const int* __restrict__ inputs, const double* __restrict__ center, const double* __restrict__ scale,
        int K0, const float* __restrict__ W0, const float* __restrict__ b0, int N,
        __nv_bfloat16* __restrict__ out, const int* __restrict__ nrows) {
    const int row = blockIdx.y;
    if (row >= *nrows) return;
    __shared__ float x[32];
    if (threadIdx.x < K0) {
        const int j = threadIdx.x;
        x[j] = (float)((theta_full[(size_t)row * P + inputs[j]] - center[j]) / scale[j]);
    }
    __syncthreads();
    const int n = blockIdx.x * blockDim.x + threadIdx.x;
    if (n >= N) return;
    float acc = b0[n];
    for (int j = 0; j < K0; ++j) acc = fmaf(W0[(size_t)n * K0 + j], x[j], acc);
    out[(size_t)row * N + n] = __float2bfloat16_rn(tanhf(acc));
}

enum { EPI_TANH = 0, EPI_OUT = 1 };

// C[M x N] = epi(A[M x K] W[N x K]^T + b).  Threads own an interleaved
// TM x TN sub-tile (rows ty + i*BM/TM, cols tx + j*BN/TN) so shared-memory
// reads and global stores are conflict-free / coalesced.
template <typename T, int BM, int BN, int BK, int TM, int TN, int EPI>
__global__ void __launch_bounds__((BM / TM) * (BN / TN))
k_gemm_simt(const T* __restrict__ A, const T* __restrict__ W, const T* __restrict__ bias,
            const T* __restrict__ out_mu, T out_sigma, T* __restrict__ C,
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
            As[c][r] = (gm < M && gk < K) ? A[(size_t)gm * K + gk] : T(0);
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
            T v = acc[i][j] + bias[gn];
            if (EPI == EPI_TANH) v = act_tanh<T>(v);
            else v = out_mu[gn] + out_sigma * v;
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

template <typename T>
static int launch_gemm_simt(const T* A, const T* W, const T* bias, const T* mu, T sigma, T* C,
                            const int* nrows, int grid_rows, int N, int K, int epi, cudaStream_t st);

template <>
int launch_gemm_simt<double>(const double* A, const double* W, const double* bias, const double* mu,
                             double sigma, double* C, const int* nrows, int grid_rows, int N, int K,
                             int epi, cudaStream_t st) {
    constexpr int BM = 64, BN = 64, BK = 8, TM = 4, TN = 4;
    dim3 grid((N + BN - 1) / BN, (grid_rows + BM - 1) / BM);
    if (epi == EPI_TANH)
        k_gemm_simt<double, BM, BN, BK, TM, TN, EPI_TANH><<<grid, 256, 0, st>>>(A, W, bias, mu, sigma, C, nrows, N, K);
    else
        k_gemm_simt<double, BM, BN, BK, TM, TN, EPI_OUT><<<grid, 256, 0, st>>>(A, W, bias, mu, sigma, C, nrows, N, K);
    NS_CUDA_TRY(cudaGetLastError());
    return NS_OK;
}

template <>
int launch_gemm_simt<float>(const float* A, const float* W, const float* bias, const float* mu, float sigma,
                            float* C, const int* nrows, int grid_rows, int N, int K, int epi,
                            cudaStream_t st) {
    constexpr int BM = 128, BN = 128, BK = 8, TM = 8, TN = 8;
    dim3 grid((N + BN - 1) / BN, (grid_rows + BM - 1) / BM);
    if (epi == EPI_TANH)
        k_gemm_simt<float, BM, BN, BK, TM, TN, EPI_TANH><<<grid, 256, 0, st>>>(A, W, bias, mu, sigma, C, nrows, N, K);
    else
        k_gemm_simt<float, BM, BN, BK, TM, TN, EPI_OUT><<<grid, 256, 0, st>>>(A, W, bias, mu, sigma, C, nrows, N, K);
    NS_CUDA_TRY(cudaGetLastError());
    return NS_OK;
}

int launch_cube_to_theta(const ns_problem* p, Workspace* ws, const double* cube, int grid_rows,
                         cudaStream_t st) {
    if (grid_rows <= 0) return NS_OK;
    k_cube_to_theta<<<grid_rows, 64, 0, st>>>(cube, p->d, p->P, p->d_pkind, p->d_pa, p->d_pb,
                                              p->d_free_of_full, ws->theta_full, ws->d_nrows);
    NS_CUDA_TRY(cudaGetLastError());
    return NS_OK;
}

template <typename T>
static int run_emulator_simt(const ns_problem* p, Workspace* ws, int grid_rows, cudaStream_t st) {
    const int L = p->n_layers;
    const int K0 = p->dims[0], H1 = p->dims[1];
    dim3 g0((H1 + 255) / 256, grid_rows);
    k_emu_input<T, T><<<g0, 256, 0, st>>>(ws->theta_full, p->P, p->d_inputs, p->d_in_center, p->d_in_scale,
                                          K0, (const T*)p->d_W[0], (const T*)p->d_b[0], H1, (T*)ws->act[0],
                                          ws->d_nrows);
    NS_CUDA_TRY(cudaGetLastError());
    int cur = 0;
    for (int l = 1; l < L; ++l) {
        const int K = p->dims[l], N = p->dims[l + 1];
        const bool last = (l == L - 1);
        T* out = last ? (T*)ws->table : (T*)ws->act[cur ^ 1];
        NS_TRY(launch_gemm_simt<T>((const T*)ws->act[cur], (const T*)p->d_W[l], (const T*)p->d_b[l],
                                   (const T*)p->d_out_mu, (T)p->out_sigma, out, ws->d_nrows, grid_rows, N, K,
                                   last ? EPI_OUT : EPI_TANH, st));
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

static int run_emulator_bf16(const ns_problem* p, Workspace* ws, int grid_rows, cudaStream_t st,
                             const StageProbe* probe = nullptr) {
    const int L = p->n_layers;
    const int K0 = p->dims[0], H1 = p->dims[1];
    dim3 g0((H1 + 255) / 256, grid_rows);
    k_emu_input<float, __nv_bfloat16><<<g0, 256, 0, st>>>(
        ws->theta_full, p->P, p->d_inputs, p->d_in_center, p->d_in_scale, K0, (const float*)p->d_W[0],
        (const float*)p->d_b[0], H1, (__nv_bfloat16*)ws->act[0], ws->d_nrows);
    NS_CUDA_TRY(cudaGetLastError());
    int cur = 0;
    for (int l = 1; l < L; ++l) {
        const int K = p->dims[l], N = p->dims[l + 1];
        const bool last = (l == L - 1);
        void* out = last ? ws->table : ws->act[cur ^ 1];
        const int stage = last ? PROBE_EMU_OUT : (l == 1 ? PROBE_EMU_HIDDEN : PROBE_NONE);
        NS_TRY(probe_begin(probe, stage, ws, st));
        NS_TRY(launch_gemm_tc(&ws->tmA[l], &p->tmB[l], p->tile_n[l], (const float*)p->d_b[l],
                              (const float*)p->d_out_mu, (float)p->out_sigma, out, ws->d_nrows, grid_rows,
                              N, K, last ? 1 : 0, ws->d_err, st));
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

int run_emulator_only(const ns_problem* p, Workspace* ws, int grid_rows, double* out, cudaStream_t st) {
    if (grid_rows <= 0) return NS_OK;
    const int n_out = p->dims.back();
    dim3 g((n_out + 255) / 256, grid_rows);
    if (p->precision == NS_PREC_FP64) {
        NS_TRY(run_emulator_simt<double>(p, ws, grid_rows, st));
        k_to_double<double><<<g, 256, 0, st>>>((const double*)ws->table, out, n_out, ws->d_nrows);
    } else {
        if (p->precision == NS_PREC_FP32) NS_TRY(run_emulator_simt<float>(p, ws, grid_rows, st));
        else NS_TRY(run_emulator_bf16(p, ws, grid_rows, st));
        k_to_double<float><<<g, 256, 0, st>>>((const float*)ws->table, out, n_out, ws->d_nrows);
    }
    NS_CUDA_TRY(cudaGetLastError());
    return NS_OK;
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
        NS_TRY(run_emulator_simt<double>(p, ws, grid_rows, st));
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
                                           ws->chi2_part, ws->chi2_done, ws->d_nrows, grid_rows, st);
    }
    // FP32 stages (FP32 / BF16 / BF16_F64CHI2)
    if (p->precision == NS_PREC_FP32) NS_TRY(run_emulator_simt<float>(p, ws, grid_rows, st));
    else NS_TRY(run_emulator_bf16(p, ws, grid_rows, st, probe));
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
                                          ws->chi2_part, ws->chi2_done, ws->d_nrows, grid_rows, st));
    else
        NS_TRY(launch_chi2<float, float>((const float*)ws->resid, sp.D, p->d_LinvT32, p->c0, logL_out,
                                         ws->chi2_part, ws->chi2_done, ws->d_nrows, grid_rows, st));
    return probe_end(probe, PROBE_CHI2, st);
}

}  // namespace gpuns

// host helpers used by the C API in problem.cu
namespace gpuns {
int launch_cube_to_free(const ns_problem* p, const double* cube, int B, double* theta, cudaStream_t st) {
    k_cube_to_free<<<B, 64, 0, st>>>(cube, p->d, p->P, p->d_pkind, p->d_pa, p->d_pb, p->d_free_of_full, theta, B);
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
