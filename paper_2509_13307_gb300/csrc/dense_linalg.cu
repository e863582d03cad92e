// Dense FP64 factorisation of a large data covariance on the device: blocked
// Cholesky C = L L^T and the explicit inverse factor L^-1.  Used at problem
// creation when D is too large for the host routine (the 7521 x 7521 CMB
// covariance); the per-evaluation whitening then reads L^-1 (or the fold
// built from it), so no triangular solve is left on the hot path.
//
// Cholesky, right-looking over 64-wide block columns j:
//   k_potrf_diag   factor the diagonal block in shared memory (one CTA);
//   k_trsm_panel   L_ij = A_ij L_jj^-T for every block row i > j;
//   k_syrk_update  A_ik -= L_ij L_kj^T for j < k <= i (lower tiles only).
// Inverse, left-looking over block rows i (X = L^-1 is lower triangular):
//   k_trinv_row    X_ic = L_ii^-1 (delta_ic I - sum_{k=c}^{i-1} L_ik X_kc), c <= i.
// Every sum runs in a fixed order, so the factors are reproducible.
#include <cmath>
#include <vector>

#include "likelihood.cuh"

namespace gpuns {

constexpr int kT = 64;     // tile edge
constexpr int kTP = kT + 1;

__device__ __forceinline__ void load_tile(double (*S)[kTP], const double* A, int D, int r0, int c0) {
    for (int q = threadIdx.x; q < kT * kT; q += blockDim.x) {
        const int r = q / kT, c = q % kT;
        S[r][c] = (r0 + r < D && c0 + c < D) ? A[(size_t)(r0 + r) * D + c0 + c] : 0.0;
    }
}

__global__ void __launch_bounds__(256) k_potrf_diag(double* A, int D, int j, int* bad) {
    __shared__ double S[kT][kTP];
    const int r0 = j * kT, bs = min(kT, D - r0);
    load_tile(S, A, D, r0, r0);
    for (int c = 0; c < bs; ++c) {
        __syncthreads();
        if (threadIdx.x == 0) {
            double d = S[c][c];
            if (!(d > 0.0)) { atomicOr(bad, 1); d = 1.0; }
            S[c][c] = sqrt(d);
        }
        __syncthreads();
        const double inv = 1.0 / S[c][c];
        for (int r = c + 1 + threadIdx.x; r < bs; r += blockDim.x) S[r][c] *= inv;
        __syncthreads();
        const int m = bs - c - 1;
        for (int q = threadIdx.x; q < m * m; q += blockDim.x) {
            const int r = c + 1 + q / m, s = c + 1 + q % m;
            if (s <= r) S[r][s] -= S[r][c] * S[s][c];
        }
    }
    __syncthreads();
    for (int q = threadIdx.x; q < bs * bs; q += blockDim.x) {
        const int r = q / bs, c = q % bs;
        A[(size_t)(r0 + r) * D + r0 + c] = (c <= r) ? S[r][c] : 0.0;
    }
}

// one CTA of 64 threads per block row i > j; thread = row of the tile
__global__ void __launch_bounds__(64) k_trsm_panel(double* A, int D, int j) {
    __shared__ double Ld[kT][kTP];
    __shared__ double X[kT][kTP];
    const int i = j + 1 + blockIdx.x;
    const int r0 = i * kT, c0 = j * kT;
    const int bs = min(kT, D - c0);
    load_tile(Ld, A, D, c0, c0);
    load_tile(X, A, D, r0, c0);
    __syncthreads();
    const int r = threadIdx.x;
    if (r0 + r < D) {
        for (int c = 0; c < bs; ++c) {
            double s = X[r][c];
            for (int m = 0; m < c; ++m) s -= X[r][m] * Ld[c][m];
            X[r][c] = s / Ld[c][c];
        }
        for (int c = 0; c < bs; ++c) A[(size_t)(r0 + r) * D + c0 + c] = X[r][c];
    }
}

// tiles (i, k), j < k <= i, numbered row by row of the lower triangle
__device__ __forceinline__ void tri_index(int idx, int& i, int& k) {
    int a = (int)((sqrt(8.0 * idx + 1.0) - 1.0) * 0.5);
    while ((a + 1) * (a + 2) / 2 <= idx) ++a;
    while (a * (a + 1) / 2 > idx) --a;
    i = a;
    k = idx - a * (a + 1) / 2;
}

__global__ void __launch_bounds__(256) k_syrk_update(double* A, int D, int j) {
    __shared__ double Li[kT][kTP];
    __shared__ double Lk[kT][kTP];
    int ii, kk;
    tri_index(blockIdx.x, ii, kk);
    const int i = j + 1 + ii, k = j + 1 + kk;
    const int ri = i * kT, rk = k * kT, cj = j * kT;
    load_tile(Li, A, D, ri, cj);
    load_tile(Lk, A, D, rk, cj);
    __syncthreads();
    const int tx = threadIdx.x % 16, ty = threadIdx.x / 16;
    double acc[4][4] = {};
    for (int m = 0; m < kT; ++m) {
        double a[4], b[4];
#pragma unroll
        for (int u = 0; u < 4; ++u) { a[u] = Li[ty + 16 * u][m]; b[u] = Lk[tx + 16 * u][m]; }
#pragma unroll
        for (int u = 0; u < 4; ++u)
#pragma unroll
            for (int v = 0; v < 4; ++v) acc[u][v] += a[u] * b[v];
    }
#pragma unroll
    for (int u = 0; u < 4; ++u)
#pragma unroll
        for (int v = 0; v < 4; ++v) {
            const int r = ri + ty + 16 * u, c = rk + tx + 16 * v;
            if (r < D && c < D && c <= r) A[(size_t)r * D + c] -= acc[u][v];
        }
}

// Block row i of X = L^-1: CTA c (c <= i) forms the tile X_ic.
__global__ void __launch_bounds__(256) k_trinv_row(const double* L, double* X, int D, int i) {
    __shared__ double Ta[kT][kTP];
    __shared__ double Tb[kT][kTP];
    const int c = blockIdx.x;
    const int ri = i * kT, cc = c * kT;
    const int tx = threadIdx.x % 16, ty = threadIdx.x / 16;
    double acc[4][4] = {};
    for (int k = c; k < i; ++k) {
        __syncthreads();
        load_tile(Ta, L, D, ri, k * kT);      // L_ik
        load_tile(Tb, X, D, k * kT, cc);      // X_kc
        __syncthreads();
        for (int m = 0; m < kT; ++m) {
            double a[4], b[4];
#pragma unroll
            for (int u = 0; u < 4; ++u) { a[u] = Ta[ty + 16 * u][m]; b[u] = Tb[m][tx + 16 * u]; }
#pragma unroll
            for (int u = 0; u < 4; ++u)
#pragma unroll
                for (int v = 0; v < 4; ++v) acc[u][v] += a[u] * b[v];
        }
    }
    __syncthreads();
    // right-hand side B = delta_ic I - acc into Tb; L_ii into Ta
#pragma unroll
    for (int u = 0; u < 4; ++u)
#pragma unroll
        for (int v = 0; v < 4; ++v) {
            const int r = ty + 16 * u, q = tx + 16 * v;
            Tb[r][q] = ((i == c && r == q) ? 1.0 : 0.0) - acc[u][v];
        }
    load_tile(Ta, L, D, ri, ri);
    __syncthreads();
    // forward substitution down the rows, one column per thread
    const int bs = min(kT, D - ri);
    if (threadIdx.x < kT) {
        const int q = threadIdx.x;
        for (int r = 0; r < bs; ++r) {
            double s = Tb[r][q];
            for (int m = 0; m < r; ++m) s -= Ta[r][m] * Tb[m][q];
            Tb[r][q] = s / Ta[r][r];
        }
    }
    __syncthreads();
    for (int q = threadIdx.x; q < kT * kT; q += blockDim.x) {
        const int r = q / kT, col = q % kT;
        if (ri + r < D && cc + col < D) X[(size_t)(ri + r) * D + cc + col] = Tb[r][col];
    }
}

__global__ void k_zero_upper(double* A, int D) {
    const size_t n = (size_t)D * D;
    for (size_t q = (size_t)blockIdx.x * blockDim.x + threadIdx.x; q < n; q += (size_t)gridDim.x * blockDim.x) {
        const int r = (int)(q / D), c = (int)(q % D);
        if (c > r) A[q] = 0.0;
    }
}

__global__ void k_transpose(const double* __restrict__ A, double* __restrict__ T, int D) {
    __shared__ double S[32][33];
    const int bx = blockIdx.x * 32, by = blockIdx.y * 32;
    for (int y = threadIdx.y; y < 32; y += blockDim.y)
        if (by + y < D && bx + threadIdx.x < D) S[y][threadIdx.x] = A[(size_t)(by + y) * D + bx + threadIdx.x];
    __syncthreads();
    for (int y = threadIdx.y; y < 32; y += blockDim.y)
        if (bx + y < D && by + threadIdx.x < D) T[(size_t)(bx + y) * D + by + threadIdx.x] = S[threadIdx.x][y];
}

__global__ void k_diag_log_sum(const double* L, int D, double* out) {
    __shared__ double part[256];
    double s = 0.0;
    for (int a = threadIdx.x; a < D; a += blockDim.x) s += log(L[(size_t)a * D + a]);
    part[threadIdx.x] = s;
    __syncthreads();
    for (int o = 128; o > 0; o >>= 1) {
        if (threadIdx.x < o) part[threadIdx.x] += part[threadIdx.x + o];
        __syncthreads();
    }
    if (threadIdx.x == 0) *out = part[0];
}

// C (device, D x D row-major, FP64) -> L^-1 (device, lower, row-major) in *Xout
// (caller frees) and sum ln L_aa.  C is overwritten by L.
int device_cholesky_inverse(double* dC, int D, double** Xout, double* sum_log_diag, cudaStream_t st) {
    const int nt = (D + kT - 1) / kT;
    int* bad = nullptr;
    double* dsum = nullptr;
    double* X = nullptr;
    auto cleanup = [&]() { cudaFree(bad); cudaFree(dsum); };
    if (cudaMalloc(&bad, sizeof(int)) != cudaSuccess || cudaMalloc(&dsum, sizeof(double)) != cudaSuccess) {
        cleanup();
        return NS_ENOMEM;
    }
    cudaMemsetAsync(bad, 0, sizeof(int), st);
    for (int j = 0; j < nt; ++j) {
        k_potrf_diag<<<1, 256, 0, st>>>(dC, D, j, bad);
        const int below = nt - j - 1;
        if (below > 0) {
            k_trsm_panel<<<below, 64, 0, st>>>(dC, D, j);
            k_syrk_update<<<below * (below + 1) / 2, 256, 0, st>>>(dC, D, j);
        }
    }
    k_zero_upper<<<1024, 256, 0, st>>>(dC, D);
    k_diag_log_sum<<<1, 256, 0, st>>>(dC, D, dsum);
    if (cudaGetLastError() != cudaSuccess) { cleanup(); return NS_ECUDA; }
    int h_bad = 0;
    if (cudaMemcpyAsync(&h_bad, bad, sizeof(int), cudaMemcpyDeviceToHost, st) != cudaSuccess ||
        cudaMemcpyAsync(sum_log_diag, dsum, sizeof(double), cudaMemcpyDeviceToHost, st) != cudaSuccess ||
        cudaStreamSynchronize(st) != cudaSuccess) {
        cleanup();
        return NS_ECUDA;
    }
    if (h_bad) { cleanup(); return NS_EINVAL; }
    if (cudaMalloc(&X, sizeof(double) * (size_t)D * D) != cudaSuccess) { cleanup(); return NS_ENOMEM; }
    cudaMemsetAsync(X, 0, sizeof(double) * (size_t)D * D, st);
    for (int i = 0; i < nt; ++i) k_trinv_row<<<i + 1, 256, 0, st>>>(dC, X, D, i);
    if (cudaGetLastError() != cudaSuccess || cudaStreamSynchronize(st) != cudaSuccess) {
        cudaFree(X);
        cleanup();
        return NS_ECUDA;
    }
    cleanup();
    *Xout = X;
    return NS_OK;
}

// T = A^T for a D x D FP64 matrix on the device.
int device_transpose(const double* dA, double* dT, int D, cudaStream_t st) {
    dim3 g((D + 31) / 32, (D + 31) / 32), b(32, 8);
    k_transpose<<<g, b, 0, st>>>(dA, dT, D);
    NS_CUDA_TRY(cudaGetLastError());
    return NS_OK;
}

}  // namespace gpuns
