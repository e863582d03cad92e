// The shear projection (App. A, rows A8-A12) and the whitened chi^2 (A13).
//
// k_projection: one CTA (8 warps) per likelihood evaluation.
//   1. background: E(a) at the nodes; chi increments over each a-interval by a
//      4-point Gauss-Legendre rule and a block prefix sum (chi_0 = 0 at a = 1);
//      growth ln D = -sum trapezoid(Omega_m(a)^gamma) dln a by a second scan.
//   2. windows: per bin the shifted Gaussian n_i(z - D_z,i), normalised on the
//      grid; W^gamma (Eq. 5) = A (chi/a) [S0 - chi S1] with exclusive suffix
//      sums S0 = sum_{m>n} w n, S1 = sum_{m>n} w n / chi (the m = n term of the
//      direct double sum is zero); W^I (Eq. 6); V_i = sqrt(w/chi^2) W^eps_i.
//   3. the emulator's log10 P table (n_z x n_k) is staged in shared memory
//      (over the background scratch) so the 16 taps of every lookup hit smem.
//   4. Limber (Eq. 3-4): multipoles in groups of G; each lane owns chi nodes,
//      forms the node's z-taps and window values once per group, then for the
//      group's multipoles the Catmull-Rom lookup at ln k = ln(ell + 1/2) -
//      ln chi and the pair sums V_i V_j P.  Warp shuffles, then a fixed-order
//      sum over warps (deterministic).
//   5. data vector (1 + m_i)(1 + m_j) C_ij(ell) + T b and residual d - m.
// k_whiten / k_chi2_finish: Y = R L^-T as a tiled product (32 rows x 64
//   columns per CTA, b <= a), per-tile row sums of y^2, then a fixed-order sum
//   and log L = c0 - chi^2 / 2 in FP64.
#include "likelihood.cuh"

namespace gpuns {

__constant__ double c_glx2[4] = {-0.86113631159405257522, -0.33998104358485626480,
                                  0.33998104358485626480, 0.86113631159405257522};
__constant__ double c_glw2[4] = {0.34785484513745385737, 0.65214515486254614263,
                                  0.65214515486254614263, 0.34785484513745385737};

template <typename T> __device__ __forceinline__ const T* pick(const double* d, const float* f);
template <> __device__ __forceinline__ const double* pick<double>(const double* d, const float*) { return d; }
template <> __device__ __forceinline__ const float* pick<float>(const double*, const float* f) { return f; }

template <typename T> __device__ __forceinline__ T pow10_(T v);
template <> __device__ __forceinline__ double pow10_<double>(double v) { return exp(v * kLn10); }
template <> __device__ __forceinline__ float pow10_<float>(float v) { return exp2f(v * 3.32192809488736234787f); }

template <typename T> __device__ __forceinline__ T sqrt_(T x) { return sqrt(x); }

constexpr int kProjThreads = 256;
constexpr int kProjWarps = kProjThreads / 32;
constexpr int kGroup = 2;   // multipoles per Limber group

template <typename T, int NB>
__global__ void __launch_bounds__(kProjThreads, 2)
k_projection(const ShearParams sp, const double* __restrict__ theta_full, const T* __restrict__ table,
             T* __restrict__ resid, double* __restrict__ model_out, const int* __restrict__ nrows) {
    constexpr int NP = NB * (NB + 1) / 2;
    constexpr int G = kGroup;
    const int row = blockIdx.x;
    if (row >= *nrows) return;
    extern __shared__ __align__(16) unsigned char smem_raw[];
    const int N = sp.N, nzk = sp.n_z * sp.n_k;
    const int usz = max(6 * N, nzk);
    T* chi = reinterpret_cast<T*>(smem_raw);
    T* lnchi = chi + N;
    T* V = lnchi + N;                 // NB x N
    // union: background scratch, then the P table; 16-byte aligned for vector stores
    T* U = chi + (((2 + NB) * N + 3) & ~3);
    T* part = U + ((usz + 3) & ~3);   // warps x G x NP
    T* Cl = part + kProjWarps * G * NP;
    T* th = Cl + NP * sp.n_ell;
    T* red = th + sp.n_params;        // 64
    T* Ez = U;
    T* Dg = U + N;
    T* omw = U + 2 * N;
    T* t0 = U + 3 * N;
    T* t1 = U + 4 * N;
    T* t2 = U + 5 * N;
    const T* a_ = pick<T>(sp.a, sp.a_f);
    const T* lna_ = pick<T>(sp.lna, sp.lna_f);
    const T* z_ = pick<T>(sp.z, sp.z_f);
    const T* wa_ = pick<T>(sp.wa, sp.wa_f);
    const int tid = threadIdx.x, nt = kProjThreads;

    for (int i = tid; i < sp.n_params; i += nt) th[i] = (T)theta_full[(size_t)row * sp.n_params + i];
    __syncthreads();
    const T h = th[2];
    const T om = (th[0] + th[1]) / (h * h);
    const T w0 = th[5], wa = th[6];
    const T pde = T(3) * (T(1) + w0 + wa);
    const T chiH = T(kCover100) / h;
    const T gamma = T(0.55) + T(0.05) * (T(1) + w0 + T(0.5) * wa);

    // 1. background
    for (int n = tid; n < N; n += nt) {
        const T a = a_[n], lna = lna_[n];
        const T e2 = om * dexp<T>(T(-3) * lna) + (T(1) - om) * dexp<T>(-pde * lna - T(3) * wa * (T(1) - a));
        Ez[n] = sqrt_<T>(e2);
        T inc = T(0);
        if (n < N - 1) {
            const T a1 = a_[n + 1];
            const T mid = T(0.5) * (a + a1), half = T(0.5) * (a - a1);
#pragma unroll
            for (int g = 0; g < 4; ++g) {
                const T ag = mid + half * (T)c_glx2[g];
                const T lg = dlog<T>(ag);
                const T eg = om * dexp<T>(T(-3) * lg) + (T(1) - om) * dexp<T>(-pde * lg - T(3) * wa * (T(1) - ag));
                inc += (T)c_glw2[g] / (ag * ag * sqrt_<T>(eg));
            }
            inc *= chiH * half;
        }
        t0[n] = inc;
    }
    __syncthreads();
    block_exclusive_scan(t0, N, red);
    for (int n = tid; n < N; n += nt) {
        const T c = t0[n];
        chi[n] = c;
        lnchi[n] = (n >= 1) ? dlog<T>(c) : T(0);
        const T oma = om * dexp<T>(T(-3) * lna_[n]) / (Ez[n] * Ez[n]);
        t1[n] = dexp<T>(gamma * dlog<T>(oma));
        omw[n] = wa_[n] * chiH / (a_[n] * a_[n] * Ez[n]);
    }
    __syncthreads();
    for (int n = tid; n < N; n += nt)
        t2[n] = (n < N - 1) ? T(0.5) * (t1[n] + t1[n + 1]) * (lna_[n] - lna_[n + 1]) : T(0);
    __syncthreads();
    block_exclusive_scan(t2, N, red);
    for (int n = tid; n < N; n += nt) Dg[n] = dexp<T>(-t2[n]);
    __syncthreads();

    // 2. windows
    const T pref = T(1.5) * om / (chiH * chiH);
    const T A_IA = th[9], eta = th[10];
#pragma unroll 1
    for (int i = 0; i < NB; ++i) {
        const T dz = th[11 + i];
        const T mu = (T)sp.nz_mean[i], sg = (T)sp.nz_sigma[i];
        T pnorm = T(0);
        for (int n = tid; n < N; n += nt) {
            const T u = (z_[n] - dz - mu) / sg;
            const T raw = dexp<T>(T(-0.5) * u * u);
            t1[n] = raw;
            pnorm += wa_[n] * raw / (a_[n] * a_[n]);
        }
        const T norm = block_sum(pnorm, red);
        for (int n = tid; n < N; n += nt) {
            const T nchi = t1[n] * Ez[n] / (chiH * norm);
            t1[n] = nchi;
            const T w_n = (n >= 1) ? omw[n] * nchi : T(0);
            t0[n] = w_n;
            t2[n] = (n >= 1) ? w_n / chi[n] : T(0);
        }
        __syncthreads();
        block_exclusive_suffix_scan(t0, N, red);
        block_exclusive_suffix_scan(t2, N, red);
        for (int n = tid; n < N; n += nt) {
            T v = T(0);
            if (n >= 1) {
                const T c = chi[n];
                const T Wg = pref * c / a_[n] * (t0[n] - c * t2[n]);
                const T amp = A_IA * dexp<T>(eta * dlog<T>((T(1) + z_[n]) / (T)sp.ia_pivot));
                const T WI = -amp * (T)sp.c1rho * om / Dg[n] * t1[n];
                v = sqrt_<T>(omw[n] / (c * c)) * (Wg + WI);
            }
            V[i * N + n] = v;
        }
        __syncthreads();
    }

    // 3. stage the log10 P table in shared memory
    {
        const T* src = table + (size_t)row * nzk;
        if (sizeof(T) == 4 && (nzk % 4) == 0 && ((reinterpret_cast<uintptr_t>(src) & 15) == 0) &&
            ((reinterpret_cast<uintptr_t>(U) & 15) == 0)) {
            const float4* s4 = reinterpret_cast<const float4*>(src);
            float4* d4 = reinterpret_cast<float4*>(U);
            for (int i = tid; i < nzk / 4; i += nt) d4[i] = __ldg(s4 + i);
        } else {
            for (int i = tid; i < nzk; i += nt) U[i] = src[i];
        }
    }
    __syncthreads();

    // 4. Limber with the Catmull-Rom lookup
    const int lane = tid & 31, wid = tid >> 5;
    const T lkmin = (T)sp.lnk_min, lkmax = (T)sp.lnk_max, inv_dk = T(1) / (T)sp.dlnk;
    const T inv_dz = T(1) / (T)sp.dz;
    const int n_k = sp.n_k, n_z = sp.n_z;
#pragma unroll 1
    for (int g0 = 0; g0 < sp.n_ell; g0 += G) {
        T acc[G][NP];
#pragma unroll
        for (int j = 0; j < G; ++j)
#pragma unroll
            for (int p = 0; p < NP; ++p) acc[j][p] = T(0);
        T lne[G];
#pragma unroll
        for (int j = 0; j < G; ++j) lne[j] = (g0 + j < sp.n_ell) ? (T)sp.lnell[g0 + j] : T(0);
        for (int n = 1 + lane + 32 * wid; n < N; n += nt) {
            const T uz = z_[n] * inv_dz;
            int jz = (int)floor(uz);
            jz = min(max(jz, 0), n_z - 2);
            T wz0[4], wz[4];
            int zr[4];
            catmull_rom<T>(uz - (T)jz, wz0);
            fold_taps<T>(jz, n_z, wz0, zr, wz);
            const T* r0 = U + zr[0] * n_k;
            const T* r1 = U + zr[1] * n_k;
            const T* r2 = U + zr[2] * n_k;
            const T* r3 = U + zr[3] * n_k;
            T vv[NB];
#pragma unroll
            for (int i = 0; i < NB; ++i) vv[i] = V[i * N + n];
            const T lc = lnchi[n];
#pragma unroll
            for (int j = 0; j < G; ++j) {
                if (g0 + j < sp.n_ell) {
                    T s = lne[j] - lc;
                    s = fmin(fmax(s, lkmin), lkmax);
                    const T uk = (s - lkmin) * inv_dk;
                    int ik = (int)floor(uk);
                    ik = min(max(ik, 0), n_k - 2);
                    T wk0[4], wk[4];
                    int kc[4];
                    catmull_rom<T>(uk - (T)ik, wk0);
                    fold_taps<T>(ik, n_k, wk0, kc, wk);
                    const T v = wz[0] * (wk[0] * r0[kc[0]] + wk[1] * r0[kc[1]] + wk[2] * r0[kc[2]] + wk[3] * r0[kc[3]]) +
                                wz[1] * (wk[0] * r1[kc[0]] + wk[1] * r1[kc[1]] + wk[2] * r1[kc[2]] + wk[3] * r1[kc[3]]) +
                                wz[2] * (wk[0] * r2[kc[0]] + wk[1] * r2[kc[1]] + wk[2] * r2[kc[2]] + wk[3] * r2[kc[3]]) +
                                wz[3] * (wk[0] * r3[kc[0]] + wk[1] * r3[kc[1]] + wk[2] * r3[kc[2]] + wk[3] * r3[kc[3]]);
                    const T P = pow10_<T>(v);
                    T tv[NB];
#pragma unroll
                    for (int i = 0; i < NB; ++i) tv[i] = vv[i] * P;
                    int p = 0;
#pragma unroll
                    for (int i = 0; i < NB; ++i)
#pragma unroll
                        for (int jj = i; jj < NB; ++jj) acc[j][p++] += tv[i] * vv[jj];
                }
            }
        }
#pragma unroll
        for (int j = 0; j < G; ++j)
#pragma unroll
            for (int p = 0; p < NP; ++p) {
                const T s = warp_sum(acc[j][p]);
                if (lane == 0) part[(wid * G + j) * NP + p] = s;
            }
        __syncthreads();
        for (int t = tid; t < G * NP; t += nt) {
            const int j = t / NP, p = t % NP;
            if (g0 + j < sp.n_ell) {
                T s = T(0);
#pragma unroll
                for (int w = 0; w < kProjWarps; ++w) s += part[(w * G + j) * NP + p];
                Cl[p * sp.n_ell + g0 + j] = s;
            }
        }
        __syncthreads();
    }

    // 5. data vector and residual
    for (int a = tid; a < sp.D; a += nt) {
        const int p = a / sp.n_ell, e = a % sp.n_ell;
        const int i = sp.pi[p], j = sp.pj[p];
        T m = (T(1) + th[11 + NB + i]) * (T(1) + th[11 + NB + j]) * Cl[p * sp.n_ell + e];
        for (int t = 0; t < sp.n_tmpl; ++t) m += (T)sp.tmpl[(size_t)a * sp.n_tmpl + t] * th[11 + 2 * NB + t];
        if (model_out) model_out[(size_t)row * sp.D + a] = (double)m;
        else resid[(size_t)row * sp.D + a] = (T)sp.data[a] - m;
    }
}

size_t projection_smem_bytes(const ShearParams& sp, int elt) {
    const int NP = sp.nb * (sp.nb + 1) / 2;
    const int usz = std::max(6 * sp.N, sp.n_z * sp.n_k);
    const size_t n = (size_t)(((2 + sp.nb) * sp.N + 3) & ~3) + ((usz + 3) & ~3) + (size_t)kProjWarps * kGroup * NP +
                     (size_t)NP * sp.n_ell + sp.n_params + 64;
    return n * elt;
}

template <typename T, int NB>
static int launch_projection_nb(const ShearParams& sp, const double* theta_full, const T* table, T* resid,
                                double* model_out, const int* nrows, int grid_rows, cudaStream_t st) {
    const size_t smem = projection_smem_bytes(sp, sizeof(T));
    if (smem > 227 * 1024) return NS_ENOTSUP;
    static bool attr_done = false;
    if (!attr_done) {
        NS_CUDA_TRY(cudaFuncSetAttribute(k_projection<T, NB>, cudaFuncAttributeMaxDynamicSharedMemorySize, 227 * 1024));
        attr_done = true;
    }
    k_projection<T, NB><<<grid_rows, kProjThreads, smem, st>>>(sp, theta_full, table, resid, model_out, nrows);
    NS_CUDA_TRY(cudaGetLastError());
    return NS_OK;
}

template <typename T>
int launch_shear(const ShearParams& sp, const double* theta_full, const T* table, T* resid, double* model_out,
                 const int* nrows, int grid_rows, cudaStream_t st) {
    switch (sp.nb) {
        case 1: return launch_projection_nb<T, 1>(sp, theta_full, table, resid, model_out, nrows, grid_rows, st);
        case 2: return launch_projection_nb<T, 2>(sp, theta_full, table, resid, model_out, nrows, grid_rows, st);
        case 3: return launch_projection_nb<T, 3>(sp, theta_full, table, resid, model_out, nrows, grid_rows, st);
        case 4: return launch_projection_nb<T, 4>(sp, theta_full, table, resid, model_out, nrows, grid_rows, st);
        case 5: return launch_projection_nb<T, 5>(sp, theta_full, table, resid, model_out, nrows, grid_rows, st);
        default: return NS_ENOTSUP;
    }
}
template int launch_shear<float>(const ShearParams&, const double*, const float*, float*, double*, const int*, int,
                                 cudaStream_t);
template int launch_shear<double>(const ShearParams&, const double*, const double*, double*, double*, const int*,
                                  int, cudaStream_t);

// ---------------------------------------------------------------- chi^2
constexpr int kWR = 32;   // rows per whitening tile
constexpr int kWC = 64;   // columns per whitening tile
constexpr int kWK = 32;   // reduction chunk

template <typename TR, typename TA>
__global__ void __launch_bounds__(256)
k_whiten(const TR* __restrict__ resid, int D, const TA* __restrict__ LinvT, TA* __restrict__ partial,
         int ntile, const int* __restrict__ nrows) {
    const int M = *nrows;
    const int row0 = blockIdx.y * kWR;
    if (row0 >= M) return;
    const int a0 = blockIdx.x * kWC;
    __shared__ TA Rs[kWR][kWK + 1];
    __shared__ TA Ls[kWK][kWC + 1];
    const int tid = threadIdx.x, tx = tid & 31, ty = tid >> 5;
    TA acc[4][2];
#pragma unroll
    for (int i = 0; i < 4; ++i) { acc[i][0] = TA(0); acc[i][1] = TA(0); }
    const int b_end = min(D, a0 + kWC);
    for (int b0 = 0; b0 < b_end; b0 += kWK) {
        for (int q = tid; q < kWR * kWK; q += 256) {
            const int r = q / kWK, c = q % kWK;
            Rs[r][c] = (row0 + r < M && b0 + c < D) ? (TA)resid[(size_t)(row0 + r) * D + b0 + c] : TA(0);
        }
        for (int q = tid; q < kWK * kWC; q += 256) {
            const int bb = q / kWC, aa = q % kWC;
            Ls[bb][aa] = (b0 + bb < D && a0 + aa < D) ? LinvT[(size_t)(b0 + bb) * D + a0 + aa] : TA(0);
        }
        __syncthreads();
#pragma unroll 8
        for (int kk = 0; kk < kWK; ++kk) {
            const TA l0 = Ls[kk][tx], l1 = Ls[kk][tx + 32];
#pragma unroll
            for (int i = 0; i < 4; ++i) {
                const TA rv = Rs[ty + 8 * i][kk];
                acc[i][0] += rv * l0;
                acc[i][1] += rv * l1;
            }
        }
        __syncthreads();
    }
#pragma unroll
    for (int i = 0; i < 4; ++i) {
        TA s = TA(0);
        if (a0 + tx < D) s += acc[i][0] * acc[i][0];
        if (a0 + tx + 32 < D) s += acc[i][1] * acc[i][1];
        s = warp_sum(s);
        const int r = row0 + ty + 8 * i;
        if (tx == 0 && r < M) partial[(size_t)r * ntile + blockIdx.x] = s;
    }
}

template <typename TA>
__global__ void k_chi2_finish(const TA* __restrict__ partial, int ntile, double c0, double* __restrict__ logL,
                              const int* __restrict__ nrows) {
    const int r = blockIdx.x * blockDim.x + threadIdx.x;
    if (r >= *nrows) return;
    TA s = TA(0);
    for (int t = 0; t < ntile; ++t) s += partial[(size_t)r * ntile + t];
    logL[r] = c0 - 0.5 * (double)s;
}

template <typename TR, typename TA>
int launch_chi2(const TR* resid, int D, const TA* LinvT, double c0, double* logL, void* partial, const int* nrows,
                int grid_rows, cudaStream_t st) {
    const int ntile = (D + kWC - 1) / kWC;
    dim3 g(ntile, (grid_rows + kWR - 1) / kWR);
    k_whiten<TR, TA><<<g, 256, 0, st>>>(resid, D, LinvT, (TA*)partial, ntile, nrows);
    k_chi2_finish<TA><<<(grid_rows + 127) / 128, 128, 0, st>>>((const TA*)partial, ntile, c0, logL, nrows);
    NS_CUDA_TRY(cudaGetLastError());
    return NS_OK;
}
template int launch_chi2<float, float>(const float*, int, const float*, double, double*, void*, const int*, int,
                                       cudaStream_t);
template int launch_chi2<float, double>(const float*, int, const double*, double, double*, void*, const int*, int,
                                        cudaStream_t);
template int launch_chi2<double, double>(const double*, int, const double*, double, double*, void*, const int*, int,
                                         cudaStream_t);

}  // namespace gpuns
