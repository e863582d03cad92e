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
//      ln chi and the pair sums V_i V_j P.  A transposed warp reduction, then
//      a fixed-order sum over warps (deterministic).
//   5. data vector (1 + m_i)(1 + m_j) C_ij(ell) + T b and residual d - m.
// k_whiten / k_chi2_finish: Y = R L^-T in tiles of 16 rows x 64 columns
//   (b <= a), per-tile row sums of y^2, then a fixed-order sum and
//   log L = c0 - chi^2 / 2 added in FP64.
#include "likelihood.cuh"

namespace gpuns {

__constant__ double c_glx2[4] = {-0.86113631159405257522, -0.33998104358485626480,
                                  0.33998104358485626480, 0.86113631159405257522};
__constant__ double c_glw2[4] = {0.34785484513745385737, 0.65214515486254614263,
                                  0.65214515486254614263, 0.34785484513745385737};

template <typename T> __device__ __forceinline__ const T* pick(const double* d, const float* f);
template <> __device__ __forceinline__ const double* pick<double>(const double* d, const float*) { return d; }
template <> __device__ __forceinline__ const float* pick<float>(const double*, const float* f) { return f; }

// Transcendentals: accurate library versions, or (FAST, BF16 modes) the SFU
// approximations, whose ~1e-6 relative error is far below the bf16 emulator's.
template <typename T, bool FAST> struct Math;
template <> struct Math<double, false> {
    static __device__ __forceinline__ double ex(double x) { return exp(x); }
    static __device__ __forceinline__ double lg(double x) { return log(x); }
    static __device__ __forceinline__ double p10(double v) { return exp(v * kLn10); }
};
template <> struct Math<float, false> {
    static __device__ __forceinline__ float ex(float x) { return expf(x); }
    static __device__ __forceinline__ float lg(float x) { return logf(x); }
    static __device__ __forceinline__ float p10(float v) { return exp2f(v * 3.32192809488736234787f); }
};
template <> struct Math<float, true> {
    static __device__ __forceinline__ float ex(float x) { return __expf(x); }
    static __device__ __forceinline__ float lg(float x) { return __logf(x); }
    static __device__ __forceinline__ float p10(float v) {
        float y;
        asm("ex2.approx.ftz.f32 %0, %1;" : "=f"(y) : "f"(v * 3.32192809488736234787f));
        return y;
    }
};

template <typename T> __device__ __forceinline__ T sqrt_(T x) { return sqrt(x); }

constexpr int kProjThreads = 256;
constexpr int kProjWarps = kProjThreads / 32;

// Reduce 32 per-lane values across the warp so that lane l ends with the sum
// over lanes of value l (recursive halving: 31 shuffles instead of 32 x 5).
template <typename T>
__device__ __forceinline__ T warp_transpose_sum(T (&v)[32]) {
    const int lane = threadIdx.x & 31;
#pragma unroll
    for (int off = 16; off >= 1; off >>= 1) {
        const bool upper = (lane & off) != 0;
#pragma unroll
        for (int i = 0; i < off; ++i) {
            const T send = upper ? v[i] : v[i + off];
            const T keep = upper ? v[i + off] : v[i];
            v[i] = keep + __shfl_xor_sync(0xffffffffu, send, off);
        }
    }
    return v[0];
}

// 16 values per lane -> lane l holds the warp sum of value (l & 15).
template <typename T>
__device__ __forceinline__ T warp_transpose_sum16(T (&v)[16]) {
    const int lane = threadIdx.x & 31;
#pragma unroll
    for (int off = 8; off >= 1; off >>= 1) {
        const bool upper = (lane & off) != 0;
#pragma unroll
        for (int i = 0; i < off; ++i) {
            const T send = upper ? v[i] : v[i + off];
            const T keep = upper ? v[i + off] : v[i];
            v[i] = keep + __shfl_xor_sync(0xffffffffu, send, off);
        }
    }
    return v[0] + __shfl_xor_sync(0xffffffffu, v[0], 16);
}

template <typename T>
struct ProjArgs {
    ShearParams sp;
    const double* theta_full;
    const T* table;
    T* resid;             // rows x D residuals (unused when model_out is set)
    double* model_out;
    const int* nrows;
};

template <typename T, int NB, bool FAST>
__global__ void __launch_bounds__(kProjThreads, sizeof(T) == 8 ? 1 : 3)
k_projection(const ProjArgs<T> args) {
    using M = Math<T, FAST>;
    constexpr int NP = NB * (NB + 1) / 2;
    static_assert(NP <= 16, "pair sums per item must fit one 16-value warp transpose");
    const ShearParams& sp = args.sp;
    const int row = blockIdx.x;
    if (row >= *args.nrows) return;
    extern __shared__ __align__(16) unsigned char smem_raw[];
    const int N = sp.N, nzk = sp.n_z * sp.n_k;
    const int PK = sp.n_k + 2;                        // padded table row length
    const int usz = max(6 * N, (sp.n_z + 2) * PK);
    const int n_items = sp.n_ell * 2;                 // (multipole, half of the nodes)
    T* chi = reinterpret_cast<T*>(smem_raw);
    T* lnchi = chi + N;
    T* V = lnchi + N;                          // NB x N
    T* U = chi + (((2 + NB) * N + 3) & ~3);    // union (16-byte aligned): scratch, P table, residual
    T* part = U + ((usz + 3) & ~3);            // max(warps x 32, items x 16)
    T* Cl = part + max(kProjWarps * 32, n_items * 16);   // NP x n_ell
    T* th = Cl + NP * sp.n_ell;
    T* red = th + sp.n_params;                 // 96
    T* Ez = U;
    T* Dg = U + N;
    T* omw = U + 2 * N;
    T* t0 = U + 3 * N;
    T* t1 = U + 4 * N;
    const T* a_ = pick<T>(sp.a, sp.a_f);
    const T* lna_ = pick<T>(sp.lna, sp.lna_f);
    const T* z_ = pick<T>(sp.z, sp.z_f);
    const T* wa_ = pick<T>(sp.wa, sp.wa_f);
    const int tid = threadIdx.x, nt = kProjThreads;
    const int lane = tid & 31, wid = tid >> 5;

    for (int i = tid; i < sp.n_params; i += nt) th[i] = (T)args.theta_full[(size_t)row * sp.n_params + i];
    __syncthreads();
    const T h = th[2];
    const T om = (th[0] + th[1]) / (h * h);
    const T w0 = th[5], wa = th[6];
    const T pde = T(3) * (T(1) + w0 + wa);
    const T chiH = T(kCover100) / h;
    const T gamma = T(0.55) + T(0.05) * (T(1) + w0 + T(0.5) * wa);

    // 1. background: E(a), chi by composite 4-point Gauss-Legendre + scan, growth
    for (int n = tid; n < N; n += nt) {
        const T a = a_[n], lna = lna_[n];
        const T e2 = om * M::ex(T(-3) * lna) + (T(1) - om) * M::ex(-pde * lna - T(3) * wa * (T(1) - a));
        Ez[n] = sqrt_<T>(e2);
        T inc = T(0);
        if (n < N - 1) {
            const T a1 = a_[n + 1];
            const T mid = T(0.5) * (a + a1), half = T(0.5) * (a - a1);
#pragma unroll
            for (int g = 0; g < 4; ++g) {
                const T ag = mid + half * (T)c_glx2[g];
                const T lg = M::lg(ag);
                const T ia = T(1) / ag;
                const T eg = om * ia * ia * ia + (T(1) - om) * M::ex(-pde * lg - T(3) * wa * (T(1) - ag));
                inc += (T)c_glw2[g] * ia * ia / sqrt_<T>(eg);
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
        lnchi[n] = (n >= 1) ? M::lg(c) : T(0);
        const T oma = om * M::ex(T(-3) * lna_[n]) / (Ez[n] * Ez[n]);
        t1[n] = M::ex(gamma * M::lg(oma));
        omw[n] = wa_[n] * chiH / (a_[n] * a_[n] * Ez[n]);
    }
    __syncthreads();
    for (int n = tid; n < N; n += nt)
        t0[n] = (n < N - 1) ? T(0.5) * (t1[n] + t1[n + 1]) * (lna_[n] - lna_[n + 1]) : T(0);
    __syncthreads();
    block_exclusive_scan(t0, N, red);
    for (int n = tid; n < N; n += nt) Dg[n] = M::ex(-t0[n]);

    // 2. windows for all bins at once: n_i(chi) into V, then one multi-value
    //    exclusive suffix scan of (w n_i, w n_i / chi) over contiguous chunks.
    T pn[NB];
#pragma unroll
    for (int i = 0; i < NB; ++i) pn[i] = T(0);
    for (int n = tid; n < N; n += nt) {
        const T wz = wa_[n] / (a_[n] * a_[n]);
#pragma unroll
        for (int i = 0; i < NB; ++i) {
            const T u = (z_[n] - th[11 + i] - (T)sp.nz_mean[i]) / (T)sp.nz_sigma[i];
            const T raw = M::ex(T(-0.5) * u * u);
            V[i * N + n] = raw;
            pn[i] += wz * raw;
        }
    }
    // block sums of the NB normalisations
#pragma unroll
    for (int i = 0; i < NB; ++i) {
        const T s = warp_sum(pn[i]);
        if (lane == 0) part[wid * 32 + i] = s;
    }
    __syncthreads();
    T inv_norm[NB];
#pragma unroll
    for (int i = 0; i < NB; ++i) {
        T s = T(0);
#pragma unroll
        for (int w = 0; w < kProjWarps; ++w) s += part[w * 32 + i];
        inv_norm[i] = T(1) / (chiH * s);
    }
    const int chunk = (N + nt - 1) / nt;
    const int lo = min(N, tid * chunk), hi = min(N, lo + chunk);
    T s0[NB], s1[NB];
#pragma unroll
    for (int i = 0; i < NB; ++i) { s0[i] = T(0); s1[i] = T(0); }
    for (int n = lo; n < hi; ++n) {
        const T e = Ez[n];
#pragma unroll
        for (int i = 0; i < NB; ++i) {
            const T nchi = V[i * N + n] * e * inv_norm[i];
            V[i * N + n] = nchi;
            if (n >= 1) {
                const T wn = omw[n] * nchi;
                s0[i] += wn;
                s1[i] += wn / chi[n];
            }
        }
    }
    // exclusive suffix over threads of the 2 NB chunk totals
    T e0[NB], e1[NB];
#pragma unroll
    for (int i = 0; i < NB; ++i) {
        T x0 = s0[i], x1 = s1[i];
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
            const T y0 = __shfl_down_sync(0xffffffffu, x0, o);
            const T y1 = __shfl_down_sync(0xffffffffu, x1, o);
            if (lane + o < 32) { x0 += y0; x1 += y1; }
        }
        e0[i] = x0 - s0[i];     // exclusive within the warp (lanes above)
        e1[i] = x1 - s1[i];
        if (lane == 0) { red[wid * 2 * NB + i] = x0; red[wid * 2 * NB + NB + i] = x1; }
    }
    __syncthreads();
#pragma unroll
    for (int i = 0; i < NB; ++i)
        for (int w = wid + 1; w < kProjWarps; ++w) { e0[i] += red[w * 2 * NB + i]; e1[i] += red[w * 2 * NB + NB + i]; }
    const T pref = T(1.5) * om / (chiH * chiH);
    const T A_IA = th[9], eta = th[10];
    for (int n = hi - 1; n >= lo; --n) {
        const T c = chi[n];
        const T sq = (n >= 1) ? sqrt_<T>(omw[n] / (c * c)) : T(0);
        const T amp = A_IA * M::ex(eta * M::lg((T(1) + z_[n]) / (T)sp.ia_pivot)) * (T)sp.c1rho * om / Dg[n];
        const T pc = pref * c / a_[n];
#pragma unroll
        for (int i = 0; i < NB; ++i) {
            const T nchi = V[i * N + n];
            T v = T(0);
            if (n >= 1) {
                v = sq * (pc * (e0[i] - c * e1[i]) - amp * nchi);
                const T wn = omw[n] * nchi;
                e0[i] += wn;
                e1[i] += wn / c;
            }
            V[i * N + n] = v;
        }
    }
    __syncthreads();

    // 3. stage the log10 P table in shared memory with one ghost row/column on
    //    each side (linear extrapolation, rows first, then columns), so every
    //    Catmull-Rom tap is an in-range read.
    {
        const T* src = args.table + (size_t)row * nzk;
        const int n_k = sp.n_k, n_z = sp.n_z;
        if (sizeof(T) == 4 && (nzk % 4) == 0 && ((reinterpret_cast<uintptr_t>(src) & 15) == 0)) {
            const float4* s4 = reinterpret_cast<const float4*>(src);
            for (int i = tid; i < nzk / 4; i += nt) {
                const float4 q = __ldg(s4 + i);
                const int e = 4 * i;
                const T vals[4] = {(T)q.x, (T)q.y, (T)q.z, (T)q.w};
#pragma unroll
                for (int c = 0; c < 4; ++c) {
                    const int r = (e + c) / n_k, k = (e + c) % n_k;
                    U[(r + 1) * PK + k + 1] = vals[c];
                }
            }
        } else {
            for (int i = tid; i < nzk; i += nt) U[(i / n_k + 1) * PK + i % n_k + 1] = src[i];
        }
        __syncthreads();
        for (int k = 1 + tid; k <= n_k; k += nt) {
            U[k] = T(2) * U[PK + k] - U[2 * PK + k];
            U[(n_z + 1) * PK + k] = T(2) * U[n_z * PK + k] - U[(n_z - 1) * PK + k];
        }
        __syncthreads();
        for (int r = tid; r < n_z + 2; r += nt) {
            U[r * PK] = T(2) * U[r * PK + 1] - U[r * PK + 2];
            U[r * PK + n_k + 1] = T(2) * U[r * PK + n_k] - U[r * PK + n_k - 1];
        }
    }
    __syncthreads();

    // 4. Limber with the Catmull-Rom lookup.  Work items are (multipole, half
    //    of the chi nodes), spread over the warps; each lane walks nodes of its
    //    item, reads the node's precomputed z-taps (doubled weights), forms the
    //    k-taps (doubled) and the pair sums V_i V_j P; one transposed warp
    //    reduction per item, then the two halves are added in fixed order.
    const T lkmin = (T)sp.lnk_min, lkmax = (T)sp.lnk_max, inv_dk = T(1) / (T)sp.dlnk;
    const int n_k = sp.n_k;
    const int* zrp = sp.zrp;
    const T* zwp = pick<T>(sp.zw4d, sp.zw4f);
    const int half_len = (N - 1 + 1) / 2;
#pragma unroll 1
    for (int item = wid; item < n_items; item += kProjWarps) {
        const int l = item >> 1;
        const int nb0 = 1 + (item & 1) * half_len, nb1 = min(N, nb0 + half_len);
        T acc[16];
#pragma unroll
        for (int q = 0; q < 16; ++q) acc[q] = T(0);
        const T lne = (T)sp.lnell[l];
        for (int n = nb0 + lane; n < nb1; n += 32) {
            const T* rz = U + zrp[n] * PK;
            const T wz0 = zwp[4 * n], wz1 = zwp[4 * n + 1], wz2 = zwp[4 * n + 2], wz3 = zwp[4 * n + 3];
            T sk = lne - lnchi[n];
            sk = fmin(fmax(sk, lkmin), lkmax);
            const T uk = (sk - lkmin) * inv_dk;
            int ik = (int)floor(uk);
            ik = min(max(ik, 0), n_k - 2);
            const T t = uk - (T)ik, t2 = t * t;
            // doubled Catmull-Rom weights
            const T k0 = t * (t * (T(2) - t) - T(1));
            const T k1 = T(2) + t2 * (T(3) * t - T(5));
            const T k2 = t * (T(1) + t * (T(4) - T(3) * t));
            const T k3 = t2 * (t - T(1));
            const T* c = rz + ik;
            const T v = wz0 * (k0 * c[0] + k1 * c[1] + k2 * c[2] + k3 * c[3]) +
                        wz1 * (k0 * c[PK] + k1 * c[PK + 1] + k2 * c[PK + 2] + k3 * c[PK + 3]) +
                        wz2 * (k0 * c[2 * PK] + k1 * c[2 * PK + 1] + k2 * c[2 * PK + 2] + k3 * c[2 * PK + 3]) +
                        wz3 * (k0 * c[3 * PK] + k1 * c[3 * PK + 1] + k2 * c[3 * PK + 2] + k3 * c[3 * PK + 3]);
            const T P = M::p10(T(0.25) * v);
            T vv[NB], tv[NB];
#pragma unroll
            for (int i = 0; i < NB; ++i) { vv[i] = V[i * N + n]; tv[i] = vv[i] * P; }
            int p = 0;
#pragma unroll
            for (int i = 0; i < NB; ++i)
#pragma unroll
                for (int jj = i; jj < NB; ++jj) { acc[p] += tv[i] * vv[jj]; ++p; }
        }
        const T mine = warp_transpose_sum16(acc);
        if (lane < NP) part[item * 16 + lane] = mine;
    }
    __syncthreads();
    for (int t = tid; t < NP * sp.n_ell; t += nt) {
        const int p = t / sp.n_ell, l = t % sp.n_ell;
        Cl[t] = part[(2 * l) * 16 + p] + part[(2 * l + 1) * 16 + p];
    }
    __syncthreads();

    // 5. data vector (1 + m_i)(1 + m_j) C_ij(ell) + T b; residual d - m
    for (int a = tid; a < sp.D; a += nt) {
        const int p = a / sp.n_ell, e = a % sp.n_ell;
        const int i = sp.pi[p], j = sp.pj[p];
        T m = (T(1) + th[11 + NB + i]) * (T(1) + th[11 + NB + j]) * Cl[p * sp.n_ell + e];
        for (int t = 0; t < sp.n_tmpl; ++t) m += (T)sp.tmpl[(size_t)a * sp.n_tmpl + t] * th[11 + 2 * NB + t];
        if (args.model_out) args.model_out[(size_t)row * sp.D + a] = (double)m;
        else args.resid[(size_t)row * sp.D + a] = (T)sp.data[a] - m;
    }
}

// Whitening Y = R L^-T over tiles of 16 rows x 64 columns (b <= a), the next
// 32-deep chunk of R and L^-T prefetched into registers while the current one
// is multiplied from shared memory; per-tile row sums of y^2.
constexpr int kWR = 16, kWC = 64, kWK = 32;

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
    const int tid = threadIdx.x, tx = tid & 31, ty = tid >> 5;   // ty: 8 row pairs
    const int b_end = min(D, a0 + kWC);
    // per-thread share of a chunk: R 16 x 32 = 512 (2 each), L 32 x 64 = 2048 (8 each)
    TA pr[2], pl[8];
    auto fetch = [&](int b0) {
#pragma unroll
        for (int q = 0; q < 2; ++q) {
            const int idx = tid + 256 * q, r = idx / kWK, c = idx % kWK;
            pr[q] = (row0 + r < M && b0 + c < D) ? (TA)resid[(size_t)(row0 + r) * D + b0 + c] : TA(0);
        }
#pragma unroll
        for (int q = 0; q < 8; ++q) {
            const int idx = tid + 256 * q, bb = idx / kWC, aa = idx % kWC;
            pl[q] = (b0 + bb < D && a0 + aa < D) ? LinvT[(size_t)(b0 + bb) * D + a0 + aa] : TA(0);
        }
    };
    TA acc[2][2] = {{TA(0), TA(0)}, {TA(0), TA(0)}};
    fetch(0);
    for (int b0 = 0; b0 < b_end; b0 += kWK) {
#pragma unroll
        for (int q = 0; q < 2; ++q) { const int idx = tid + 256 * q; Rs[idx / kWK][idx % kWK] = pr[q]; }
#pragma unroll
        for (int q = 0; q < 8; ++q) { const int idx = tid + 256 * q; Ls[idx / kWC][idx % kWC] = pl[q]; }
        __syncthreads();
        if (b0 + kWK < b_end) fetch(b0 + kWK);
#pragma unroll 8
        for (int kk = 0; kk < kWK; ++kk) {
            const TA l0 = Ls[kk][tx], l1 = Ls[kk][tx + 32];
            const TA r0 = Rs[ty][kk], r1 = Rs[ty + 8][kk];
            acc[0][0] += r0 * l0; acc[0][1] += r0 * l1;
            acc[1][0] += r1 * l0; acc[1][1] += r1 * l1;
        }
        __syncthreads();
    }
#pragma unroll
    for (int i = 0; i < 2; ++i) {
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

size_t projection_smem_bytes(const ShearParams& sp, int elt, int elt_acc) {
    const int NP = sp.nb * (sp.nb + 1) / 2;
    const int usz = std::max(6 * sp.N, (sp.n_z + 2) * (sp.n_k + 2));
    (void)elt_acc;
    const size_t n = (size_t)(((2 + sp.nb) * sp.N + 3) & ~3) + ((usz + 3) & ~3) +
                     (size_t)std::max(kProjWarps * 32, sp.n_ell * 2 * 16) + (size_t)NP * sp.n_ell + sp.n_params + 96;
    return n * elt;
}

template <typename T, int NB, bool FAST>
static int launch_nb(const ProjArgs<T>& a, int grid_rows, cudaStream_t st) {
    const size_t smem = projection_smem_bytes(a.sp, sizeof(T), sizeof(T));
    if (smem > 227 * 1024) return NS_ENOTSUP;
    static bool attr_done = false;
    if (!attr_done) {
        NS_CUDA_TRY(cudaFuncSetAttribute(k_projection<T, NB, FAST>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                         227 * 1024));
        attr_done = true;
    }
    k_projection<T, NB, FAST><<<grid_rows, kProjThreads, smem, st>>>(a);
    NS_CUDA_TRY(cudaGetLastError());
    return NS_OK;
}

template <typename T, bool FAST>
int launch_projection(const ShearParams& sp, const double* theta_full, const T* table, T* resid, double* model_out,
                      const int* nrows, int grid_rows, cudaStream_t st) {
    ProjArgs<T> a{sp, theta_full, table, resid, model_out, nrows};
    switch (sp.nb) {
        case 1: return launch_nb<T, 1, FAST>(a, grid_rows, st);
        case 2: return launch_nb<T, 2, FAST>(a, grid_rows, st);
        case 3: return launch_nb<T, 3, FAST>(a, grid_rows, st);
        case 4: return launch_nb<T, 4, FAST>(a, grid_rows, st);
        case 5: return launch_nb<T, 5, FAST>(a, grid_rows, st);
        default: return NS_ENOTSUP;
    }
}
template int launch_projection<double, false>(const ShearParams&, const double*, const double*, double*, double*,
                                              const int*, int, cudaStream_t);
template int launch_projection<float, false>(const ShearParams&, const double*, const float*, float*, double*,
                                             const int*, int, cudaStream_t);
template int launch_projection<float, true>(const ShearParams&, const double*, const float*, float*, double*,
                                            const int*, int, cudaStream_t);

}  // namespace gpuns
