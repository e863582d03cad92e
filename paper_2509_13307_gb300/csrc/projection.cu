// The shear projection (App. A, rows A8-A12) and the whitened chi^2 (A13).
//
// k_windows: one CTA (8 warps) per likelihood evaluation; needs only theta,
// so it runs on a second stream beside the emulator.
//   1. background: E(a) at the nodes; chi increments over each a-interval by a
//      4-point Gauss-Legendre rule and a block prefix sum (chi_0 = 0 at a = 1);
//      growth ln D = -sum trapezoid(Omega_m(a)^gamma) dln a by a second scan.
//   2. windows: per bin the shifted Gaussian n_i(z - D_z,i), normalised on the
//      grid; W^gamma (Eq. 5) = A (chi/a) [S0 - chi S1] with exclusive suffix
//      sums S0 = sum_{m>n} w n, S1 = sum_{m>n} w n / chi (the m = n term of the
//      direct double sum is zero); W^I (Eq. 6); V_i = sqrt(w/chi^2) W^eps_i.
//      ln chi and V go to a per-evaluation buffer.
// k_limber: one CTA per (evaluation, group of 4 multipoles).
//   3. the emulator's log10 P table (n_z x n_k) and the evaluation's windows
//      are staged in shared memory by bulk (TMA) copies, so the 16 taps of
//      every lookup and the node data hit shared memory.
//   4. Limber (Eq. 3-4): lanes own chi nodes; per node the Catmull-Rom lookup
//      at ln k = ln(ell + 1/2) - ln chi for two multipoles at once (packed
//      FP32x2 arithmetic) and the pair sums V_i V_j P.  A transposed warp
//      reduction, then a fixed-order sum over warps (deterministic).
//   5. data vector (1 + m_i)(1 + m_j) C_ij(ell) + T b and residual d - m.
// k_whiten: Y = R L^-T for blocks of rows, the 64-column tiles (b <= a) of a
//   row block split over the CTAs of a thread-block cluster; rank 0 adds the
//   ranks' row sums of y^2 in fixed order and writes log L = c0 - chi^2 / 2
//   in FP64.
#include <algorithm>

#include <cooperative_groups.h>

#include "likelihood.cuh"
#include "async_copy.cuh"

namespace gpuns {

namespace cg = cooperative_groups;

// 4-point Gauss-Legendre nodes and weights on [-1, 1] as compile-time
// constants of the kernel's own type (no double -> float conversions at run
// time).
template <typename T> __device__ __forceinline__ T gl4_x(int g) {
    return g == 0 ? T(-0.86113631159405257522) : g == 1 ? T(-0.33998104358485626480)
         : g == 2 ? T(0.33998104358485626480) : T(0.86113631159405257522);
}
template <typename T> __device__ __forceinline__ T gl4_w(int g) {
    return (g == 0 || g == 3) ? T(0.34785484513745385737) : T(0.65214515486254614263);
}

template <typename T> __device__ __forceinline__ const T* pick(const double* d, const float* f);
template <> __device__ __forceinline__ const double* pick<double>(const double* d, const float*) { return d; }
template <> __device__ __forceinline__ const float* pick<float>(const double*, const float* f) { return f; }
template <typename T> __device__ __forceinline__ T pick_s(double d, float f);
template <> __device__ __forceinline__ double pick_s<double>(double d, float) { return d; }
template <> __device__ __forceinline__ float pick_s<float>(double, float f) { return f; }

// Transcendentals: accurate library versions, or (FAST, BF16 modes) the SFU
// approximations, whose ~1e-6 relative error is far below the bf16 emulator's.
template <typename T, bool FAST> struct Math;
// div / rsq: IEEE quotient and 1/sqrt, or (FAST) the SFU reciprocal forms.
template <> struct Math<double, false> {
    static __device__ __forceinline__ double ex(double x) { return exp(x); }
    static __device__ __forceinline__ double lg(double x) { return log(x); }
    static __device__ __forceinline__ double p10(double v) { return exp(v * kLn10); }
    static __device__ __forceinline__ double div(double a, double b) { return a / b; }
    static __device__ __forceinline__ double rsq(double x) { return 1.0 / sqrt(x); }
};
template <> struct Math<float, false> {
    static __device__ __forceinline__ float ex(float x) { return expf(x); }
    static __device__ __forceinline__ float lg(float x) { return logf(x); }
    static __device__ __forceinline__ float p10(float v) { return exp2f(v * 3.32192809488736234787f); }
    static __device__ __forceinline__ float e2(float v) { return exp2f(v); }
    static __device__ __forceinline__ float div(float a, float b) { return a / b; }
    static __device__ __forceinline__ float rsq(float x) { return 1.f / sqrtf(x); }
};
template <> struct Math<float, true> {
    static __device__ __forceinline__ float ex(float x) { return __expf(x); }
    static __device__ __forceinline__ float lg(float x) { return __logf(x); }
    static __device__ __forceinline__ float div(float a, float b) { return __fdividef(a, b); }
    static __device__ __forceinline__ float rsq(float x) { return rsqrtf(x); }
    static __device__ __forceinline__ float p10(float v) {
        float y;
        asm("ex2.approx.ftz.f32 %0, %1;" : "=f"(y) : "f"(v * 3.32192809488736234787f));
        return y;
    }
    static __device__ __forceinline__ float e2(float v) {
        float y;
        asm("ex2.approx.ftz.f32 %0, %1;" : "=f"(y) : "f"(v));
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


// Stage A (per evaluation): distances, growth and windows.  Writes, per row,
// ln chi and V_i = sqrt(w / chi^2) W^eps_i, (NB + 1) vectors of pitch
// win_pitch(N) (16-byte multiples, for the Limber stage's bulk copy), to `win`.
__host__ __device__ inline int win_pitch(int N) { return (N + 3) & ~3; }

template <typename T, int NB, bool FAST>
__global__ void __launch_bounds__(kProjThreads)
k_windows(const ShearParams sp, const double* __restrict__ theta_full, T* __restrict__ win,
          const int* __restrict__ nrows) {
    using M = Math<T, FAST>;
    const int row = blockIdx.x;
    if (row >= *nrows) return;
    extern __shared__ __align__(16) unsigned char smem_raw[];
    const int N = sp.N;
    T* chi = reinterpret_cast<T*>(smem_raw);
    T* lnchi = chi + N;
    T* V = lnchi + N;                          // NB x N
    T* U = V + NB * N;                         // 6 N scratch
    T* part = U + 6 * N;                       // warps x 32
    T* th = part + kProjWarps * 32;
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
    (void)lane;

    for (int i = tid; i < sp.n_params; i += nt) th[i] = (T)theta_full[(size_t)row * sp.n_params + i];
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
                const T ag = mid + half * gl4_x<T>(g);
                const T lg = M::lg(ag);
                const T ia = M::div(T(1), ag);
                const T eg = om * ia * ia * ia + (T(1) - om) * M::ex(-pde * lg - T(3) * wa * (T(1) - ag));
                inc += gl4_w<T>(g) * ia * ia * M::rsq(eg);
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
        const T oma = M::div(om * M::ex(T(-3) * lna_[n]), Ez[n] * Ez[n]);
        t1[n] = M::ex(gamma * M::lg(oma));
        omw[n] = M::div(wa_[n] * chiH, a_[n] * a_[n] * Ez[n]);
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
    const T* nz_mu = pick<T>(sp.nz_mean, sp.nz_mean_f);
    const T* nz_sg = pick<T>(sp.nz_sigma, sp.nz_sigma_f);
    T zc[NB], isg[NB];
#pragma unroll
    for (int i = 0; i < NB; ++i) {
        zc[i] = th[11 + i] + nz_mu[i];
        isg[i] = M::div(T(1), nz_sg[i]);
    }
    for (int n = tid; n < N; n += nt) {
        const T wz = M::div(wa_[n], a_[n] * a_[n]);
#pragma unroll
        for (int i = 0; i < NB; ++i) {
            const T u = FAST ? (z_[n] - zc[i]) * isg[i] : (z_[n] - th[11 + i] - nz_mu[i]) / nz_sg[i];
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
        const T ichi = (FAST && n >= 1) ? M::div(T(1), chi[n]) : T(0);
#pragma unroll
        for (int i = 0; i < NB; ++i) {
            const T nchi = V[i * N + n] * e * inv_norm[i];
            V[i * N + n] = nchi;
            if (n >= 1) {
                const T wn = omw[n] * nchi;
                s0[i] += wn;
                s1[i] += FAST ? wn * ichi : wn / chi[n];
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
    const T pivot = pick_s<T>(sp.ia_pivot, sp.ia_pivot_f), c1rho = pick_s<T>(sp.c1rho, sp.c1rho_f);
    const T ipiv = M::div(T(1), pivot);
    const T c1om = c1rho * om;
    for (int n = hi - 1; n >= lo; --n) {
        const T c = chi[n];
        const T ic = (FAST && n >= 1) ? M::div(T(1), c) : T(0);
        const T sq = (n >= 1) ? (FAST ? sqrt_<T>(omw[n]) * ic : sqrt_<T>(omw[n] / (c * c))) : T(0);
        const T amp = FAST ? M::div(A_IA * M::ex(eta * M::lg((T(1) + z_[n]) * ipiv)) * c1om, Dg[n])
                           : A_IA * M::ex(eta * M::lg((T(1) + z_[n]) / pivot)) * c1rho * om / Dg[n];
        const T pc = FAST ? pref * c * M::div(T(1), a_[n]) : pref * c / a_[n];
#pragma unroll
        for (int i = 0; i < NB; ++i) {
            const T nchi = V[i * N + n];
            T v = T(0);
            if (n >= 1) {
                v = sq * (pc * (e0[i] - c * e1[i]) - amp * nchi);
                const T wn = omw[n] * nchi;
                e0[i] += wn;
                e1[i] += FAST ? wn * ic : wn / c;
            }
            V[i * N + n] = v;
        }
    }
    __syncthreads();

    // write ln chi and V for the Limber stage
    const int Np = win_pitch(N);
    T* out = win + (size_t)row * (NB + 1) * Np;
    for (int n = tid; n < N; n += nt) out[n] = lnchi[n];
    for (int i = 0; i < NB; ++i)
        for (int n = tid; n < N; n += nt) out[(i + 1) * Np + n] = V[i * N + n];
}

// Stage B: Limber sums, one CTA per evaluation.  The CTA stages the
// evaluation's log10 P table in shared memory with bulk (TMA) row copies
// (issued by the lanes of warp 0 in parallel), then adds ghost rows/columns by
// linear extrapolation.  Padded layout: row r + 1 holds z row r, data column k
// sits at padded column k + 4 (16-byte aligned rows for the copies), ghosts at
// columns 3 and n_k + 4; the row pitch PK is a multiple of 4 chosen so that
// the 4-word tap windows of up to 8 consecutive rows fall in distinct banks.
// Warp w takes multipole pairs (2 w, 2 w + 1), (2 (w + nw), ...), each lane
// walking chi nodes (node z-taps, ln chi and the windows from the stage-A
// output), doing the Catmull-Rom lookup and the pair sums; a transposed warp
// reduction leaves lane q with pair sum q, and that lane forms the data-vector
// entry (1 + m_i)(1 + m_j) C_ij(ell) + T b and writes the residual d - m (or
// the model).  The sums are in fixed order (deterministic).
constexpr int kLimberWarps = 10;

__host__ __device__ inline int limber_pitch(int n_k) {
    int pk = (n_k + 5 + 3) & ~3;
    if ((pk & 31) == 0 || (pk & 31) == 16) pk += 4;
    return pk;
}

// FP32 Limber inner loop for the multipole pair (ell0, ell1) of a warp: the two
// lookups and their pair sums run as packed f32x2 arithmetic (one FFMA2 per
// two FMAs).  Nodes n0, n0 + stride, ...; acc[p] / acc[NP + p] receive the pair
// sums of ell0 / ell1.  With a single multipole left, ell1 = ell0 and the
// second half is discarded by the caller.  The node constants come from shared
// memory: zoff[n] = offset of the node's first z-tap row (+ the 3 ghost/pad
// columns) in the padded table, zw[n] = its four doubled z-weights.  With a
// compile-time row pitch PKC the four tap rows sit at immediate offsets.
template <int NB, bool FAST, int PKC>
__device__ __forceinline__ void limber_pair_f32(const float* __restrict__ U, int PKr, int N, int n_k,
                                                const int* __restrict__ zoff, const float4* __restrict__ zw,
                                                const float* __restrict__ lnchi, const float* __restrict__ V,
                                                int Np, float lne0, float lne1, float lkmin, float lkmax,
                                                float inv_dk, int n0, int stride, float* acc) {
    using M = Math<float, FAST>;
    const int PK = PKC ? PKC : PKr;
    constexpr int NP = NB * (NB + 1) / 2;
    const float2 one = make_float2(1.f, 1.f), m1 = make_float2(-1.f, -1.f), two = make_float2(2.f, 2.f);
    const float2 three = make_float2(3.f, 3.f), m3 = make_float2(-3.f, -3.f), four = make_float2(4.f, 4.f);
    const float2 m5 = make_float2(-5.f, -5.f);
    const float gmax = 8388608.f + (float)(n_k - 2);
    const float umax = (lkmax - lkmin) * inv_dk;
    // table coordinate u = (ln(ell + 1/2) - ln chi - lnk_min) / dlnk of both
    // multipoles as one FFMA2: u = a - ln chi / dlnk
    const float2 ua = make_float2((lne0 - lkmin) * inv_dk, (lne1 - lkmin) * inv_dk);
    const float2 minv = make_float2(-inv_dk, -inv_dk);
    const float2 half = make_float2(8388607.5f, 8388607.5f), p23 = make_float2(8388608.f, 8388608.f);
    float2 a2[NP];
#pragma unroll
    for (int p = 0; p < NP; ++p) a2[p] = make_float2(0.f, 0.f);
    // two nodes per trip: independent lookups interleave (same per-lane order)
#pragma unroll 2
    for (int n = n0; n < N; n += stride) {
        const float* rz = U + zoff[n];
        const float4 wz = zw[n];
        const float lc = lnchi[n];
        float2 vv[NB];
#pragma unroll
        for (int i = 0; i < NB; ++i) { const float x = V[i * Np + n]; vv[i] = make_float2(x, x); }
        // ln k clamped to the table (u to [0, n_k - 1])
        float2 u = __ffma2_rn(make_float2(lc, lc), minv, ua);
        u.x = fminf(fmaxf(u.x, 0.f), umax);
        u.y = fminf(fmaxf(u.y, 0.f), umax);
        // cell index without conversion instructions: g = u + (2^23 - 1/2),
        // correctly rounded, is 2^23 + round(u - 1/2), an integer held in the
        // low mantissa bits (u >= 0, so g >= 2^23).  round(u - 1/2) = floor(u)
        // except at exact integers, where the cell below with t = 1 gives the
        // same interpolant.  The clamp to cell n_k - 2 is taken on g (exact).
        float2 g = __fadd2_rn(u, half);
        g.x = fminf(g.x, gmax);
        g.y = fminf(g.y, gmax);
        const int ik0 = __float_as_int(g.x) - 0x4B000000;
        const int ik1 = __float_as_int(g.y) - 0x4B000000;
        // t = u - (g - 2^23); 2^23 - g is exact (Sterbenz) and so is the sum
        const float2 t = __fadd2_rn(u, __ffma2_rn(g, m1, p23));
        const float2 t2 = __fmul2_rn(t, t);
        // doubled Catmull-Rom weights (the z-taps are doubled too)
        const float2 k0 = __fmul2_rn(t, __ffma2_rn(t, __ffma2_rn(t, m1, two), m1));
        const float2 k1 = __ffma2_rn(t2, __ffma2_rn(three, t, m5), two);
        const float2 k2 = __fmul2_rn(t, __ffma2_rn(t, __ffma2_rn(m3, t, four), one));
        const float2 k3 = __fmul2_rn(t2, __fadd2_rn(t, m1));
        const float* c0 = rz + ik0;
        const float* c1 = rz + ik1;
        const float wzr[4] = {wz.x, wz.y, wz.z, wz.w};
        float2 v;
#pragma unroll
        for (int r = 0; r < 4; ++r) {
            const int o = r * PK;
            float2 sr = __fmul2_rn(k0, make_float2(c0[o], c1[o]));
            sr = __ffma2_rn(k1, make_float2(c0[o + 1], c1[o + 1]), sr);
            sr = __ffma2_rn(k2, make_float2(c0[o + 2], c1[o + 2]), sr);
            sr = __ffma2_rn(k3, make_float2(c0[o + 3], c1[o + 3]), sr);
            const float2 w = make_float2(wzr[r], wzr[r]);
            v = (r == 0) ? __fmul2_rn(w, sr) : __ffma2_rn(w, sr, v);
        }
        // the z-weights carry the factor log2(10) / 4 (doubled k- and z-weights):
        // P = 10^(log10 P) = 2^v
        const float2 P = make_float2(M::e2(v.x), M::e2(v.y));
        float2 tv[NB];
#pragma unroll
        for (int i = 0; i < NB; ++i) tv[i] = __fmul2_rn(vv[i], P);
        int p = 0;
#pragma unroll
        for (int i = 0; i < NB; ++i)
#pragma unroll
            for (int j = i; j < NB; ++j) { a2[p] = __ffma2_rn(tv[i], vv[j], a2[p]); ++p; }
    }
#pragma unroll
    for (int p = 0; p < NP; ++p) { acc[p] = a2[p].x; acc[NP + p] = a2[p].y; }
}

template <typename T, int NB, bool FAST, int PKC>
__global__ void __launch_bounds__(32 * kLimberWarps, sizeof(T) == 8 ? 1 : 2)
k_limber(const ShearParams sp, const double* __restrict__ theta_full, const T* __restrict__ table,
         const T* __restrict__ win, T* __restrict__ resid, double* __restrict__ model_out,
         const int* __restrict__ nrows, int* __restrict__ err) {
    using M = Math<T, FAST>;
    constexpr int NP = NB * (NB + 1) / 2;
    static_assert(2 * NP <= 32, "two multipoles of pair sums must fit one warp transpose");
    // Only the emulator table comes from the preceding kernel (programmatic
    // dependency).  The row count and parameters (slice kernel) and the
    // windows (side stream) reach this kernel through the likelihood's
    // fork / join events, full dependencies: they are staged before the wait.
    const int row = blockIdx.x;
    if (row >= *nrows) return;
    extern __shared__ __align__(16) unsigned char smem_raw[];
    __shared__ __align__(8) uint64_t s_bar;
    const int N = sp.N, n_k = sp.n_k, n_z = sp.n_z, n_ell = sp.n_ell;
    const int PK = PKC ? PKC : limber_pitch(n_k);
    const int Np = win_pitch(N);
    T* U = reinterpret_cast<T*>(smem_raw);          // padded table
    T* W = U + (n_z + 2) * PK;                      // ln chi, V_1..V_NB (pitch Np)
    // FP32: the nodes' z-weights (float4) and first-tap offsets, staged once per CTA
    float4* ZW = reinterpret_cast<float4*>(W + (NB + 1) * Np);
    int* ZO = reinterpret_cast<int*>(ZW + (sizeof(T) == 4 ? N : 0));
    T* thr = reinterpret_cast<T*>(ZO + (sizeof(T) == 4 ? N : 0));   // the row's parameters in T (n_params)
    const int tid = threadIdx.x, nt = blockDim.x;
    const int lane = tid & 31, wid = tid >> 5, nw = nt >> 5;
    const int n_lp = (n_ell + 1) / 2;               // multipole pairs, one warp each
    const T* src = table + (size_t)row * n_z * n_k;
    const T* wsrc = win + (size_t)row * (NB + 1) * Np;
    const uint32_t row_bytes = (uint32_t)(n_k * sizeof(T));
    const uint32_t win_bytes = (uint32_t)((NB + 1) * Np * sizeof(T));
    const bool bulk = (row_bytes % 16) == 0 && (reinterpret_cast<uintptr_t>(src) & 15) == 0 &&
                      (reinterpret_cast<uintptr_t>(wsrc) & 15) == 0;
    auto stage_nodes = [&]() {
        if constexpr (sizeof(T) == 4) {
            const float4* zsrc = reinterpret_cast<const float4*>(sp.zw4f);
            // z-weights scaled by log2(10) / 4 so the lookup yields log2 P directly
            constexpr float c = 0.25f * 3.32192809488736234787f;
            for (int n = tid; n < N; n += nt) {
                const float4 q = zsrc[n];
                ZW[n] = make_float4(c * q.x, c * q.y, c * q.z, c * q.w);
                ZO[n] = sp.zrp[n] * PK + 3;
            }
        }
    };
    // every output of the row is NaN when a bounded wait gives up
    auto fail_row = [&]() {
        if (tid == 0 && err) atomicOr(err, NS_BIT_TIMEOUT);
        for (int a = tid; a < sp.D; a += nt) {
            if (model_out) model_out[(size_t)row * sp.D + a] = NAN;
            else resid[(size_t)row * sp.D + a] = (T)NAN;
        }
    };
    if (bulk) {
        const uint32_t bar = smem_u32(&s_bar);
        if (tid == 0) {
            mbar_init(bar, 1);
            mbar_init_fence();
        }
        __syncthreads();
        // one arrival with the whole transaction count and the windows copy;
        // the table's row copies (lanes of warp 0 in parallel) after the wait
        if (wid == 0 && lane == 0) {
            mbar_expect_tx(bar, row_bytes * n_z + win_bytes);
            bulk_g2s(smem_u32(W), wsrc, win_bytes, bar);
        }
        for (int i = tid; i < sp.n_params; i += nt) thr[i] = (T)theta_full[(size_t)row * sp.n_params + i];
        stage_nodes();
        pdl_begin();
        if (wid == 0) {
            __syncwarp();
            for (int r = lane; r < n_z; r += 32)
                bulk_g2s(smem_u32(U + (r + 1) * PK + 4), src + (size_t)r * n_k, row_bytes, bar);
        }
        // warp 0 polls the barrier while the others sleep at the CTA barrier;
        // afterwards every thread observes the completed phase (acquire).
        int fail = 0;
        if (wid == 0) fail = !mbar_wait(bar, 0);
        if (!__syncthreads_or(fail)) mbar_try_wait(bar, 0);
        else {
            // give copies still in flight a second bounded wait before leaving
            if (wid == 0) mbar_wait(bar, 0);
            __syncthreads();
            fail_row();
            return;
        }
    } else {
        for (int i = tid; i < (NB + 1) * Np; i += nt) W[i] = wsrc[i];
        for (int i = tid; i < sp.n_params; i += nt) thr[i] = (T)theta_full[(size_t)row * sp.n_params + i];
        stage_nodes();
        pdl_begin();
        for (int r = wid; r < n_z; r += nw)
            for (int k = lane; k < n_k; k += 32) U[(r + 1) * PK + 4 + k] = src[(size_t)r * n_k + k];
        __syncthreads();
    }
    for (int k = 4 + tid; k < 4 + n_k; k += nt) {
        U[k] = T(2) * U[PK + k] - U[2 * PK + k];
        U[(n_z + 1) * PK + k] = T(2) * U[n_z * PK + k] - U[(n_z - 1) * PK + k];
    }
    __syncthreads();
    for (int r = tid; r < n_z + 2; r += nt) {
        U[r * PK + 3] = T(2) * U[r * PK + 4] - U[r * PK + 5];
        U[r * PK + n_k + 4] = T(2) * U[r * PK + n_k + 3] - U[r * PK + n_k + 2];
    }
    __syncthreads();
    const T lkmin = pick_s<T>(sp.lnk_min, sp.lnk_min_f), lkmax = pick_s<T>(sp.lnk_max, sp.lnk_max_f);
    const T inv_dk = pick_s<T>(1.0 / sp.dlnk, sp.inv_dlnk_f);
    const int* zrp = sp.zrp;
    const T* zwp = pick<T>(sp.zw4d, sp.zw4f);
    const T* lnchi = W;
    const T* V = W + Np;
    const T* lnell = pick<T>(sp.lnell, sp.lnell_f);
    const T* tm = pick<T>(sp.tmpl, sp.tmpl_f);
    const T* dat = pick<T>(sp.data, sp.data_f);
    for (int lp = wid; lp < n_lp; lp += nw) {
        const int l0 = 2 * lp;
        const bool has1 = l0 + 1 < n_ell;
        const T lne0 = lnell[l0], lne1 = has1 ? lnell[l0 + 1] : lne0;
        T acc[32];
#pragma unroll
        for (int q = 0; q < 32; ++q) acc[q] = T(0);
        if constexpr (sizeof(T) == 4) {
            limber_pair_f32<NB, FAST, PKC>(U, PK, N, n_k, ZO, ZW,
                                      reinterpret_cast<const float*>(lnchi), reinterpret_cast<const float*>(V), Np,
                                      (float)lne0, (float)lne1, (float)lkmin, (float)lkmax, (float)inv_dk, 1 + lane,
                                      32, reinterpret_cast<float*>(acc));
        } else {
            for (int n = 1 + lane; n < N; n += 32) {
                const T* rz = U + zrp[n] * PK + 3;
                const T wz0 = zwp[4 * n], wz1 = zwp[4 * n + 1], wz2 = zwp[4 * n + 2], wz3 = zwp[4 * n + 3];
                const T lc = lnchi[n];
                T vv[NB];
#pragma unroll
                for (int i = 0; i < NB; ++i) vv[i] = V[i * Np + n];
#pragma unroll
                for (int j = 0; j < 2; ++j) {
                    if (j == 1 && !has1) break;
                    T sk = (j == 0 ? lne0 : lne1) - lc;
                    sk = fmin(fmax(sk, lkmin), lkmax);
                    const T uk = (sk - lkmin) * inv_dk;
                    int ik = (int)floor(uk);
                    ik = min(max(ik, 0), n_k - 2);
                    const T t = uk - (T)ik, t2 = t * t;
                    // doubled Catmull-Rom weights (the z-taps are doubled too)
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
                    T tv[NB];
#pragma unroll
                    for (int i = 0; i < NB; ++i) tv[i] = vv[i] * P;
                    int p = 0;
#pragma unroll
                    for (int i = 0; i < NB; ++i)
#pragma unroll
                        for (int jj = i; jj < NB; ++jj) { acc[j * NP + p] += tv[i] * vv[jj]; ++p; }
                }
            }
        }
        // lane q < 2 NP ends with the sum of value q: multipole l0 + q / NP, pair q % NP
        const T cl = warp_transpose_sum(acc);
        const int l = l0 + lane / NP, p = lane % NP;
        if (lane < 2 * NP && l < n_ell) {
            // data vector (1 + m_i)(1 + m_j) C_ij(ell) + T b; residual d - m
            const int a = p * n_ell + l;
            T m = (T(1) + thr[11 + NB + sp.pi[p]]) * (T(1) + thr[11 + NB + sp.pj[p]]) * cl;
            for (int t = 0; t < sp.n_tmpl; ++t) m += tm[(size_t)a * sp.n_tmpl + t] * thr[11 + 2 * NB + t];
            if (model_out) model_out[(size_t)row * sp.D + a] = (double)m;
            else resid[(size_t)row * sp.D + a] = dat[a] - m;
        }
    }
}

// Whitening Y = R L^-T for a block of WR rows (16; the kernel also takes
// 8).  The ntile column tiles of 64 (b <= a) are split over the cs
// CTAs of a cluster (rank q takes tiles q, q + cs, ...).  Per tile the
// reduction range (rounded up to 32, zero-filled) is staged in shared memory
// with 16-byte cp.async copies, in as few chunks as fit; the 8 warps split it
// (warp w takes the w-th eighth), each lane accumulating WR rows x 2 columns
// (one packed FP32x2 FMA per row and k in FP32), with the four R values of a
// row read as one vector.  The warps' partial tiles are added in warp order
// and the squares of y of a row in a fixed lane tree; warp r keeps row r's
// sum over the CTA's tiles in tile order; rank 0 adds the ranks' sums in rank
// order (cluster shared memory) and writes log L = c0 - chi^2 / 2.
constexpr int kWC = 64, kWarps = 8, kWClusterMax = 8;

__device__ __forceinline__ void cp_async16(void* dst, const void* src) {
    asm volatile("cp.async.cg.shared.global [%0], [%1], 16;" ::"r"((uint32_t)__cvta_generic_to_shared(dst)), "l"(src)
                 : "memory");
}
__device__ __forceinline__ void cp_async4(void* dst, const void* src) {
    asm volatile("cp.async.ca.shared.global [%0], [%1], 4;" ::"r"((uint32_t)__cvta_generic_to_shared(dst)), "l"(src) : "memory");
}
__device__ __forceinline__ void cp_async8(void* dst, const void* src) {
    asm volatile("cp.async.ca.shared.global [%0], [%1], 8;" ::"r"((uint32_t)__cvta_generic_to_shared(dst)), "l"(src) : "memory");
}
__device__ __forceinline__ void cp_async_wait_all() { asm volatile("cp.async.wait_all;" ::: "memory"); }

template <typename T>
__device__ __forceinline__ void cp_async_elt(T* dst, const T* src) {
    if (sizeof(T) == 4) cp_async4(dst, src); else cp_async8(dst, src);
}

// four consecutive values (16-byte aligned for float, 16-byte aligned pairs for double)
__device__ __forceinline__ void ld4(const float* p, float (&v)[4]) {
    const float4 q = *reinterpret_cast<const float4*>(p);
    v[0] = q.x; v[1] = q.y; v[2] = q.z; v[3] = q.w;
}
__device__ __forceinline__ void ld4(const double* p, double (&v)[4]) {
    const double2 q0 = *reinterpret_cast<const double2*>(p), q1 = *reinterpret_cast<const double2*>(p + 2);
    v[0] = q0.x; v[1] = q0.y; v[2] = q1.x; v[3] = q1.y;
}

template <typename TR, typename TA, int WR>
__global__ void __launch_bounds__(256)
k_whiten(const TR* __restrict__ resid, int D, const TA* __restrict__ LinvT, int ntile, int KC, double c0,
         double* __restrict__ logL, const int* __restrict__ nrows, int rows_ready) {
    static_assert(WR == 8 || WR == 16, "8 or 16 rows per block");
    // rows_ready: the row count (slice kernel) reaches this kernel through
    // the shear likelihood's fork / join events (full dependencies), so it is
    // read, and the first tile's first chunk of the constant L^-T requested,
    // before the dependency wait; the residuals (the preceding kernel's
    // output) always after it.
    const int row0 = blockIdx.y * WR;
    int M = 0;
    if (rows_ready) {
        M = *nrows;
        if (row0 >= M) return;                     // every CTA of the cluster has this row block
    }
    cg::cluster_group cluster = cg::this_cluster();
    const int cs = (int)cluster.num_blocks(), rank = (int)cluster.block_rank();
    extern __shared__ __align__(16) unsigned char smem_raw[];
    TA* Ls = reinterpret_cast<TA*>(smem_raw);                 // KC x kWC
    TR* Rs = reinterpret_cast<TR*>(Ls + (size_t)KC * kWC);    // WR x KC
    TA* red = Ls;                                             // kWarps x WR x kWC, after a tile's last chunk
    __shared__ TA s_rank_sum[kWClusterMax][WR];               // rank 0: the ranks' row sums
    const int tid = threadIdx.x, lane = tid & 31, wid = tid >> 5;
    const bool vecL = (D * sizeof(TA)) % 16 == 0 && (reinterpret_cast<uintptr_t>(LinvT) & 15) == 0;
    const bool vecR = (D * sizeof(TR)) % 16 == 0 && (reinterpret_cast<uintptr_t>(resid) & 15) == 0;
    // rows handled by this thread in the per-tile finish: WR = 8: warp w -> row w,
    // two columns per lane; WR = 16: half-warps -> rows, four columns per lane
    constexpr int TPR = 256 / WR;                  // threads per row (32 or 16)
    constexpr int CPT = kWC / TPR;                 // columns per thread (2 or 4)
    const int fr = tid / TPR, fc = (tid % TPR) * CPT;
    // L^-T rows k0 .. k0 + len of the tile at column a0 (zero beyond b_end and beyond column D)
    auto stage_L = [&](int a0, int b_end, int k0, int len) {
        const int lv = max(0, min(len, b_end - k0));
        if (vecL) {
            constexpr int per = 16 / sizeof(TA), vpr = kWC / per;
            for (int q = tid; q < len * vpr; q += 256) {
                const int bb = q / vpr, v = q % vpr;
                TA* dst = Ls + bb * kWC + v * per;
                if (bb < lv && a0 + v * per < D) cp_async16(dst, LinvT + (size_t)(k0 + bb) * D + a0 + v * per);
                else for (int e = 0; e < per; ++e) dst[e] = TA(0);
            }
        } else {
            for (int q = tid; q < len * kWC; q += 256) {
                const int bb = q / kWC, aa = q % kWC;
                if (bb < lv && a0 + aa < D) cp_async_elt(Ls + bb * kWC + aa, LinvT + (size_t)(k0 + bb) * D + a0 + aa);
                else Ls[bb * kWC + aa] = TA(0);
            }
        }
    };
    bool prefetched = false;
    if (rows_ready && rank < ntile) {
        const int a0 = rank * kWC, b_end = min(D, a0 + kWC);
        stage_L(a0, b_end, 0, min(KC, (b_end + 31) & ~31));
        prefetched = true;
    }
    pdl_begin();
    if (!rows_ready) {
        M = *nrows;
        if (row0 >= M) return;                     // every CTA of the cluster has this row block
    }
    TA run = TA(0);                                // row fr: sum of y^2 over this CTA's tiles
    for (int tile = rank; tile < ntile; tile += cs) {
        const int a0 = tile * kWC;
        const int b_end = min(D, a0 + kWC);
        const int Kp = (b_end + 31) & ~31;
        TA acc[WR][2];
#pragma unroll
        for (int r = 0; r < WR; ++r) { acc[r][0] = TA(0); acc[r][1] = TA(0); }
        for (int k0 = 0; k0 < Kp; k0 += KC) {
            const int len = min(KC, Kp - k0);          // multiple of 32
            const int lv = max(0, min(len, b_end - k0)); // rows holding data
            if (prefetched) prefetched = false;        // this chunk's L^-T is already in flight
            else {
                __syncthreads();                       // previous chunk / tile finish done with Ls, Rs
                stage_L(a0, b_end, k0, len);
            }
            // R rows row0 .. row0 + WR, columns k0 .. k0 + len (zero beyond b_end / M)
            if (vecR) {
                constexpr int per = 16 / sizeof(TR);
                const int vpr = len / per;
                for (int q = tid; q < WR * vpr; q += 256) {
                    const int rr = q / vpr, v = q % vpr;
                    TR* dst = Rs + rr * KC + v * per;
                    if (row0 + rr < M && v * per < lv) cp_async16(dst, resid + (size_t)(row0 + rr) * D + k0 + v * per);
                    else for (int e = 0; e < per; ++e) dst[e] = TR(0);
                }
            } else {
                for (int q = tid; q < WR * len; q += 256) {
                    const int rr = q / len, cc = q % len;
                    if (row0 + rr < M && cc < lv) cp_async_elt(Rs + rr * KC + cc, resid + (size_t)(row0 + rr) * D + k0 + cc);
                    else Rs[rr * KC + cc] = TR(0);
                }
            }
            cp_async_wait_all();
            __syncthreads();
            const int kw = len / kWarps;               // multiple of 4
            const int kb = wid * kw;
            for (int k = kb; k < kb + kw; k += 4) {
                TA l0[4], l1[4];
#pragma unroll
                for (int j = 0; j < 4; ++j) { l0[j] = Ls[(k + j) * kWC + lane]; l1[j] = Ls[(k + j) * kWC + lane + 32]; }
#pragma unroll
                for (int r = 0; r < WR; ++r) {
                    TR rv[4];
                    ld4(Rs + r * KC + k, rv);
                    if constexpr (sizeof(TA) == 4) {
                        float2 a2 = make_float2(acc[r][0], acc[r][1]);
#pragma unroll
                        for (int j = 0; j < 4; ++j)
                            a2 = __ffma2_rn(make_float2((float)rv[j], (float)rv[j]), make_float2(l0[j], l1[j]), a2);
                        acc[r][0] = a2.x;
                        acc[r][1] = a2.y;
                    } else {
#pragma unroll
                        for (int j = 0; j < 4; ++j) {
                            acc[r][0] = fma((TA)rv[j], l0[j], acc[r][0]);
                            acc[r][1] = fma((TA)rv[j], l1[j], acc[r][1]);
                        }
                    }
                }
            }
        }
        __syncthreads();
#pragma unroll
        for (int r = 0; r < WR; ++r) {
            red[(wid * WR + r) * kWC + lane] = acc[r][0];
            red[(wid * WR + r) * kWC + lane + 32] = acc[r][1];
        }
        __syncthreads();
        TA sq = TA(0);
#pragma unroll
        for (int e = 0; e < CPT; ++e) {
            TA y = TA(0);
#pragma unroll
            for (int w = 0; w < kWarps; ++w) y += red[(w * WR + fr) * kWC + fc + e];
            if (a0 + fc + e < D) sq += y * y;
        }
#pragma unroll
        for (int o = TPR / 2; o > 0; o >>= 1) sq += __shfl_xor_sync(0xffffffffu, sq, o, TPR);
        run += sq;
    }
    // rank 0 collects the ranks' row sums in its shared memory
    if (tid % TPR == 0) {
        TA* dst = cluster.map_shared_rank(&s_rank_sum[0][0], 0);
        dst[rank * WR + fr] = run;
    }
    cluster.sync();
    if (rank == 0 && tid < WR && row0 + tid < M) {
        TA s2 = TA(0);
        for (int q = 0; q < cs; ++q) s2 += s_rank_sum[q][tid];
        logL[row0 + tid] = c0 - 0.5 * (double)s2;
    }
}

template <typename TR, typename TA>
static size_t whiten_smem(int KC, int WR) {
    return std::max((size_t)KC * kWC * sizeof(TA) + (size_t)WR * KC * sizeof(TR),
                    (size_t)kWarps * WR * kWC * sizeof(TA));
}

template <typename TR, typename TA, int WR>
static int launch_whiten(const TR* resid, int D, const TA* LinvT, double c0, double* logL, const int* nrows,
                         int grid_rows, size_t smem_cap, cudaStream_t st, bool rows_ready) {
    const int ntile = (D + kWC - 1) / kWC;
    const int cs = std::min(ntile, kWClusterMax);
    // the whole (padded) reduction range in one chunk when it fits smem_cap
    const int Kp = (D + 31) & ~31;
    const size_t per_k = (size_t)kWC * sizeof(TA) + (size_t)WR * sizeof(TR);
    int KC = (int)std::min<size_t>((size_t)Kp, (smem_cap / per_k) & ~(size_t)31);
    KC = std::max(KC, 32);
    const size_t smem = whiten_smem<TR, TA>(KC, WR);
    static bool attr = false;
    if (!attr) {
        NS_CUDA_TRY(cudaFuncSetAttribute(k_whiten<TR, TA, WR>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                         227 * 1024 - 1024));
        attr = true;
    }
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = dim3(cs, (grid_rows + WR - 1) / WR);
    cfg.blockDim = dim3(256);
    cfg.dynamicSmemBytes = smem;
    cfg.stream = st;
    cudaLaunchAttribute attr2[2];
    attr2[0].id = cudaLaunchAttributeProgrammaticStreamSerialization;
    attr2[0].val.programmaticStreamSerializationAllowed = 1;
    attr2[1].id = cudaLaunchAttributeClusterDimension;
    attr2[1].val.clusterDim.x = cs;
    attr2[1].val.clusterDim.y = 1;
    attr2[1].val.clusterDim.z = 1;
    cfg.attrs = attr2;
    cfg.numAttrs = 2;
    NS_CUDA_TRY(cudaLaunchKernelEx(&cfg, k_whiten<TR, TA, WR>, resid, D, LinvT, ntile, KC, c0, logL, nrows,
                                   rows_ready ? 1 : 0));
    return NS_OK;
}

template <typename TR, typename TA>
int launch_chi2(const TR* resid, int D, const TA* LinvT, double c0, double* logL, const int* nrows, int grid_rows,
                cudaStream_t st, bool rows_ready) {
    // 16-row blocks.  Short data vectors: CTAs of up to ~100 KB (two per SM),
    // so the clusters of a ~460-row batch fit one wave (8-row blocks needed
    // 58 five-CTA clusters there, two waves: 114.7 -> 111.6 us per 39-d
    // nested-sampling round).  Long ones: the whole SM, half the passes over
    // L^-T of 8-row blocks.
    if ((D + kWC - 1) / kWC <= kWClusterMax)
        return launch_whiten<TR, TA, 16>(resid, D, LinvT, c0, logL, nrows, grid_rows, 100 * 1024, st, rows_ready);
    return launch_whiten<TR, TA, 16>(resid, D, LinvT, c0, logL, nrows, grid_rows, 200 * 1024, st, rows_ready);
}
template int launch_chi2<float, float>(const float*, int, const float*, double, double*, const int*, int,
                                       cudaStream_t, bool);
template int launch_chi2<float, double>(const float*, int, const double*, double, double*, const int*, int,
                                        cudaStream_t, bool);
template int launch_chi2<double, double>(const double*, int, const double*, double, double*, const int*, int,
                                         cudaStream_t, bool);

template <typename T>
static size_t windows_smem(const ShearParams& sp) {
    return ((size_t)(2 + sp.nb) * sp.N + 6 * (size_t)sp.N + kProjWarps * 32 + sp.n_params + 96) * sizeof(T);
}
// dynamic shared memory left beside the Limber kernel's static barrier
constexpr size_t kLimberSmemMax = 227 * 1024 - 64;
template <typename T>
static size_t limber_smem(const ShearParams& sp) {
    const size_t nodes = sizeof(T) == 4 ? (size_t)sp.N * (sizeof(float4) + sizeof(int)) : 0;
    return ((size_t)(sp.n_z + 2) * limber_pitch(sp.n_k) + (size_t)(sp.nb + 1) * win_pitch(sp.N) + sp.n_params) *
           sizeof(T) + nodes;
}

bool projection_fits(const ShearParams& sp, int elt) {
    const size_t lim = 227 * 1024;
    return elt == 8 ? (windows_smem<double>(sp) <= lim && limber_smem<double>(sp) <= kLimberSmemMax)
                    : (windows_smem<float>(sp) <= lim && limber_smem<float>(sp) <= kLimberSmemMax);
}

template <typename T, int NB, bool FAST>
static int windows_nb(const ShearParams& sp, const double* theta_full, T* win, const int* nrows, int grid_rows,
                      cudaStream_t st) {
    const size_t smem = windows_smem<T>(sp);
    if (smem > 227 * 1024) return NS_ENOTSUP;
    static bool attr_done = false;
    if (!attr_done) {
        NS_CUDA_TRY(cudaFuncSetAttribute(k_windows<T, NB, FAST>, cudaFuncAttributeMaxDynamicSharedMemorySize, 227 * 1024));
        attr_done = true;
    }
    k_windows<T, NB, FAST><<<grid_rows, kProjThreads, smem, st>>>(sp, theta_full, win, nrows);
    NS_CUDA_TRY(cudaGetLastError());
    return NS_OK;
}

template <typename T, int NB, bool FAST, int PKC>
static int limber_launch(const ShearParams& sp, const double* theta_full, const T* table, const T* win, T* resid,
                         double* model_out, const int* nrows, int grid_rows, int* err, cudaStream_t st) {
    const size_t smem = limber_smem<T>(sp);
    if (smem > kLimberSmemMax) return NS_ENOTSUP;
    static bool attr_done = false;
    if (!attr_done) {
        cudaFuncAttributes fa;
        NS_CUDA_TRY(cudaFuncGetAttributes(&fa, k_limber<T, NB, FAST, PKC>));
        NS_CUDA_TRY(cudaFuncSetAttribute(k_limber<T, NB, FAST, PKC>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                         (int)(227 * 1024 - fa.sharedSizeBytes)));
        attr_done = true;
    }
    const int warps = std::min(kLimberWarps, (sp.n_ell + 1) / 2);
    NS_CUDA_TRY(launch_pdl(k_limber<T, NB, FAST, PKC>, dim3(grid_rows), dim3(32 * warps), smem, st, sp, theta_full,
                           table, win, resid, model_out, nrows, err));
    return NS_OK;
}

// The 39-d table (200 k nodes, padded row pitch 212) gets a compile-time pitch.
constexpr int kPitch39 = 212;
static_assert(kPitch39 % 4 == 0, "padded rows stay 16-byte aligned");

template <typename T, int NB, bool FAST>
static int limber_nb(const ShearParams& sp, const double* theta_full, const T* table, const T* win, T* resid,
                     double* model_out, const int* nrows, int grid_rows, int* err, cudaStream_t st) {
    if constexpr (sizeof(T) == 4 && NB == 5) {
        if (limber_pitch(sp.n_k) == kPitch39)
            return limber_launch<T, NB, FAST, kPitch39>(sp, theta_full, table, win, resid, model_out, nrows,
                                                        grid_rows, err, st);
    }
    return limber_launch<T, NB, FAST, 0>(sp, theta_full, table, win, resid, model_out, nrows, grid_rows, err, st);
}

template <typename T, bool FAST>
int launch_windows(const ShearParams& sp, const double* theta_full, T* win, const int* nrows, int grid_rows,
                   cudaStream_t st) {
    switch (sp.nb) {
        case 1: return windows_nb<T, 1, FAST>(sp, theta_full, win, nrows, grid_rows, st);
        case 2: return windows_nb<T, 2, FAST>(sp, theta_full, win, nrows, grid_rows, st);
        case 3: return windows_nb<T, 3, FAST>(sp, theta_full, win, nrows, grid_rows, st);
        case 4: return windows_nb<T, 4, FAST>(sp, theta_full, win, nrows, grid_rows, st);
        case 5: return windows_nb<T, 5, FAST>(sp, theta_full, win, nrows, grid_rows, st);
        default: return NS_ENOTSUP;
    }
}

template <typename T, bool FAST>
int launch_limber(const ShearParams& sp, const double* theta_full, const T* table, const T* win, T* resid,
                  double* model_out, const int* nrows, int grid_rows, int* err, cudaStream_t st) {
    switch (sp.nb) {
        case 1: return limber_nb<T, 1, FAST>(sp, theta_full, table, win, resid, model_out, nrows, grid_rows, err, st);
        case 2: return limber_nb<T, 2, FAST>(sp, theta_full, table, win, resid, model_out, nrows, grid_rows, err, st);
        case 3: return limber_nb<T, 3, FAST>(sp, theta_full, table, win, resid, model_out, nrows, grid_rows, err, st);
        case 4: return limber_nb<T, 4, FAST>(sp, theta_full, table, win, resid, model_out, nrows, grid_rows, err, st);
        case 5: return limber_nb<T, 5, FAST>(sp, theta_full, table, win, resid, model_out, nrows, grid_rows, err, st);
        default: return NS_ENOTSUP;
    }
}

template int launch_windows<double, false>(const ShearParams&, const double*, double*, const int*, int, cudaStream_t);
template int launch_windows<float, false>(const ShearParams&, const double*, float*, const int*, int, cudaStream_t);
template int launch_windows<float, true>(const ShearParams&, const double*, float*, const int*, int, cudaStream_t);
template int launch_limber<double, false>(const ShearParams&, const double*, const double*, const double*, double*,
                                          double*, const int*, int, int*, cudaStream_t);
template int launch_limber<float, false>(const ShearParams&, const double*, const float*, const float*, float*,
                                         double*, const int*, int, int*, cudaStream_t);
template int launch_limber<float, true>(const ShearParams&, const double*, const float*, const float*, float*,
                                        double*, const int*, int, int*, cudaStream_t);

}  // namespace gpuns
