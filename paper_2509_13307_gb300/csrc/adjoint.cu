// Hand-written adjoint of the shear likelihood (row A14): d log L / d theta.
//
// k_projection_adj (one CTA per evaluation) recomputes the forward projection
// into per-evaluation scratch (distances, growth, windows, padded P table,
// Limber sums, data vector, residual r, y = L^-1 r, log L) and then runs the
// reverse pass:
//   g_m = Sigma^-1 r = L^-T y                       (chi^2, Gaussian)
//   g_C[p][ell] = g_m (1+m_i)(1+m_j); g_b = T^T g_m; g_m_i from the bias products
//   Limber / lookup: per node, per multipole, g_P = sum_p g_C V_i V_j;
//     g_V_i += g_C V_j P; g_v = ln10 P g_P scattered onto the 16 table taps;
//     d v / d ln k (Catmull-Rom derivative) gives g_ln chi
//   windows (Eq. 5-6): the exclusive suffix sums transpose to exclusive prefix
//     sums of their adjoints; n(z) normalisation and the D_z shifts
//   growth: suffix sums of g_ln D through the trapezoid segments
//   distances: suffix sums of g_chi onto each Gauss-Legendre interval,
//     then d E^2 / d(Omega_m, w0, wa) at every quadrature point
//   scalars: Omega_m = (omega_b + omega_cdm)/h^2, c/H0 = c/(100 h), gamma(w0, wa)
// The table gradient (ghost rows/columns folded back) feeds the emulator
// backward pass (transposed GEMMs, tanh' from stored activations); the
// emulator-input gradient is added to the parameter gradient in
// k_finish_grad.
#include <cstring>
#include <mutex>
#include <vector>

#include "likelihood.cuh"

namespace gpuns {

namespace adj {

// 4-point Gauss-Legendre nodes and weights as compile-time constants of the
// kernel's type (no double -> float conversions at run time).
template <typename T> __device__ __forceinline__ T glx(int g) {
    return g == 0 ? T(-0.86113631159405257522) : g == 1 ? T(-0.33998104358485626480)
         : g == 2 ? T(0.33998104358485626480) : T(0.86113631159405257522);
}
template <typename T> __device__ __forceinline__ T glw(int g) {
    return (g == 0 || g == 3) ? T(0.34785484513745385737) : T(0.65214515486254614263);
}

template <typename T> __device__ __forceinline__ const T* pick(const double* d, const float* f);
template <> __device__ __forceinline__ const double* pick<double>(const double* d, const float*) { return d; }
template <> __device__ __forceinline__ const float* pick<float>(const double*, const float* f) { return f; }
template <typename T> __device__ __forceinline__ T pick_s(double d, float f);
template <> __device__ __forceinline__ double pick_s<double>(double d, float) { return d; }
template <> __device__ __forceinline__ float pick_s<float>(double, float f) { return f; }

template <typename T> __device__ __forceinline__ T ex(T x);
template <> __device__ __forceinline__ double ex<double>(double x) { return exp(x); }
template <> __device__ __forceinline__ float ex<float>(float x) { return expf(x); }
template <typename T> __device__ __forceinline__ T lg(T x);
template <> __device__ __forceinline__ double lg<double>(double x) { return log(x); }
template <> __device__ __forceinline__ float lg<float>(float x) { return logf(x); }

// Scalar adjoints accumulated in shared memory.
enum { S_OM = 0, S_CHIH, S_W0, S_WA, S_GAMMA, S_PREF, S_AIA, S_ETA, S_COUNT };

struct AdjArgs {
    ShearParams sp;
    const double* theta_full;
    const void* table;       // rows x (n_z n_k), T
    const void* LinvT;       // D x D, T: LinvT[b*D + a] = (L^-1)[a][b]
    double c0;
    void* scratch;           // rows x per_eval, T
    long long per_eval;
    void* gtab_out;          // rows x (n_z n_k), T: d log L / d table
    double* gfull;           // rows x n_params: d log L / d theta_full (emulator inputs excluded)
    double* logL;
    const int* nrows;
};

template <typename T>
__device__ __forceinline__ void cr_w(T t, T w[4]) {   // doubled Catmull-Rom weights
    const T t2 = t * t;
    w[0] = t * (t * (T(2) - t) - T(1));
    w[1] = T(2) + t2 * (T(3) * t - T(5));
    w[2] = t * (T(1) + t * (T(4) - T(3) * t));
    w[3] = t2 * (t - T(1));
}
template <typename T>
__device__ __forceinline__ void cr_dw(T t, T w[4]) {  // d/dt of the doubled weights
    w[0] = T(-1) + t * (T(4) - T(3) * t);
    w[1] = t * (T(9) * t - T(10));
    w[2] = T(1) + t * (T(8) - T(9) * t);
    w[3] = t * (T(3) * t - T(2));
}

template <typename T, int NB>
__global__ void __launch_bounds__(256)
k_projection_adj(const AdjArgs A) {
    constexpr int NP = NB * (NB + 1) / 2;
    const ShearParams& sp = A.sp;
    const int row = blockIdx.x;
    if (row >= *A.nrows) return;
    const int N = sp.N, n_k = sp.n_k, n_z = sp.n_z, PK = n_k + 2, PT = (n_z + 2) * PK, D = sp.D;
    const int tid = threadIdx.x, nt = blockDim.x;
    const int lane = tid & 31, wid = tid >> 5;
    T* S = reinterpret_cast<T*>(A.scratch) + (size_t)row * A.per_eval;
    T* chi = S;
    T* lnchi = S + N;
    T* Ez = S + 2 * N;
    T* Dg = S + 3 * N;
    T* omw = S + 4 * N;
    T* fg = S + 5 * N;
    T* gchi = S + 6 * N;
    T* gE = S + 7 * N;
    T* gomw = S + 8 * N;
    T* gD = S + 9 * N;
    T* t1 = S + 10 * N;
    T* t2 = S + 11 * N;
    T* raw = S + 12 * N;
    T* nchi = raw + NB * N;
    T* E0 = nchi + NB * N;
    T* E1 = E0 + NB * N;
    T* V = E1 + NB * N;
    T* gV = V + NB * N;
    T* tab = gV + NB * N;      // PT
    T* gtab = tab + PT;        // PT
    T* r = gtab + PT;          // D
    T* gm = r + D;             // D
    const T* nz_mu = pick<T>(sp.nz_mean, sp.nz_mean_f);
    const T* nz_sg = pick<T>(sp.nz_sigma, sp.nz_sigma_f);
    const T* lnell = pick<T>(sp.lnell, sp.lnell_f);
    const T* tmplT = pick<T>(sp.tmpl, sp.tmpl_f);
    const T* dataT = pick<T>(sp.data, sp.data_f);
    const T ia_piv = pick_s<T>(sp.ia_pivot, sp.ia_pivot_f), c1rho = pick_s<T>(sp.c1rho, sp.c1rho_f);
    const T* a_ = pick<T>(sp.a, sp.a_f);
    const T* lna_ = pick<T>(sp.lna, sp.lna_f);
    const T* z_ = pick<T>(sp.z, sp.z_f);
    const T* wa_ = pick<T>(sp.wa, sp.wa_f);
    const T* zwp = pick<T>(sp.zw4d, sp.zw4f);

    __shared__ T th[128];
    __shared__ T gth[128];
    __shared__ T gs[S_COUNT];
    __shared__ T red[64];
    __shared__ T red2[8 * NP];                 // per-warp pair sums of one multipole
    __shared__ T Cl[NP * 64];
    __shared__ T gC[NP * 64];
    __shared__ T norm[NB];
    for (int i = tid; i < sp.n_params; i += nt) {
        th[i] = (T)A.theta_full[(size_t)row * sp.n_params + i];
        gth[i] = T(0);
    }
    if (tid < S_COUNT) gs[tid] = T(0);
    __syncthreads();
    const T h = th[2];
    const T om = (th[0] + th[1]) / (h * h);
    const T w0 = th[5], wa = th[6];
    const T pde = T(3) * (T(1) + w0 + wa);
    const T chiH = T(kCover100) / h;
    const T gamma = T(0.55) + T(0.05) * (T(1) + w0 + T(0.5) * wa);
    const T pref = T(1.5) * om / (chiH * chiH);
    const T A_IA = th[9], eta = th[10];

    // ===================== forward (recorded) =====================
    for (int n = tid; n < N; n += nt) {
        const T a = a_[n], lna = lna_[n];
        const T de = ex<T>(-pde * lna - T(3) * wa * (T(1) - a));
        Ez[n] = sqrt(om * ex<T>(T(-3) * lna) + (T(1) - om) * de);
        T inc = T(0);
        if (n < N - 1) {
            const T a1 = a_[n + 1];
            const T mid = T(0.5) * (a + a1), half = T(0.5) * (a - a1);
            for (int g = 0; g < 4; ++g) {
                const T ag = mid + half * glx<T>(g);
                const T lgg = lg<T>(ag);
                const T e2 = om / (ag * ag * ag) + (T(1) - om) * ex<T>(-pde * lgg - T(3) * wa * (T(1) - ag));
                inc += glw<T>(g) / (ag * ag * sqrt(e2));
            }
            inc *= chiH * half;
        }
        t1[n] = inc;
    }
    __syncthreads();
    block_exclusive_scan(t1, N, red);
    for (int n = tid; n < N; n += nt) {
        const T c = t1[n];
        chi[n] = c;
        lnchi[n] = (n >= 1) ? lg<T>(c) : T(0);
        const T oma = om * ex<T>(T(-3) * lna_[n]) / (Ez[n] * Ez[n]);
        fg[n] = ex<T>(gamma * lg<T>(oma));
        omw[n] = wa_[n] * chiH / (a_[n] * a_[n] * Ez[n]);
        gchi[n] = T(0); gE[n] = T(0); gomw[n] = T(0); gD[n] = T(0);
    }
    __syncthreads();
    for (int n = tid; n < N; n += nt) t2[n] = (n < N - 1) ? T(0.5) * (fg[n] + fg[n + 1]) * (lna_[n] - lna_[n + 1]) : T(0);
    __syncthreads();
    block_exclusive_scan(t2, N, red);
    for (int n = tid; n < N; n += nt) Dg[n] = ex<T>(-t2[n]);
    __syncthreads();
    for (int i = 0; i < NB; ++i) {
        T part = T(0);
        for (int n = tid; n < N; n += nt) {
            const T u = (z_[n] - th[11 + i] - nz_mu[i]) / nz_sg[i];
            const T rw = ex<T>(T(-0.5) * u * u);
            raw[i * N + n] = rw;
            part += wa_[n] * rw / (a_[n] * a_[n]);
        }
        const T s = block_sum(part, red);
        if (tid == 0) norm[i] = s;
        __syncthreads();
        for (int n = tid; n < N; n += nt) {
            const T nc = raw[i * N + n] * Ez[n] / (chiH * s);
            nchi[i * N + n] = nc;
            E0[i * N + n] = (n >= 1) ? omw[n] * nc : T(0);
            E1[i * N + n] = (n >= 1) ? omw[n] * nc / chi[n] : T(0);
            gV[i * N + n] = T(0);
        }
        __syncthreads();
        block_exclusive_suffix_scan(E0 + i * N, N, red);
        block_exclusive_suffix_scan(E1 + i * N, N, red);
    }
    for (int n = tid; n < N; n += nt) {
        const T c = chi[n];
        const T amp = A_IA * ex<T>(eta * lg<T>((T(1) + z_[n]) / ia_piv)) * c1rho * om / Dg[n];
        for (int i = 0; i < NB; ++i) {
            T v = T(0);
            if (n >= 1) {
                const T W = pref * c / a_[n] * (E0[i * N + n] - c * E1[i * N + n]) - amp * nchi[i * N + n];
                v = sqrt(omw[n]) / c * W;
            }
            V[i * N + n] = v;
        }
    }
    // padded table (ghosts by linear extrapolation) and its zeroed gradient
    {
        const T* src = reinterpret_cast<const T*>(A.table) + (size_t)row * n_z * n_k;
        for (int i = tid; i < n_z * n_k; i += nt) tab[(i / n_k + 1) * PK + i % n_k + 1] = src[i];
        for (int i = tid; i < PT; i += nt) gtab[i] = T(0);
        __syncthreads();
        for (int k = 1 + tid; k <= n_k; k += nt) {
            tab[k] = T(2) * tab[PK + k] - tab[2 * PK + k];
            tab[(n_z + 1) * PK + k] = T(2) * tab[n_z * PK + k] - tab[(n_z - 1) * PK + k];
        }
        __syncthreads();
        for (int rr = tid; rr < n_z + 2; rr += nt) {
            tab[rr * PK] = T(2) * tab[rr * PK + 1] - tab[rr * PK + 2];
            tab[rr * PK + n_k + 1] = T(2) * tab[rr * PK + n_k] - tab[rr * PK + n_k - 1];
        }
    }
    __syncthreads();
    const T lkmin = pick_s<T>(sp.lnk_min, sp.lnk_min_f), lkmax = pick_s<T>(sp.lnk_max, sp.lnk_max_f);
    const T inv_dk = pick_s<T>(1.0 / sp.dlnk, sp.inv_dlnk_f);
    // Limber: C_p(ell) (block reductions, fixed order)
    for (int l = 0; l < sp.n_ell; ++l) {
        T acc[NP];
        for (int p = 0; p < NP; ++p) acc[p] = T(0);
        const T lne = lnell[l];
        for (int n = 1 + tid; n < N; n += nt) {
            T s = fmin(fmax(lne - lnchi[n], lkmin), lkmax);
            const T uk = (s - lkmin) * inv_dk;
            int ik = min(max((int)floor(uk), 0), n_k - 2);
            T wk[4];
            cr_w<T>(uk - (T)ik, wk);
            const T* c = tab + sp.zrp[n] * PK + ik;
            T v = T(0);
            for (int pz = 0; pz < 4; ++pz)
                v += zwp[4 * n + pz] * (wk[0] * c[pz * PK] + wk[1] * c[pz * PK + 1] + wk[2] * c[pz * PK + 2] + wk[3] * c[pz * PK + 3]);
            const T P = ex<T>(T(0.25) * v * (T)kLn10);
            int p = 0;
            for (int i = 0; i < NB; ++i)
                for (int j = i; j < NB; ++j) { acc[p] += V[i * N + n] * V[j * N + n] * P; ++p; }
        }
        // all NP pair sums at once: warp sums, then a fixed-order sum over warps
#pragma unroll
        for (int p = 0; p < NP; ++p) {
            const T s = warp_sum(acc[p]);
            if (lane == 0) red2[wid * NP + p] = s;
        }
        __syncthreads();
        if (tid < NP) {
            T s = T(0);
            for (int w = 0; w < (nt >> 5); ++w) s += red2[w * NP + tid];
            Cl[tid * sp.n_ell + l] = s;
        }
        __syncthreads();
    }
    __syncthreads();
    // data vector, residual, whitening, log L
    for (int a = tid; a < D; a += nt) {
        const int p = a / sp.n_ell, e = a % sp.n_ell;
        const int i = sp.pi[p], j = sp.pj[p];
        T m = (T(1) + th[11 + NB + i]) * (T(1) + th[11 + NB + j]) * Cl[p * sp.n_ell + e];
        for (int t = 0; t < sp.n_tmpl; ++t) m += tmplT[(size_t)a * sp.n_tmpl + t] * th[11 + 2 * NB + t];
        r[a] = dataT[a] - m;
    }
    __syncthreads();
    const T* LT = reinterpret_cast<const T*>(A.LinvT);
    T sq = T(0);
    for (int a = tid; a < D; a += nt) {
        T y = T(0);
        for (int b = 0; b <= a; ++b) y += LT[(size_t)b * D + a] * r[b];
        gm[a] = y;                      // y stored temporarily in gm
        sq += y * y;
    }
    sq = block_sum(sq, red);
    if (tid == 0) A.logL[row] = A.c0 - 0.5 * (double)sq;
    // ===================== reverse =====================
    // g_m = L^-T y: (g_m)_a = sum_{b >= a} (L^-1)[b][a] y_b = sum_{b >= a} LinvT[a*D + b] y_b
    for (int a = tid; a < D; a += nt) {
        T g = T(0);
        for (int b = a; b < D; ++b) g += LT[(size_t)a * D + b] * gm[b];
        r[a] = g;                       // r now holds g_m
    }
    __syncthreads();
    // bias, templates, g_C
    for (int a = tid; a < D; a += nt) {
        const int p = a / sp.n_ell, e = a % sp.n_ell;
        const int i = sp.pi[p], j = sp.pj[p];
        const T g = r[a];
        const T fi = T(1) + th[11 + NB + i], fj = T(1) + th[11 + NB + j];
        const T C = Cl[p * sp.n_ell + e];
        gC[p * sp.n_ell + e] = g * fi * fj;
        atomicAdd(&gth[11 + NB + i], g * C * fj);
        atomicAdd(&gth[11 + NB + j], g * C * fi);
        for (int t = 0; t < sp.n_tmpl; ++t) atomicAdd(&gth[11 + 2 * NB + t], g * tmplT[(size_t)a * sp.n_tmpl + t]);
    }
    __syncthreads();
    // Limber + lookup reverse: threads own nodes, loop over multipoles
    for (int n = 1 + tid; n < N; n += nt) {
        T vv[NB], gv_[NB];
        for (int i = 0; i < NB; ++i) { vv[i] = V[i * N + n]; gv_[i] = T(0); }
        T glnc = T(0);
        const int zr = sp.zrp[n];
        T wz[4];
        for (int pz = 0; pz < 4; ++pz) wz[pz] = zwp[4 * n + pz];
        for (int l = 0; l < sp.n_ell; ++l) {
            const T s_raw = lnell[l] - lnchi[n];
            const bool clamped = (s_raw < lkmin) || (s_raw > lkmax);
            const T s = fmin(fmax(s_raw, lkmin), lkmax);
            const T uk = (s - lkmin) * inv_dk;
            int ik = min(max((int)floor(uk), 0), n_k - 2);
            const T t = uk - (T)ik;
            T wk[4], dwk[4];
            cr_w<T>(t, wk);
            cr_dw<T>(t, dwk);
            const T* c = tab + zr * PK + ik;
            T v = T(0), dv = T(0);
            for (int pz = 0; pz < 4; ++pz) {
                const T* cr = c + pz * PK;
                v += wz[pz] * (wk[0] * cr[0] + wk[1] * cr[1] + wk[2] * cr[2] + wk[3] * cr[3]);
                dv += wz[pz] * (dwk[0] * cr[0] + dwk[1] * cr[1] + dwk[2] * cr[2] + dwk[3] * cr[3]);
            }
            const T P = ex<T>(T(0.25) * v * (T)kLn10);
            T gP = T(0);
            int p = 0;
            for (int i = 0; i < NB; ++i)
                for (int j = i; j < NB; ++j) {
                    const T g = gC[p * sp.n_ell + l];
                    gP += g * vv[i] * vv[j];
                    gv_[i] += g * vv[j] * P;
                    gv_[j] += g * vv[i] * P;
                    ++p;
                }
            const T gvv = gP * P * (T)kLn10 * T(0.25);   // d log L / d (doubled-weight sum)
            T* gc = gtab + zr * PK + ik;
            for (int pz = 0; pz < 4; ++pz)
                for (int q = 0; q < 4; ++q) atomicAdd(gc + pz * PK + q, gvv * wz[pz] * wk[q]);
            if (!clamped) glnc -= gvv * dv * inv_dk;     // s = ln(ell+1/2) - ln chi
        }
        for (int i = 0; i < NB; ++i) gV[i * N + n] = gv_[i];
        gchi[n] += glnc / chi[n];
    }
    __syncthreads();
    // fold the ghost-cell gradients back onto the table (reverse of the padding)
    for (int rr = tid; rr < n_z + 2; rr += nt) {
        const T g0 = gtab[rr * PK], g1 = gtab[rr * PK + n_k + 1];
        gtab[rr * PK + 1] += T(2) * g0; gtab[rr * PK + 2] -= g0;
        gtab[rr * PK + n_k] += T(2) * g1; gtab[rr * PK + n_k - 1] -= g1;
    }
    __syncthreads();
    for (int k = 1 + tid; k <= n_k; k += nt) {
        const T g0 = gtab[k], g1 = gtab[(n_z + 1) * PK + k];
        gtab[PK + k] += T(2) * g0; gtab[2 * PK + k] -= g0;
        gtab[n_z * PK + k] += T(2) * g1; gtab[(n_z - 1) * PK + k] -= g1;
    }
    __syncthreads();
    {
        T* dst = reinterpret_cast<T*>(A.gtab_out) + (size_t)row * n_z * n_k;
        for (int i = tid; i < n_z * n_k; i += nt) dst[i] = gtab[(i / n_k + 1) * PK + i % n_k + 1];
    }
    // windows reverse: V = sqrt(omw)/chi * W, W = pc (E0 - chi E1) - amp nchi
    T l_pref = T(0), l_aia = T(0), l_eta = T(0), l_om = T(0);
    for (int n = 1 + tid; n < N; n += nt) {
        const T c = chi[n], an = a_[n];
        const T so = sqrt(omw[n]);
        const T q = ex<T>(eta * lg<T>((T(1) + z_[n]) / ia_piv));
        const T ampc = q * c1rho * om / Dg[n];       // amp = A_IA * ampc
        const T pc = pref * c / an;
        T g_so = T(0), g_c = T(0), g_amp = T(0);
        for (int i = 0; i < NB; ++i) {
            const T e0 = E0[i * N + n], e1 = E1[i * N + n], nc = nchi[i * N + n];
            const T W = pc * (e0 - c * e1) - A_IA * ampc * nc;
            const T gVv = gV[i * N + n];
            const T gW = gVv * so / c;
            g_so += gVv * W / c;
            g_c += -gVv * so * W / (c * c);
            // W partials
            const T gpc = gW * (e0 - c * e1);
            l_pref += gpc * c / an;
            g_c += gpc * pref / an - gW * pc * e1;
            E0[i * N + n] = gW * pc;            // reuse E0/E1 storage as their adjoints
            E1[i * N + n] = -gW * pc * c;
            g_amp += -gW * nc;
            raw[i * N + n] = -gW * A_IA * ampc; // reuse raw as g_nchi (direct term)
        }
        gomw[n] += g_so * T(0.5) / so;
        gchi[n] += g_c;
        // amp = A_IA q c1rho Om / D
        l_aia += g_amp * ampc;
        l_eta += g_amp * A_IA * ampc * lg<T>((T(1) + z_[n]) / ia_piv);
        l_om += g_amp * A_IA * ampc / om;
        gD[n] += -g_amp * A_IA * ampc / Dg[n];
    }
    if (true) {   // node 0 carries no window value; its direct g_nchi is zero
        for (int i = 0; i < NB; ++i) if (tid == 0) { raw[i * N] = T(0); E0[i * N] = T(0); E1[i * N] = T(0); }
    }
    l_pref = block_sum(l_pref, red);
    l_aia = block_sum(l_aia, red);
    l_eta = block_sum(l_eta, red);
    l_om = block_sum(l_om, red);
    if (tid == 0) {
        gs[S_PREF] += l_pref; gs[S_AIA] += l_aia; gs[S_ETA] += l_eta; gs[S_OM] += l_om;
    }
    __syncthreads();
    // E0_i(n) = sum_{m>n} omw_m nchi_m  ->  G0(m) = sum_{n<m} gE0(n) (exclusive prefix)
    for (int i = 0; i < NB; ++i) {
        block_exclusive_scan(E0 + i * N, N, red);
        block_exclusive_scan(E1 + i * N, N, red);
        T gdz = T(0), gnorm = T(0);
        for (int m = tid; m < N; m += nt) {
            T gnc = raw[i * N + m];
            if (m >= 1) {
                const T G0 = E0[i * N + m], G1 = E1[i * N + m];
                const T nc = nchi[i * N + m], c = chi[m];
                gomw[m] += nc * (G0 + G1 / c);
                gnc += omw[m] * (G0 + G1 / c);
                gchi[m] += -omw[m] * nc * G1 / (c * c);
            }
            raw[i * N + m] = gnc;   // total g_nchi
        }
        __syncthreads();
        // nchi = raw E / (chiH norm)
        const T nrm = norm[i];
        T l_chih = T(0);
        for (int m = tid; m < N; m += nt) {
            const T gnc = raw[i * N + m];
            const T nc = nchi[i * N + m];
            const T u = (z_[m] - th[11 + i] - nz_mu[i]) / nz_sg[i];
            gE[m] += gnc * nc / Ez[m];
            l_chih += -gnc * nc / chiH;
            gnorm += -gnc * nc / nrm;
            // d raw / d Dz = raw u / sigma and nchi is proportional to raw
            gdz += gnc * nc * u / nz_sg[i];
        }
        gnorm = block_sum(gnorm, red);
        // norm = sum wa raw / a^2  ->  d norm / d Dz = sum wa raw u / sigma / a^2
        for (int m = tid; m < N; m += nt) {
            const T u = (z_[m] - th[11 + i] - nz_mu[i]) / nz_sg[i];
            const T rw = ex<T>(T(-0.5) * u * u);
            gdz += gnorm * wa_[m] * rw * u / nz_sg[i] / (a_[m] * a_[m]);
        }
        gdz = block_sum(gdz, red);
        l_chih = block_sum(l_chih, red);
        if (tid == 0) { gth[11 + i] += gdz; gs[S_CHIH] += l_chih; }
        __syncthreads();
    }
    // omw = wa chiH / (a^2 E)
    {
        T l_chih = T(0);
        for (int n = tid; n < N; n += nt) {
            l_chih += gomw[n] * omw[n] / chiH;
            gE[n] += -gomw[n] * omw[n] / Ez[n];
        }
        l_chih = block_sum(l_chih, red);
        if (tid == 0) gs[S_CHIH] += l_chih;
    }
    // growth: D_n = exp(-S_n), S_n = sum_{m<n} seg_m, seg_m = (f_m + f_{m+1}) / 2 * dlna_m
    for (int n = tid; n < N; n += nt) t1[n] = -gD[n] * Dg[n];   // g_S
    __syncthreads();
    block_exclusive_suffix_scan(t1, N, red);                     // g_seg_m = sum_{n>m} g_S_n
    {
        T l_om = T(0), l_gam = T(0);
        for (int m = tid; m < N; m += nt) {
            T gf = T(0);
            if (m < N - 1) gf += T(0.5) * t1[m] * (lna_[m] - lna_[m + 1]);
            if (m >= 1) gf += T(0.5) * t1[m - 1] * (lna_[m - 1] - lna_[m]);
            const T oma = om * ex<T>(T(-3) * lna_[m]) / (Ez[m] * Ez[m]);
            l_gam += gf * fg[m] * lg<T>(oma);
            const T goma = gf * fg[m] * gamma / oma;
            l_om += goma * oma / om;
            gE[m] += goma * T(-2) * oma / Ez[m];
        }
        l_om = block_sum(l_om, red);
        l_gam = block_sum(l_gam, red);
        if (tid == 0) { gs[S_OM] += l_om; gs[S_GAMMA] += l_gam; }
    }
    __syncthreads();
    // distances: chi_n = sum_{m<n} dchi_m  ->  g_dchi_m = sum_{n>m} g_chi_n
    for (int n = tid; n < N; n += nt) t2[n] = gchi[n];
    __syncthreads();
    block_exclusive_suffix_scan(t2, N, red);
    {
        T l_om = T(0), l_w0 = T(0), l_wa = T(0), l_chih = T(0);
        for (int n = tid; n < N; n += nt) {
            const T a = a_[n], lna = lna_[n];
            const T de = ex<T>(-pde * lna - T(3) * wa * (T(1) - a));
            // node E: E^2 = om a^-3 + (1 - om) de
            const T ge2 = gE[n] / (T(2) * Ez[n]);
            l_om += ge2 * (ex<T>(T(-3) * lna) - de);
            l_w0 += ge2 * (T(1) - om) * de * (T(-3) * lna);
            l_wa += ge2 * (T(1) - om) * de * (T(-3) * lna - T(3) * (T(1) - a));
            if (n < N - 1) {
                const T g = t2[n];
                const T a1 = a_[n + 1];
                const T mid = T(0.5) * (a + a1), half = T(0.5) * (a - a1);
                T inc = T(0);
                for (int q = 0; q < 4; ++q) {
                    const T ag = mid + half * glx<T>(q);
                    const T lgg = lg<T>(ag);
                    const T deg = ex<T>(-pde * lgg - T(3) * wa * (T(1) - ag));
                    const T e2 = om / (ag * ag * ag) + (T(1) - om) * deg;
                    const T F = T(1) / (ag * ag * sqrt(e2));
                    inc += glw<T>(q) * F;
                    const T gF = g * chiH * half * glw<T>(q);
                    const T gE2 = gF * T(-0.5) * F / e2;
                    l_om += gE2 * (T(1) / (ag * ag * ag) - deg);
                    l_w0 += gE2 * (T(1) - om) * deg * (T(-3) * lgg);
                    l_wa += gE2 * (T(1) - om) * deg * (T(-3) * lgg - T(3) * (T(1) - ag));
                }
                l_chih += g * half * inc;
            }
        }
        l_om = block_sum(l_om, red);
        l_w0 = block_sum(l_w0, red);
        l_wa = block_sum(l_wa, red);
        l_chih = block_sum(l_chih, red);
        if (tid == 0) { gs[S_OM] += l_om; gs[S_W0] += l_w0; gs[S_WA] += l_wa; gs[S_CHIH] += l_chih; }
    }
    __syncthreads();
    if (tid == 0) {
        // pref = 1.5 om / chiH^2; gamma = 0.55 + 0.05 (1 + w0 + wa/2)
        const T g_om = gs[S_OM] + gs[S_PREF] * pref / om;
        const T g_chih = gs[S_CHIH] - T(2) * gs[S_PREF] * pref / chiH;
        const T g_w0 = gs[S_W0] + T(0.05) * gs[S_GAMMA];
        const T g_wa = gs[S_WA] + T(0.025) * gs[S_GAMMA];
        // om = (wb + wc) / h^2; chiH = c / (100 h)
        gth[0] += g_om / (h * h);
        gth[1] += g_om / (h * h);
        gth[2] += -T(2) * g_om * om / h - g_chih * chiH / h;
        gth[5] += g_w0;
        gth[6] += g_wa;
        gth[9] += gs[S_AIA];
        gth[10] += gs[S_ETA];
    }
    __syncthreads();
    for (int i = tid; i < sp.n_params; i += nt) A.gfull[(size_t)row * sp.n_params + i] = (double)gth[i];
}

template <typename T, int NB>
size_t per_eval_elems(const ShearParams& sp) {
    return (size_t)(12 + 6 * NB) * sp.N + 2 * (size_t)(sp.n_z + 2) * (sp.n_k + 2) + 2 * (size_t)sp.D;
}

}  // namespace adj

int adjoint_scratch_elems(const ShearParams& sp) {
    return (12 + 6 * sp.nb) * sp.N + 2 * (sp.n_z + 2) * (sp.n_k + 2) + 2 * sp.D;
}

template <typename T>
int launch_projection_adj(const ShearParams& sp, const double* theta_full, const T* table, const T* LinvT, double c0,
                          T* scratch, T* gtab, double* gfull, double* logL, const int* nrows, int grid_rows,
                          cudaStream_t st) {
    if (sp.n_ell > 64 || sp.n_params > 128) return NS_ENOTSUP;
    adj::AdjArgs A{sp, theta_full, table, LinvT, c0, scratch, (long long)adjoint_scratch_elems(sp), gtab, gfull,
                   logL, nrows};
    auto go = [&](auto kern) -> int {
        kern<<<grid_rows, 256, 0, st>>>(A);
        return NS_OK;
    };
    switch (sp.nb) {
        case 1: NS_TRY(go(adj::k_projection_adj<T, 1>)); break;
        case 2: NS_TRY(go(adj::k_projection_adj<T, 2>)); break;
        case 3: NS_TRY(go(adj::k_projection_adj<T, 3>)); break;
        case 4: NS_TRY(go(adj::k_projection_adj<T, 4>)); break;
        case 5: NS_TRY(go(adj::k_projection_adj<T, 5>)); break;
        default: return NS_ENOTSUP;
    }
    NS_CUDA_TRY(cudaGetLastError());
    return NS_OK;
}
template int launch_projection_adj<double>(const ShearParams&, const double*, const double*, const double*, double,
                                           double*, double*, double*, double*, const int*, int, cudaStream_t);
template int launch_projection_adj<float>(const ShearParams&, const double*, const float*, const float*, double,
                                          float*, float*, double*, double*, const int*, int, cudaStream_t);

// ------------------------------------------------------------------ emulator backward
namespace adj {

// Forward layer with stored activation: out = tanh(A W^T + b) (hidden) or
// mu + sigma (A W^T + b) (output); A: rows x K, W: N x K.
template <typename T, int BM, int BN, int BK, int TM, int TN>
__global__ void __launch_bounds__((BM / TM) * (BN / TN))
k_dense(const T* __restrict__ A, const T* __restrict__ W, const T* __restrict__ bias, const T* __restrict__ mu,
        T sigma, T* __restrict__ C, const int* __restrict__ nrows, int N, int K, int mode,
        const T* __restrict__ aux) {
    // mode 0: tanh(acc + b); 1: mu + sigma (acc + b); 2: acc * (1 - aux^2)  [W read transposed: W is K_out x N]
    constexpr int TX = BN / TN, TY = BM / TM, NT = TX * TY;
    const int M = *nrows;
    const int m0 = blockIdx.y * BM, n0 = blockIdx.x * BN;
    if (m0 >= M) return;
    __shared__ T As[BK][BM + 1];
    __shared__ T Bs[BK][BN + 1];
    const int tid = threadIdx.x, tx = tid % TX, ty = tid / TX;
    T acc[TM][TN];
    for (int i = 0; i < TM; ++i)
        for (int j = 0; j < TN; ++j) acc[i][j] = T(0);
    for (int k0 = 0; k0 < K; k0 += BK) {
        for (int i = tid; i < BM * BK; i += NT) {
            const int rr = i / BK, c = i % BK;
            As[c][rr] = (m0 + rr < M && k0 + c < K) ? A[(size_t)(m0 + rr) * K + k0 + c] : T(0);
        }
        if (mode == 2) {
            // contraction index k over rows of W (K x N row-major): element (n, k) = W[k * N + n]
            for (int i = tid; i < BN * BK; i += NT) {
                const int c = i / BN, nn = i % BN;
                Bs[c][nn] = (n0 + nn < N && k0 + c < K) ? W[(size_t)(k0 + c) * N + n0 + nn] : T(0);
            }
        } else {
            for (int i = tid; i < BN * BK; i += NT) {
                const int rr = i / BK, c = i % BK;
                Bs[c][rr] = (n0 + rr < N && k0 + c < K) ? W[(size_t)(n0 + rr) * K + k0 + c] : T(0);
            }
        }
        __syncthreads();
        for (int kk = 0; kk < BK; ++kk) {
            T a[TM], b[TN];
            for (int i = 0; i < TM; ++i) a[i] = As[kk][ty + i * TY];
            for (int j = 0; j < TN; ++j) b[j] = Bs[kk][tx + j * TX];
            for (int i = 0; i < TM; ++i)
                for (int j = 0; j < TN; ++j) acc[i][j] = fma(a[i], b[j], acc[i][j]);
        }
        __syncthreads();
    }
    for (int i = 0; i < TM; ++i) {
        const int gm = m0 + ty + i * TY;
        if (gm >= M) continue;
        for (int j = 0; j < TN; ++j) {
            const int gn = n0 + tx + j * TX;
            if (gn >= N) continue;
            T v = acc[i][j];
            if (mode == 0) v = tanh(v + bias[gn]);
            else if (mode == 1) v = mu[gn] + sigma * (v + bias[gn]);
            else { const T hh = aux[(size_t)gm * N + gn]; v = v * (T(1) - hh * hh); }
            C[(size_t)gm * N + gn] = v;
        }
    }
}

template <typename T>
__global__ void k_emu_in_store(const double* __restrict__ theta_full, int P, const int* __restrict__ inputs,
                               const double* __restrict__ center, const double* __restrict__ scale, int K0,
                               const T* __restrict__ W0, const T* __restrict__ b0, int N, T* __restrict__ out,
                               const int* __restrict__ nrows) {
    const int row = blockIdx.y;
    if (row >= *nrows) return;
    const int n = blockIdx.x * blockDim.x + threadIdx.x;
    if (n >= N) return;
    T acc = b0[n];
    for (int j = 0; j < K0; ++j)
        acc += W0[(size_t)n * K0 + j] * (T)((theta_full[(size_t)row * P + inputs[j]] - center[j]) / scale[j]);
    out[(size_t)row * N + n] = tanh(acc);
}

// g_pre_1 (rows x N1) -> g_x (rows x K0) = g_pre_1 W0; then add to the full gradient.
template <typename T>
__global__ void k_emu_in_back(const T* __restrict__ gpre, const T* __restrict__ W0, int N1, int K0,
                              const int* __restrict__ inputs, const double* __restrict__ scale, double* __restrict__ gfull,
                              int P, const int* __restrict__ nrows) {
    const int row = blockIdx.x;
    if (row >= *nrows) return;
    __shared__ T red[32];
    for (int j = 0; j < K0; ++j) {
        T s = T(0);
        for (int n = threadIdx.x; n < N1; n += blockDim.x) s += gpre[(size_t)row * N1 + n] * W0[(size_t)n * K0 + j];
        s = block_sum(s, red);
        if (threadIdx.x == 0) gfull[(size_t)row * P + inputs[j]] += (double)s / scale[j];
    }
}

template <typename T>
__global__ void k_scale(const T* __restrict__ in, T* __restrict__ out, T s, int n_per_row, const int* __restrict__ nrows) {
    const int row = blockIdx.y;
    if (row >= *nrows) return;
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < n_per_row; i += gridDim.x * blockDim.x)
        out[(size_t)row * n_per_row + i] = s * in[(size_t)row * n_per_row + i];
}

// Transpose of the coarse -> fine Catmull-Rom z interpolation:
// g_coarse[j][k] = sum_{jz, q: zr[jz][q] = j} w[jz][q] g_fine[jz][k].
template <typename T>
__global__ void k_zinterp_adj(const T* __restrict__ gfine, int nz, const int* __restrict__ zr,
                              const double* __restrict__ zw, T* __restrict__ gcoarse, int nzc, int nk,
                              const int* __restrict__ nrows) {
    const int row = blockIdx.y;
    if (row >= *nrows) return;
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < nzc * nk; i += gridDim.x * blockDim.x) {
        const int j = i / nk, k = i % nk;
        T s = T(0);
        for (int jz = 0; jz < nz; ++jz)
            for (int q = 0; q < 4; ++q)
                if (zr[jz * 4 + q] == j) s += (T)zw[jz * 4 + q] * gfine[(size_t)row * nz * nk + jz * nk + k];
        gcoarse[(size_t)row * nzc * nk + i] = s;
    }
}

__global__ void k_gather_grad(const double* __restrict__ gfull, int P, const int* __restrict__ free_of_full,
                              double* __restrict__ grad, int d, int B) {
    const int row = blockIdx.x;
    if (row >= B) return;
    for (int i = threadIdx.x; i < P; i += blockDim.x) {
        const int f = free_of_full[i];
        if (f >= 0) grad[(size_t)row * d + f] = gfull[(size_t)row * P + i];
    }
}

// BF16 problems, split path.  Input layer: h = tanh(W0 x + b0) in FP32 with
// x standardised once per row (reciprocal scale), written as a bf16 (hi, lo)
// pair: layer 1's A operand and the stored activation for the backward pass.
__global__ void k_emu_in_split(const double* __restrict__ theta_full, int P, const int* __restrict__ inputs,
                               const double* __restrict__ center, const double* __restrict__ inv_scale, int K0,
                               const float* __restrict__ W0, const float* __restrict__ b0, int N,
                               __nv_bfloat16* __restrict__ hi, __nv_bfloat16* __restrict__ lo,
                               const int* __restrict__ nrows) {
    const int row = blockIdx.y;
    if (row >= *nrows) return;
    __shared__ float x[32];
    if (threadIdx.x < K0) {
        const int j = threadIdx.x;
        x[j] = (float)((theta_full[(size_t)row * P + inputs[j]] - center[j]) * inv_scale[j]);
    }
    __syncthreads();
    const int n = blockIdx.x * blockDim.x + threadIdx.x;
    if (n >= N) return;
    float acc = b0[n];
    for (int j = 0; j < K0; ++j) acc = fmaf(W0[(size_t)n * K0 + j], x[j], acc);
    const float h = tanhf(acc);
    const __nv_bfloat16 hh = __float2bfloat16_rn(h);
    hi[(size_t)row * N + n] = hh;
    lo[(size_t)row * N + n] = __float2bfloat16_rn(h - __bfloat162float(hh));
}

// g = s * in (rows x n) written as a bf16 (hi, lo) pair.
__global__ void k_scale_split(const float* __restrict__ in, float s, int n, __nv_bfloat16* __restrict__ hi,
                              __nv_bfloat16* __restrict__ lo, const int* __restrict__ nrows) {
    const int row = blockIdx.y;
    if (row >= *nrows) return;
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x) {
        const float g = s * in[(size_t)row * n + i];
        const __nv_bfloat16 gh = __float2bfloat16_rn(g);
        hi[(size_t)row * n + i] = gh;
        lo[(size_t)row * n + i] = __float2bfloat16_rn(g - __bfloat162float(gh));
    }
}

template <typename T>
static int dense(const T* A, const T* W, const T* bias, const T* mu, T sigma, T* C, const int* nrows, int grid_rows,
                 int N, int K, int mode, const T* aux, cudaStream_t st) {
    constexpr int BM = 64, BN = 64, BK = 8, TM = 4, TN = 4;
    dim3 g((N + BN - 1) / BN, (grid_rows + BM - 1) / BM);
    k_dense<T, BM, BN, BK, TM, TN><<<g, 256, 0, st>>>(A, W, bias, mu, sigma, C, nrows, N, K, mode, aux);
    NS_CUDA_TRY(cudaGetLastError());
    return NS_OK;
}

}  // namespace adj

struct GradWorkspace {
    int cap = 0;
    std::vector<void*> H;      // stored activations per hidden layer (index 1..L-1)
    void* gA = nullptr;        // ping-pong adjoint buffers (cap x max(hidden, n_out))
    void* gB = nullptr;
    void* gtab = nullptr;      // cap x n_z n_k
    void* table = nullptr;     // cap x n_out (emulator output)
    void* table_fine = nullptr;
    void* scratch = nullptr;   // cap x adjoint_scratch_elems
    double* gfull = nullptr;   // cap x P
    std::vector<void*> owned;
};

static std::mutex g_grad_mu;

template <typename T>
static int grad_ws_create(const ns_problem* p, int cap, GradWorkspace* g) {
    g->cap = cap;
    auto alloc = [&](size_t bytes, void** out) -> int {
        if (cudaMalloc(out, bytes) != cudaSuccess) return NS_ENOMEM;
        g->owned.push_back(*out);
        return NS_OK;
    };
    const int L = p->n_layers;
    const int n_out = p->dims.back();
    const int nzk = p->sp.n_z * p->sp.n_k;
    g->H.assign(L, nullptr);
    for (int l = 1; l < L; ++l) NS_TRY(alloc(sizeof(T) * (size_t)cap * p->dims[l], &g->H[l]));
    const size_t wmax = std::max(p->hidden_max, std::max(n_out, nzk));
    NS_TRY(alloc(sizeof(T) * (size_t)cap * wmax, &g->gA));
    NS_TRY(alloc(sizeof(T) * (size_t)cap * wmax, &g->gB));
    NS_TRY(alloc(sizeof(T) * (size_t)cap * nzk, &g->gtab));
    NS_TRY(alloc(sizeof(T) * (size_t)cap * n_out, &g->table));
    if (p->n_z_emu != p->sp.n_z) NS_TRY(alloc(sizeof(T) * (size_t)cap * nzk, &g->table_fine));
    NS_TRY(alloc(sizeof(T) * (size_t)cap * adjoint_scratch_elems(p->sp), &g->scratch));
    void* gf;
    NS_TRY(alloc(sizeof(double) * (size_t)cap * p->P, &gf));
    g->gfull = (double*)gf;
    return NS_OK;
}

// Weights of the gradient path in its arithmetic type (FP64 problems: as
// stored; FP32 / BF16 problems: FP32 copies made here from the FP64 master).
struct GradWeights {
    std::vector<void*> W, b;
    void* mu = nullptr;
    std::vector<void*> owned;
};

template <typename T>
static int run_grad(const ns_problem* p, GradWorkspace* g, const GradWeights* gw, const double* theta_full,
                    const int* d_nrows, int B, double* logL, double* grad, cudaStream_t st) {
    const int L = p->n_layers;
    const ShearParams& sp = p->sp;
    const int n_out = p->dims.back();
    const int nzk = sp.n_z * sp.n_k;
    // forward emulator with stored activations
    {
        dim3 g0((p->dims[1] + 255) / 256, B);
        adj::k_emu_in_store<T><<<g0, 256, 0, st>>>(theta_full, p->P, p->d_inputs, p->d_in_center, p->d_in_scale,
                                                   p->dims[0], (const T*)gw->W[0], (const T*)gw->b[0], p->dims[1],
                                                   (T*)g->H[1], d_nrows);
        NS_CUDA_TRY(cudaGetLastError());
        for (int l = 1; l < L; ++l) {
            const bool last = (l == L - 1);
            T* out = last ? (T*)g->table : (T*)g->H[l + 1];
            NS_TRY(adj::dense<T>((const T*)g->H[l], (const T*)gw->W[l], (const T*)gw->b[l], (const T*)gw->mu,
                                 (T)p->out_sigma, out, d_nrows, B, p->dims[l + 1], p->dims[l], last ? 1 : 0, nullptr,
                                 st));
        }
    }
    const T* tab = (const T*)g->table;
    if (p->n_z_emu != sp.n_z) {
        // forward coarse -> fine interpolation
        NS_TRY(launch_zinterp_generic(p, g->table, g->table_fine, d_nrows, B, (int)sizeof(T), st));
        tab = (const T*)g->table_fine;
    }
    const T* LT = (sizeof(T) == 8) ? (const T*)(const void*)p->d_LinvT64 : (const T*)(const void*)p->d_LinvT32;
    NS_TRY(launch_projection_adj<T>(sp, theta_full, tab, LT, p->c0, (T*)g->scratch, (T*)g->gtab, g->gfull, logL,
                                    d_nrows, B, st));
    // table adjoint -> emulator output adjoint (transpose of the z interpolation) -> g_pre_L
    T* gcur = (T*)g->gA;
    T* gnext = (T*)g->gB;
    if (p->n_z_emu != sp.n_z) {
        dim3 gz((p->n_z_emu * sp.n_k + 255) / 256, B);
        adj::k_zinterp_adj<T><<<gz, 256, 0, st>>>((const T*)g->gtab, sp.n_z, p->d_zi_row, p->d_zi_w, gnext,
                                                  p->n_z_emu, sp.n_k, d_nrows);
        dim3 gs((n_out + 255) / 256, B);
        adj::k_scale<T><<<gs, 256, 0, st>>>(gnext, gcur, (T)p->out_sigma, n_out, d_nrows);
    } else {
        dim3 gs((n_out + 255) / 256, B);
        adj::k_scale<T><<<gs, 256, 0, st>>>((const T*)g->gtab, gcur, (T)p->out_sigma, n_out, d_nrows);
    }
    NS_CUDA_TRY(cudaGetLastError());
    // g_pre_{l} = (g_pre_{l+1} W_l) * (1 - h_l^2), l = L-1 .. 1
    for (int l = L - 1; l >= 1; --l) {
        NS_TRY(adj::dense<T>(gcur, (const T*)gw->W[l], nullptr, nullptr, T(0), gnext, d_nrows, B, p->dims[l],
                             p->dims[l + 1], 2, (const T*)g->H[l], st));
        std::swap(gcur, gnext);
    }
    adj::k_emu_in_back<T><<<B, 256, 0, st>>>(gcur, (const T*)gw->W[0], p->dims[1], p->dims[0], p->d_inputs,
                                             p->d_in_scale, g->gfull, p->P, d_nrows);
    adj::k_gather_grad<<<B, 64, 0, st>>>(g->gfull, p->P, p->d_free_of_full, grad, p->d, B);
    NS_CUDA_TRY(cudaGetLastError());
    return NS_OK;
}

// BF16 problems: the emulator forward and backward on the tensor cores
// (split-BF16 activations and gradients, exact bf16 weights, FP32 accumulate),
// the projection adjoint in FP32.  Layer l (1 .. L-1) maps dims[l] -> dims[l+1].
struct SplitGrad {
    int rows_pad = 0;
    std::vector<__nv_bfloat16*> Hhi, Hlo;   // input activations of layer l (rows_pad x dims[l])
    __nv_bfloat16* Ghi[2] = {nullptr, nullptr};
    __nv_bfloat16* Glo[2] = {nullptr, nullptr};  // backward ping-pong (rows_pad x wmax)
    float* G1 = nullptr;                     // gradient of layer 1's pre-activations (rows_pad x dims[1])
    std::vector<__nv_bfloat16*> WT;          // W_l^T (dims[l] x dims[l+1])
    std::vector<CUtensorMap> tmHhi, tmHlo, tmW, tmGhi, tmGlo, tmWT;
    std::vector<void*> owned;
};

constexpr int kSplitHiddenTile = 128;        // forward hidden layers and every backward layer
constexpr int kSplitOutTile = 256;           // forward output layer

static bool split_supported(const ns_problem* p) {
    if (p->kind != NS_KIND_SHEAR || (p->precision != NS_PREC_BF16 && p->precision != NS_PREC_BF16_F64CHI2)) return false;
    if (p->act != NS_ACT_TANH || p->d_out_sig || p->n_layers < 2 || p->dims[0] > 32) return false;
    for (int l = 1; l <= p->n_layers; ++l)
        if (p->dims[l] % 8) return false;
    return true;
}

static int split_grad_create(const ns_problem* p, int cap, SplitGrad* g) {
    const int L = p->n_layers;
    const int rows_pad = ((cap + 127) / 128) * 128;
    g->rows_pad = rows_pad;
    auto alloc = [&](size_t bytes, void** out) -> int {
        if (cudaMalloc(out, bytes) != cudaSuccess) return NS_ENOMEM;
        g->owned.push_back(*out);
        return cudaMemset(*out, 0, bytes) == cudaSuccess ? NS_OK : NS_ECUDA;
    };
    void* v;
    g->Hhi.assign(L, nullptr);
    g->Hlo.assign(L, nullptr);
    for (int l = 1; l < L; ++l) {
        NS_TRY(alloc(sizeof(__nv_bfloat16) * (size_t)rows_pad * p->dims[l], &v)); g->Hhi[l] = (__nv_bfloat16*)v;
        NS_TRY(alloc(sizeof(__nv_bfloat16) * (size_t)rows_pad * p->dims[l], &v)); g->Hlo[l] = (__nv_bfloat16*)v;
    }
    int wmax = 0;
    for (int l = 1; l <= L; ++l) wmax = std::max(wmax, p->dims[l]);
    for (int i = 0; i < 2; ++i) {
        NS_TRY(alloc(sizeof(__nv_bfloat16) * (size_t)rows_pad * wmax, &v)); g->Ghi[i] = (__nv_bfloat16*)v;
        NS_TRY(alloc(sizeof(__nv_bfloat16) * (size_t)rows_pad * wmax, &v)); g->Glo[i] = (__nv_bfloat16*)v;
    }
    NS_TRY(alloc(sizeof(float) * (size_t)rows_pad * p->dims[1], &v)); g->G1 = (float*)v;
    // W_l^T in bf16 (the problem's tensor-core weights are bf16 already)
    g->WT.assign(L, nullptr);
    for (int l = 1; l < L; ++l) {
        const int No = p->dims[l + 1], Ki = p->dims[l];
        std::vector<uint16_t> w((size_t)No * Ki), wt((size_t)No * Ki);
        NS_CUDA_TRY(cudaMemcpy(w.data(), p->d_W[l], w.size() * 2, cudaMemcpyDeviceToHost));
        for (int n = 0; n < No; ++n)
            for (int k = 0; k < Ki; ++k) wt[(size_t)k * No + n] = w[(size_t)n * Ki + k];
        if (cudaMalloc(&v, wt.size() * 2) != cudaSuccess) return NS_ENOMEM;
        g->owned.push_back(v);
        NS_CUDA_TRY(cudaMemcpy(v, wt.data(), wt.size() * 2, cudaMemcpyHostToDevice));
        g->WT[l] = (__nv_bfloat16*)v;
    }
    g->tmHhi.resize(L); g->tmHlo.resize(L); g->tmW.resize(L); g->tmGhi.resize(L); g->tmGlo.resize(L); g->tmWT.resize(L);
    for (int l = 1; l < L; ++l) {
        const bool last = (l == L - 1);
        NS_TRY(make_tensor_map_bf16(&g->tmHhi[l], g->Hhi[l], rows_pad, p->dims[l], 128));
        NS_TRY(make_tensor_map_bf16(&g->tmHlo[l], g->Hlo[l], rows_pad, p->dims[l], 128));
        NS_TRY(make_tensor_map_bf16(&g->tmW[l], p->d_W[l], p->dims[l + 1], p->dims[l],
                                    last ? kSplitOutTile : kSplitHiddenTile));
        // backward step l reads G_{l+1} (K = dims[l+1]) from buffer (L - l - 1) % 2
        const int b = (L - l - 1) % 2;
        NS_TRY(make_tensor_map_bf16(&g->tmGhi[l], g->Ghi[b], rows_pad, p->dims[l + 1], 128));
        NS_TRY(make_tensor_map_bf16(&g->tmGlo[l], g->Glo[b], rows_pad, p->dims[l + 1], 128));
        NS_TRY(make_tensor_map_bf16(&g->tmWT[l], g->WT[l], p->dims[l], p->dims[l + 1], kSplitHiddenTile));
    }
    return NS_OK;
}

static int run_grad_split(const ns_problem* p, GradWorkspace* gw_, SplitGrad* g, const double* theta_full,
                          const int* d_nrows, int B, double* logL, double* grad, int* d_err, cudaStream_t st) {
    const int L = p->n_layers;
    const ShearParams& sp = p->sp;
    const int n_out = p->dims.back();
    // forward: input layer, hidden layers (split tanh), output layer (FP32 table)
    {
        dim3 g0((p->dims[1] + 255) / 256, B);
        adj::k_emu_in_split<<<g0, 256, 0, st>>>(theta_full, p->P, p->d_inputs, p->d_in_center, p->d_in_inv_scale,
                                                p->dims[0], (const float*)p->d_W[0], (const float*)p->d_b[0],
                                                p->dims[1], g->Hhi[1], g->Hlo[1], d_nrows);
        NS_CUDA_TRY(cudaGetLastError());
        for (int l = 1; l < L; ++l) {
            const bool last = (l == L - 1);
            if (last)
                NS_TRY(launch_gemm_split(&g->tmHhi[l], &g->tmHlo[l], &g->tmW[l], kSplitOutTile,
                                         (const float*)p->d_b[l], (const float*)p->d_out_mu, (float)p->out_sigma,
                                         gw_->table, nullptr, nullptr, nullptr, d_nrows, B, n_out, p->dims[l], SPL_OUT,
                                         d_err, st));
            else
                NS_TRY(launch_gemm_split(&g->tmHhi[l], &g->tmHlo[l], &g->tmW[l], kSplitHiddenTile,
                                         (const float*)p->d_b[l], nullptr, 0.f, g->Hhi[l + 1], g->Hlo[l + 1], nullptr,
                                         nullptr, d_nrows, B, p->dims[l + 1], p->dims[l], SPL_TANH, d_err, st));
        }
    }
    const float* tab = (const float*)gw_->table;
    if (p->n_z_emu != sp.n_z) {
        NS_TRY(launch_zinterp_generic(p, gw_->table, gw_->table_fine, d_nrows, B, (int)sizeof(float), st));
        tab = (const float*)gw_->table_fine;
    }
    NS_TRY(launch_projection_adj<float>(sp, theta_full, tab, p->d_LinvT32, p->c0, (float*)gw_->scratch,
                                        (float*)gw_->gtab, gw_->gfull, logL, d_nrows, B, st));
    // d log L / d (output pre-scaling) = sigma * d log L / d table, split
    const float* gtab = (const float*)gw_->gtab;
    if (p->n_z_emu != sp.n_z) {
        dim3 gz((p->n_z_emu * sp.n_k + 255) / 256, B);
        adj::k_zinterp_adj<float><<<gz, 256, 0, st>>>((const float*)gw_->gtab, sp.n_z, p->d_zi_row, p->d_zi_w,
                                                      (float*)gw_->gA, p->n_z_emu, sp.n_k, d_nrows);
        gtab = (const float*)gw_->gA;
    }
    {
        dim3 gs((n_out + 255) / 256, B);
        adj::k_scale_split<<<gs, 256, 0, st>>>(gtab, (float)p->out_sigma, n_out, g->Ghi[0], g->Glo[0], d_nrows);
        NS_CUDA_TRY(cudaGetLastError());
    }
    // backward: G_l = (G_{l+1} W_l) (1 - h_l^2), l = L-1 .. 1 (the last in FP32)
    for (int l = L - 1; l >= 1; --l) {
        const int out = (L - l) % 2;
        const bool first = (l == 1);
        NS_TRY(launch_gemm_split(&g->tmGhi[l], &g->tmGlo[l], &g->tmWT[l], kSplitHiddenTile, nullptr, nullptr, 0.f,
                                 first ? (void*)g->G1 : (void*)g->Ghi[out], first ? nullptr : g->Glo[out], g->Hhi[l],
                                 g->Hlo[l], d_nrows, B, p->dims[l], p->dims[l + 1],
                                 first ? SPL_DTANH32 : SPL_DTANH, d_err, st));
    }
    adj::k_emu_in_back<float><<<B, 256, 0, st>>>(g->G1, (const float*)p->d_W[0], p->dims[1], p->dims[0], p->d_inputs,
                                                 p->d_in_scale, gw_->gfull, p->P, d_nrows);
    adj::k_gather_grad<<<B, 64, 0, st>>>(gw_->gfull, p->P, p->d_free_of_full, grad, p->d, B);
    NS_CUDA_TRY(cudaGetLastError());
    return NS_OK;
}

}  // namespace gpuns

using namespace gpuns;

namespace {
struct GradState {
    const ns_problem* p = nullptr;
    GradWorkspace ws;
    GradWeights w;
    SplitGrad split;                 // BF16 problems on the tensor cores
    bool use_split = false;
    int* d_nrows = nullptr;
    int* d_err = nullptr;
    double* theta_full = nullptr;
};
std::vector<GradState*> g_grad_states;

template <typename T>
int make_grad_weights(const ns_problem* p, GradWeights* gw) {
    // FP64 problems keep FP64 master weights on the device already
    const int L = p->n_layers;
    gw->W.assign(L, nullptr);
    gw->b.assign(L, nullptr);
    if (p->precision == NS_PREC_FP64) {
        for (int l = 0; l < L; ++l) { gw->W[l] = p->d_W[l]; gw->b[l] = p->d_b[l]; }
        gw->mu = p->d_out_mu;
        return NS_OK;
    }
    if (p->precision == NS_PREC_FP32) {
        for (int l = 0; l < L; ++l) { gw->W[l] = p->d_W[l]; gw->b[l] = p->d_b[l]; }
        gw->mu = p->d_out_mu;
        return NS_OK;
    }
    // BF16 problems: the gradient path runs in FP32 from bf16-valued weights
    for (int l = 0; l < L; ++l) {
        const size_t nw = (size_t)p->dims[l + 1] * p->dims[l];
        if (l == 0) { gw->W[l] = p->d_W[l]; }
        else {
            std::vector<uint16_t> hb(nw);
            NS_CUDA_TRY(cudaMemcpy(hb.data(), p->d_W[l], nw * 2, cudaMemcpyDeviceToHost));
            std::vector<float> hf(nw);
            for (size_t i = 0; i < nw; ++i) { uint32_t u = (uint32_t)hb[i] << 16; std::memcpy(&hf[i], &u, 4); }
            void* d;
            if (cudaMalloc(&d, nw * 4) != cudaSuccess) return NS_ENOMEM;
            gw->owned.push_back(d);
            NS_CUDA_TRY(cudaMemcpy(d, hf.data(), nw * 4, cudaMemcpyHostToDevice));
            gw->W[l] = d;
        }
        gw->b[l] = p->d_b[l];
    }
    gw->mu = p->d_out_mu;
    (void)sizeof(T);
    return NS_OK;
}
}  // namespace

// Isotropic Gaussian test likelihood and its gradient at free parameters
// (every parameter of that kind is free).
__global__ void k_gauss_grad(const double* __restrict__ theta, int d, double mu, double sigma,
                             double* __restrict__ logL, double* __restrict__ grad, int B) {
    const int row = blockIdx.x * blockDim.x + threadIdx.x;
    if (row >= B) return;
    double s = 0.0;
    for (int i = 0; i < d; ++i) {
        const double r = (theta[(size_t)row * d + i] - mu) / sigma;
        s += r * r;
        grad[(size_t)row * d + i] = -r / sigma;
    }
    logL[row] = -0.5 * s - d * log(sigma * 2.5066282746310005024);
}

extern "C" int loglike_grad_batch(const ns_problem* p, const double* theta_dev, int B, double* logL_dev,
                                  double* grad_dev, void* stream) {
    if (!p || B < 0 || B > p->max_batch || (B > 0 && (!theta_dev || !logL_dev || !grad_dev))) return NS_EINVAL;
    if (p->kind != NS_KIND_SHEAR && p->kind != NS_KIND_GAUSS) return NS_ENOTSUP;
    if (B == 0) return NS_OK;
    cudaStream_t st = (cudaStream_t)stream;
    if (p->kind == NS_KIND_GAUSS) {
        if (p->d != p->P) return NS_ENOTSUP;
        k_gauss_grad<<<(B + 127) / 128, 128, 0, st>>>(theta_dev, p->d, p->g_mu, p->g_sigma, logL_dev, grad_dev, B);
        NS_CUDA_TRY(cudaGetLastError());
        return NS_OK;
    }
    GradState* gs = nullptr;
    {
        std::lock_guard<std::mutex> lk(g_grad_mu);
        for (GradState* s : g_grad_states) if (s->p == p) gs = s;
        if (!gs) {
            gs = new GradState();
            gs->p = p;
            const bool f64 = p->precision == NS_PREC_FP64;
            gs->use_split = split_supported(p);
            int rc = f64 ? grad_ws_create<double>(p, p->max_batch, &gs->ws) : grad_ws_create<float>(p, p->max_batch, &gs->ws);
            if (rc == NS_OK && gs->use_split) rc = split_grad_create(p, p->max_batch, &gs->split);
            else if (rc == NS_OK) rc = f64 ? make_grad_weights<double>(p, &gs->w) : make_grad_weights<float>(p, &gs->w);
            void* v = nullptr;
            if (rc == NS_OK && cudaMalloc(&v, sizeof(int)) != cudaSuccess) rc = NS_ENOMEM;
            gs->d_nrows = (int*)v;
            v = nullptr;
            if (rc == NS_OK && (cudaMalloc(&v, sizeof(int)) != cudaSuccess || cudaMemset(v, 0, sizeof(int)) != cudaSuccess))
                rc = NS_ENOMEM;
            gs->d_err = (int*)v;
            v = nullptr;
            if (rc == NS_OK && cudaMalloc(&v, sizeof(double) * (size_t)p->max_batch * p->P) != cudaSuccess) rc = NS_ENOMEM;
            gs->theta_full = (double*)v;
            if (rc != NS_OK) {
                for (void* q : gs->ws.owned) cudaFree(q);
                for (void* q : gs->w.owned) cudaFree(q);
                for (void* q : gs->split.owned) cudaFree(q);
                cudaFree(gs->d_nrows); cudaFree(gs->d_err); cudaFree(gs->theta_full);
                delete gs;
                return rc;
            }
            g_grad_states.push_back(gs);
        }
    }
    NS_TRY(launch_free_to_full_ext(p, theta_dev, B, gs->theta_full, st));
    k_set_int<<<1, 1, 0, st>>>(gs->d_nrows, B);
    NS_CUDA_TRY(cudaGetLastError());
    if (p->precision == NS_PREC_FP64)
        return run_grad<double>(p, &gs->ws, &gs->w, gs->theta_full, gs->d_nrows, B, logL_dev, grad_dev, st);
    if (gs->use_split)
        return run_grad_split(p, &gs->ws, &gs->split, gs->theta_full, gs->d_nrows, B, logL_dev, grad_dev, gs->d_err, st);
    return run_grad<float>(p, &gs->ws, &gs->w, gs->theta_full, gs->d_nrows, B, logL_dev, grad_dev, st);
}

// Called by ns_problem_free: release the gradient state of a problem.
void gpuns_release_grad_state(const ns_problem* p) {
    std::lock_guard<std::mutex> lk(g_grad_mu);
    for (size_t i = 0; i < g_grad_states.size(); ++i) {
        GradState* s = g_grad_states[i];
        if (s->p != p) continue;
        for (void* q : s->ws.owned) cudaFree(q);
        for (void* q : s->w.owned) cudaFree(q);
        for (void* q : s->split.owned) cudaFree(q);
        cudaFree(s->d_nrows);
        cudaFree(s->d_err);
        cudaFree(s->theta_full);
        delete s;
        g_grad_states.erase(g_grad_states.begin() + i);
        return;
    }
}
