// Batched nested slice sampling on the GPU (Sec. 2.1-2.2 of arXiv:2509.13307).
//
// Per iteration:
//   k_sort_delete   sort live log L by (log L, slot) (bitonic, one block), delete
//                   the k lowest, L* = the k-th, append them to the dead list
//                   and update log Z / log X / H in FP64 for k deletions
//                   with n, n-1, ..., n-k+1 live points (Sec. 2.2): log X by
//                   sequential subtraction, Z and H by fixed-order reductions.
//   k_live_mean,    covariance (ddof 1) of all n live cube points + ridge,
//   k_live_cov      one CTA per column mean and per entry (i, j <= i).
//   k_cholesky      FP64 Cholesky of that covariance (one block).
//   k_directions    every (chain, move) slice direction of the iteration.
//   k_chains_start  chain c starts at survivor floor(u (n - k)) (Philox START).
//   rounds          until every chain has made R slice moves: k_slice_advance
//                   (one warp per chain) consumes the previous proposals' log L,
//                   runs the hit-and-run slice state machine (Neal 2003:
//                   stepping out with width w, then shrinkage) through every
//                   decision that needs no likelihood (points outside the unit
//                   cube) and emits its proposals into a compacted batch (both
//                   ends of the slice while stepping out, one point while
//                   shrinking); the fused likelihood then scores the batch.
//                   Rounds are launched as a captured CUDA graph.
//   k_insert        chain c's point replaces the c-th deleted slot; the
//                   termination test ln(Z + X <L_live>) - ln Z < tol.
// All random numbers come from Philox4x32-10 with the counter layout shared
// with the CPU oracle, so both produce the same slice bookkeeping.
#include <algorithm>
#include <cmath>
#include <cstring>
#include <new>
#include <vector>

#include "evidence_seq.cuh"
#include "likelihood.cuh"

namespace gpuns {

enum Phase : int { PH_NEWMOVE = 0, PH_OUT = 1, PH_SHRINK = 3, PH_DONE = 4 };

struct Scalars {
    double logZ, logX, H, lstar;
    long long n_dead, iter, evals;
    int status, n_active, batch, converged;
    int batch2[2];        // round batch counters of chain group 0 (round i uses batch2[i & 1])
    int nonfinite;        // likelihood evaluations that returned NaN / inf (counted as outside)
};

struct RunDev {
    int n, k, d, R, cap_steps;
    double width, tol;
    unsigned long long seed;
    double* live_x;
    double* live_L;
    int* order;
    int* deleted;
    int* starts;
    double* chol;
    float* chol32;        // FP32 copy of chol (directions of reduced-precision problems)
    double* cov;
    double* mean;         // d column means of the live set
    double* dirs;         // k x R x d slice directions u = L_Sigma z / |z| of the iteration
    double* ch_x;
    double* ch_u;
    double* ch_L;
    double* ch_l;
    double* ch_r;
    double* ch_t;
    int* ch_phase;
    int* ch_move;
    int* ch_step;
    int* ch_step2;        // right-end step count while stepping out
    int* ch_evals;
    int* ch_row;
    int* ch_row2;         // pending right-end row while stepping out
    double* prop;         // the initial live points' cube coordinates (n x d)
    int* batch_ctr;       // row counter of the round's batch (shared by packed runs)
    int* batch_next;      // the next round's counter, zeroed by this round's slice kernel (or null)
    int run_id;
    int sh_c0, sh_c1;     // chains this run evolves: [sh_c0, sh_c1) of k (a shard of a run split over devices)
    int chain0;           // first chain of this group of rounds
    int grp_chains;       // chains of this group
    // prior transform fused into the proposal emission (Table 1)
    int P;                // full parameter count
    const int* pkind;     // per full parameter: ns_prior_kind
    const double* pa;
    const double* pb;
    const int* fof;       // free index of each full parameter, or -1
    int prior_f32;        // Gaussian priors through the FP32 Phi^-1 (reduced-precision problems)
    double* theta_full;   // rows x P, read by the likelihood
    const double* logL;   // likelihood output per proposal row
    Scalars* sc;
    double* dead_x;
    double* dead_L;
    int* dead_n;
};

__device__ inline double lse2(double a, double b) {
    if (a == -INFINITY) return b;
    if (b == -INFINITY) return a;
    const double m = fmax(a, b);
    return m + log(exp(a - m) + exp(b - m));
}

// Block-wide fixed-order reductions over per-thread partials (1024 threads max).
__device__ double block_reduce_max(double v, double* red) {
    for (int o = 16; o > 0; o >>= 1) v = fmax(v, __shfl_down_sync(0xffffffffu, v, o));
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5, nw = (blockDim.x + 31) >> 5;
    __syncthreads();
    if (lane == 0) red[w] = v;
    __syncthreads();
    if (threadIdx.x == 0) {
        double m = red[0];
        for (int i = 1; i < nw; ++i) m = fmax(m, red[i]);
        red[32] = m;
    }
    __syncthreads();
    return red[32];
}
__device__ double block_reduce_sum(double v, double* red) {
    for (int o = 16; o > 0; o >>= 1) v += __shfl_down_sync(0xffffffffu, v, o);
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5, nw = (blockDim.x + 31) >> 5;
    __syncthreads();
    if (lane == 0) red[w] = v;
    __syncthreads();
    if (threadIdx.x == 0) {
        double s = red[0];
        for (int i = 1; i < nw; ++i) s += red[i];
        red[32] = s;
    }
    __syncthreads();
    return red[32];
}

// k deletions at once, the j-th booked with n_first - j live points (Sec. 2.2),
// keys L[0..k) ascending in shared memory, tmp: k doubles of shared scratch.
// log X advances by sequential subtraction of 1/n_j (the same operations as one
// deletion at a time); the weights w_j = X_{j-1} - X_j and the updates
//   Z' = Z + sum_j w_j e^{L_j},   Z' (H' + ln Z') = Z (H + ln Z) + sum_j w_j e^{L_j} L_j
// (Skilling's evidence and information) are fixed-order block reductions.
// Called by every thread of the block; results valid in every thread.
__device__ void evidence_batch(const double* L, double* tmp, int k, int n_first, double& logZ, double& logX,
                               double& H, double* red) {
    const int tid = threadIdx.x, nt = blockDim.x;
    for (int j = tid; j < k; j += nt) tmp[j] = 1.0 / (double)(n_first - j);
    __syncthreads();
    if (tid == 0) {
        double lx = logX;
        for (int j = 0; j < k; ++j) {
            const double inv = tmp[j];
            tmp[j] = lx;              // ln X before the j-th deletion
            lx -= inv;
        }
        red[33] = lx;
    }
    __syncthreads();
    const double logX_new = red[33];
    double mloc = -INFINITY;
    for (int j = tid; j < k; j += nt) {
        const double logw = tmp[j] + log(-expm1(-1.0 / (double)(n_first - j)));
        const double c = L[j] + logw;
        tmp[j] = c;
        mloc = fmax(mloc, c);
    }
    const double m = fmax(block_reduce_max(mloc, red), logZ);
    double z_new = -INFINITY;
    if (m > -INFINITY) {
        double sl = 0.0;
        for (int j = tid; j < k; j += nt) sl += exp(tmp[j] - m);
        const double s = block_reduce_sum(sl, red) + ((logZ > -INFINITY) ? exp(logZ - m) : 0.0);
        z_new = m + log(s);
    } else {
        __syncthreads();
    }
    double h_new = 0.0;
    if (z_new > -INFINITY) {
        double hl = 0.0;
        for (int j = tid; j < k; j += nt)
            if (L[j] > -INFINITY) hl += exp(tmp[j] - z_new) * L[j];
        double hs = block_reduce_sum(hl, red);
        if (logZ > -INFINITY) hs += exp(logZ - z_new) * (H + logZ);
        h_new = hs - z_new;
    }
    __syncthreads();
    logZ = z_new;
    logX = logX_new;
    H = h_new;
}

// ------------------------------------------------------------------ init
__global__ void k_init_points(int n, int d, unsigned long long seed, double* __restrict__ prop) {
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    const int nch = (d + 1) / 2;
    for (int j = 0; j < nch; ++j) {
        Draw2 u = philox_uniforms(seed, P_INIT, j, 0, i, 0);
        prop[(size_t)i * d + 2 * j] = u.a;
        if (2 * j + 1 < d) prop[(size_t)i * d + 2 * j + 1] = u.b;
    }
}

// Chains start finished with no pending proposal until their first iteration.
__global__ void k_reset_chains(RunDev r) {
    const int c = blockIdx.x * blockDim.x + threadIdx.x;
    if (c < r.k) { r.ch_phase[c] = PH_DONE; r.ch_row[c] = -1; r.ch_row2[c] = -1; r.ch_evals[c] = 0; }
}

__global__ void k_init_finish(RunDev r, const double* __restrict__ logL) {
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i < r.n) {
        double v = logL[i];
        if (!isfinite(v)) { v = -INFINITY; atomicOr(&r.sc->status, NS_BIT_NONFINITE); atomicAdd(&r.sc->nonfinite, 1); }
        r.live_L[i] = v;
        for (int j = 0; j < r.d; ++j) r.live_x[(size_t)i * r.d + j] = r.prop[(size_t)i * r.d + j];
    }
    if (i == 0) {
        r.sc->logZ = -INFINITY; r.sc->logX = 0.0; r.sc->H = 0.0; r.sc->lstar = -INFINITY;
        r.sc->n_dead = 0; r.sc->iter = 0; r.sc->evals = r.n;
        r.sc->n_active = 0; r.sc->batch = 0; r.sc->converged = 0;
    }
}

// ------------------------------------------------------------------ sort / delete
// Bitonic sort of (logL, slot) ascending; n_pad power of two <= 4096.
__device__ inline bool key_less(double a, int ia, double b, int ib) {
    return (a < b) || (a == b && ia < ib);
}

__global__ void __launch_bounds__(1024) k_sort_delete(RunDev r, int n_pad, int delete_k, int do_dead) {
    extern __shared__ __align__(16) unsigned char smem_raw[];
    double* key = reinterpret_cast<double*>(smem_raw);
    int* idx = reinterpret_cast<int*>(key + n_pad);
    const int tid = threadIdx.x, nt = blockDim.x;
    for (int i = tid; i < n_pad; i += nt) {
        key[i] = (i < r.n) ? r.live_L[i] : INFINITY;
        idx[i] = i;
    }
    __syncthreads();
    for (int size = 2; size <= n_pad; size <<= 1) {
        for (int stride = size >> 1; stride > 0; stride >>= 1) {
            for (int i = tid; i < n_pad; i += nt) {
                const int j = i ^ stride;
                if (j > i) {
                    const bool up = ((i & size) == 0);
                    const bool gt = key_less(key[j], idx[j], key[i], idx[i]);
                    if (gt == up) {
                        const double tk = key[i]; key[i] = key[j]; key[j] = tk;
                        const int ti = idx[i]; idx[i] = idx[j]; idx[j] = ti;
                    }
                }
            }
            __syncthreads();
        }
    }
    for (int i = tid; i < r.n; i += nt) r.order[i] = idx[i];
    if (!do_dead) return;
    const int k = delete_k;
    const long long base = r.sc->n_dead;
    for (int j = tid; j < k; j += nt) {
        r.deleted[j] = idx[j];
        r.dead_L[base + j] = key[j];
        r.dead_n[base + j] = r.n - j;
    }
    for (int t = tid; t < k * r.d; t += nt) {
        const int j = t / r.d, c = t % r.d;
        r.dead_x[(base + j) * r.d + c] = r.live_x[(size_t)idx[j] * r.d + c];
    }
    __shared__ double red[34];
    double* tmp = reinterpret_cast<double*>(idx + n_pad);
    double logZ = r.sc->logZ, logX = r.sc->logX, H = r.sc->H;
    __syncthreads();
    evidence_batch(key, tmp, k, r.n, logZ, logX, H, red);
    if (tid == 0) {
        r.sc->logZ = logZ; r.sc->logX = logX; r.sc->H = H;
        r.sc->lstar = key[k - 1];
        r.sc->n_dead = base + k;
    }
}

// ------------------------------------------------------------------ covariance + Cholesky
// Column means of the n live cube points (one CTA per dimension).
__global__ void __launch_bounds__(256) k_live_mean(RunDev r) {
    const int c = blockIdx.x, d = r.d, n = r.n;
    __shared__ double red[32];
    double s = 0.0;
    for (int p = threadIdx.x; p < n; p += blockDim.x) s += r.live_x[(size_t)p * d + c];
    s = block_sum(s, red);
    if (threadIdx.x == 0) r.mean[c] = s / n;
}

// Covariance (ddof 1) + ridge: one CTA per pair j <= i (pairs numbered row by row).
__global__ void __launch_bounds__(256) k_live_cov(RunDev r, double ridge) {
    int i = (int)((sqrt(8.0 * blockIdx.x + 1.0) - 1.0) * 0.5);
    while ((i + 1) * (i + 2) / 2 <= (int)blockIdx.x) ++i;
    while (i * (i + 1) / 2 > (int)blockIdx.x) --i;
    const int j = blockIdx.x - i * (i + 1) / 2;
    const int d = r.d, n = r.n;
    __shared__ double red[32];
    const double mi = r.mean[i], mj = r.mean[j];
    double s = 0.0;
    for (int p = threadIdx.x; p < n; p += blockDim.x)
        s += (r.live_x[(size_t)p * d + i] - mi) * (r.live_x[(size_t)p * d + j] - mj);
    s = block_sum(s, red);
    if (threadIdx.x == 0) {
        double v = s / (n - 1);
        if (j == i) v += ridge;
        r.cov[i * d + j] = v;
        r.cov[j * d + i] = v;
    }
}

__global__ void k_cholesky(RunDev r) {
    const int d = r.d;
    __shared__ double A[64 * 64];
    __shared__ double red[32];
    __shared__ int bad;
    for (int t = threadIdx.x; t < d * d; t += blockDim.x) A[t] = r.cov[t];
    if (threadIdx.x == 0) bad = 0;
    __syncthreads();
    for (int j = 0; j < d; ++j) {
        double s = 0.0;
        for (int q = threadIdx.x; q < j; q += blockDim.x) s += A[j * d + q] * A[j * d + q];
        s = block_sum(s, red);
        if (threadIdx.x == 0) {
            const double v = A[j * d + j] - s;
            if (!(v > 0.0)) bad = 1;
            A[j * d + j] = sqrt(fmax(v, 1e-300));
        }
        __syncthreads();
        const double ljj = A[j * d + j];
        for (int i = j + 1 + threadIdx.x; i < d; i += blockDim.x) {
            double t = A[i * d + j];
            for (int q = 0; q < j; ++q) t -= A[i * d + q] * A[j * d + q];
            A[i * d + j] = t / ljj;
        }
        __syncthreads();
    }
    for (int t = threadIdx.x; t < d * d; t += blockDim.x) {
        const int i = t / d, j = t % d;
        r.chol[t] = (j <= i) ? A[t] : 0.0;
        r.chol32[t] = (j <= i) ? (float)A[t] : 0.f;
    }
    if (threadIdx.x == 0 && bad) atomicOr(&r.sc->status, NS_BIT_NONFINITE);
}

// ------------------------------------------------------------------ chains
__global__ void k_chains_start(RunDev r) {
    const int c = blockIdx.x * blockDim.x + threadIdx.x;
    const int it = (int)r.sc->iter;
    if (c < r.k) {
        const Draw2 u = philox_uniforms(r.seed, P_START, 0, (uint32_t)it, (uint32_t)c, 0);
        const int s = r.order[r.k + (int)floor(u.a * (double)(r.n - r.k))];
        r.starts[c] = s;
        for (int j = 0; j < r.d; ++j) r.ch_x[(size_t)c * r.d + j] = r.live_x[(size_t)s * r.d + j];
        r.ch_L[c] = r.live_L[s];
        r.ch_phase[c] = PH_NEWMOVE;
        r.ch_move[c] = 0;
        r.ch_step[c] = 0;
        r.ch_step2[c] = 0;
        r.ch_evals[c] = 0;
        r.ch_row[c] = -1;
        r.ch_row2[c] = -1;
    }
    if (c == 0) {
        r.sc->n_active = r.sh_c1 - r.sh_c0;
        r.sc->batch = 0; r.sc->batch2[0] = 0; r.sc->batch2[1] = 0;
    }
}

// Slice directions for every (chain, move) of the iteration, one warp each:
// z ~ N(0, I) by Box-Muller on the Philox DIR chunks, u = L_Sigma (z / |z|).
// They depend only on the counters and the iteration's Cholesky factor, so
// they are formed once, fully parallel, instead of inside the latency-bound
// round (FP64 transcendentals run at a small fraction of the FP32 rate).
__global__ void __launch_bounds__(256) k_directions(RunDev r) {
    __shared__ double zs[8][64];
    __shared__ float zsf[8][64];
    const int wib = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const long long g = (long long)blockIdx.x * 8 + wib;
    if (g >= (long long)(r.sh_c1 - r.sh_c0) * r.R) return;
    const int c = r.sh_c0 + (int)(g / r.R), move = (int)(g % r.R);
    const int d = r.d;
    const int it = (int)r.sc->iter;
    double* zsw = zs[wib];
    const int nch = (d + 1) / 2;
    if (r.prior_f32) {
        // reduced-precision problems: the same Philox draws, Box-Muller and
        // the triangular product in FP32 (GB300's FP64 pipe is a small
        // fraction of its FP32 rate); the direction is stored in FP64
        float f0 = 0.f, f1 = 0.f;
        if (lane < nch) {
            const Draw2 q = philox_uniforms(r.seed, P_DIR, lane, (uint32_t)it, (uint32_t)c, (uint32_t)move);
            const float rad = sqrtf(-2.f * logf((float)q.a));
            float sn, cs;
            sincospif(2.f * (float)q.b, &sn, &cs);
            f0 = rad * cs;
            f1 = (2 * lane + 1 < d) ? rad * sn : 0.f;
        }
        const float nrm = sqrtf(warp_sum(f0 * f0 + f1 * f1));
        float* zf = zsf[wib];
        if (lane < nch) {
            zf[2 * lane] = f0 / nrm;
            if (2 * lane + 1 < d) zf[2 * lane + 1] = f1 / nrm;
        }
        __syncwarp();
        double* outf = r.dirs + ((size_t)c * r.R + move) * d;
        if (lane < d) {
            float a0 = 0.f;
            for (int b = 0; b <= lane; ++b) a0 = fmaf(r.chol32[lane * d + b], zf[b], a0);
            outf[lane] = (double)a0;
        }
        if (lane + 32 < d) {
            float a1 = 0.f;
            for (int b = 0; b <= lane + 32; ++b) a1 = fmaf(r.chol32[(lane + 32) * d + b], zf[b], a1);
            outf[lane + 32] = (double)a1;
        }
        return;
    }
    double z0 = 0.0, z1 = 0.0;
    if (lane < nch) {
        const Draw2 q = philox_uniforms(r.seed, P_DIR, lane, (uint32_t)it, (uint32_t)c, (uint32_t)move);
        const double rad = sqrt(-2.0 * log(q.a));
        double sn, cs;
        sincos(6.283185307179586 * q.b, &sn, &cs);
        z0 = rad * cs;
        z1 = (2 * lane + 1 < d) ? rad * sn : 0.0;
    }
    const double nrm = sqrt(warp_sum(z0 * z0 + z1 * z1));
    // z / |z| once per component (each quotient computed by one lane)
    if (lane < nch) {
        zsw[2 * lane] = z0 / nrm;
        if (2 * lane + 1 < d) zsw[2 * lane + 1] = z1 / nrm;
    }
    __syncwarp();
    double* out = r.dirs + ((size_t)c * r.R + move) * d;
    if (lane < d) {
        double a0 = 0.0;
        for (int b = 0; b <= lane; ++b) a0 += r.chol[lane * d + b] * zsw[b];
        out[lane] = a0;
    }
    if (lane + 32 < d) {
        double a1 = 0.0;
        for (int b = 0; b <= lane + 32; ++b) a1 += r.chol[(lane + 32) * d + b] * zsw[b];
        out[lane + 32] = a1;
    }
}

// Prior-transform constants (Table 1) of the full parameters lane and
// lane + 32, read once per chain: they are problem constants, so a kernel may
// read them before its dependency wait.  Parameters from 64 on are read when
// a row is written.
struct PriorRegs {
    int f0, f1, kind0, kind1;
    double a0, a1, b0, b1;
};
__device__ __forceinline__ PriorRegs load_prior_regs(const RunDev& r, int lane) {
    PriorRegs q;
    const int i0 = lane, i1 = lane + 32;
    q.f0 = (i0 < r.P) ? r.fof[i0] : -1;
    q.kind0 = (i0 < r.P) ? r.pkind[i0] : 0;
    q.a0 = (i0 < r.P) ? r.pa[i0] : 0.0;
    q.b0 = (i0 < r.P) ? r.pb[i0] : 0.0;
    q.f1 = (i1 < r.P) ? r.fof[i1] : -1;
    q.kind1 = (i1 < r.P) ? r.pkind[i1] : 0;
    q.a1 = (i1 < r.P) ? r.pa[i1] : 0.0;
    q.b1 = (i1 < r.P) ? r.pb[i1] : 0.0;
    return q;
}

// Physical parameters of proposal row `row` (Table 1 prior transform), written
// by the chain's warp: lane l writes the full parameters l, l + 32, ... and
// fetches each one's cube coordinate from the lane holding it (y0: dims < 32,
// y1: dims >= 32).
__device__ __forceinline__ void emit_theta(const RunDev& r, const PriorRegs& q, int row, double y0, double y1,
                                           int lane) {
    for (int i0 = 0; i0 < r.P; i0 += 32) {          // the same trip count in every lane
        const int i = i0 + lane;
        int f, kind;
        double a, b;
        if (i0 == 0) { f = q.f0; kind = q.kind0; a = q.a0; b = q.b0; }
        else if (i0 == 32) { f = q.f1; kind = q.kind1; a = q.a1; b = q.b1; }
        else {
            f = (i < r.P) ? r.fof[i] : -1;
            kind = (i < r.P) ? r.pkind[i] : 0;
            a = (i < r.P) ? r.pa[i] : 0.0;
            b = (i < r.P) ? r.pb[i] : 0.0;
        }
        const int src = (f >= 0) ? (f & 31) : 0;
        const double c0 = __shfl_sync(0xffffffffu, y0, src);
        const double c1 = __shfl_sync(0xffffffffu, y1, src);
        if (i < r.P) {
            double v;
            if (f < 0) {
                v = a;
            } else {
                const double c = (f < 32) ? c0 : c1;
                if (kind == NS_PRIOR_UNIFORM) v = a + (b - a) * c;
                else v = a + b * gauss_quantile(c, r.prior_f32 != 0);
            }
            r.theta_full[(size_t)row * r.P + i] = v;
        }
    }
}

// One warp per chain; lanes own dimensions lane and lane + 32.
// Stepping out (Neal 2003) widens the two ends of the slice independently:
// the left end's tests never depend on the right end's and neither draws
// random numbers, so both ends are proposed in the same round (up to two rows
// per chain).  The points evaluated, their order within each end, the caps,
// the final interval and every random number are those of widening the left
// end first and then the right, so the bookkeeping equals the sequential
// sampler's exactly.  Phase word: phase | done_ends << 8 (bit 0 left, bit 1
// right); ch_row / ch_row2 hold the pending left (or shrinkage) / right rows,
// ch_step / ch_step2 the left (or shrinkage) / right step counts.
__device__ void advance_chain(const RunDev& r, const PriorRegs& q, int c, int lane) {
    const int pw = r.ch_phase[c];
    int phase = pw & 0xff, ends = (pw >> 8) & 3;
    if (phase == PH_DONE) return;
    const int d = r.d;
    const int it = (int)r.sc->iter;
    const double w = r.width;
    const double lstar = r.sc->lstar;
    double* x = r.ch_x + (size_t)c * d;
    double* u = r.ch_u + (size_t)c * d;
    const bool has0 = lane < d, has1 = lane + 32 < d;
    double x0 = has0 ? x[lane] : 0.0, x1 = has1 ? x[lane + 32] : 0.0;
    double u0v = has0 ? u[lane] : 0.0, u1v = has1 ? u[lane + 32] : 0.0;
    int move = r.ch_move[c], step = r.ch_step[c], step2 = r.ch_step2[c];
    int row = r.ch_row[c], row2 = r.ch_row2[c], evals = r.ch_evals[c];
    double l = r.ch_l[c], rr = r.ch_r[c], t = r.ch_t[c], chL = r.ch_L[c];
    int flags = 0, n_nonfinite = 0;
    auto inside_of = [&](int rw) {
        const double v = r.logL[rw];
        const bool fin = isfinite(v);
        if (!fin) { flags |= NS_BIT_NONFINITE; ++n_nonfinite; }
        return fin && (v > lstar);
    };

    if (phase == PH_OUT) {
        if (row >= 0) { if (inside_of(row)) { l -= w; ++step; } else ends |= 1; row = -1; }
        if (row2 >= 0) { if (inside_of(row2)) { rr += w; ++step2; } else ends |= 2; row2 = -1; }
    } else if (phase == PH_SHRINK && row >= 0) {
        const double v = r.logL[row];
        if (inside_of(row)) {
            x0 = __dadd_rn(x0, __dmul_rn(t, u0v));
            x1 = __dadd_rn(x1, __dmul_rn(t, u1v));
            chL = v;
            ++move;
            phase = PH_NEWMOVE;
        } else {
            if (t < 0.0) l = t; else rr = t;
            ++step;
        }
        row = -1;
    }
    // the proposal at s along the direction, or -1 (no evaluation) when it
    // leaves the open unit cube
    auto propose = [&](double s) -> int {
        const double y0 = __dadd_rn(x0, __dmul_rn(s, u0v)), y1 = __dadd_rn(x1, __dmul_rn(s, u1v));
        const bool inc = (!has0 || (y0 > 0.0 && y0 < 1.0)) && (!has1 || (y1 > 0.0 && y1 < 1.0));
        if (!__all_sync(0xffffffffu, inc)) return -1;
        int rw = 0;
        if (lane == 0) rw = atomicAdd(r.batch_ctr, 1);
        rw = __shfl_sync(0xffffffffu, rw, 0);
        emit_theta(r, q, rw, has0 ? y0 : 0.0, has1 ? y1 : 0.0, lane);
        ++evals;
        return rw;
    };
    for (int guard = 0; guard < 4 * r.cap_steps + 8; ++guard) {
        if (phase == PH_NEWMOVE) {
            if (move >= r.R) { phase = PH_DONE; break; }
            // direction of this move (k_directions)
            const double* dir = r.dirs + ((size_t)c * r.R + move) * d;
            u0v = has0 ? dir[lane] : 0.0;
            u1v = has1 ? dir[lane + 32] : 0.0;
            const double s0 = philox_uniforms(r.seed, P_STEPOUT, 0, (uint32_t)it, (uint32_t)c, (uint32_t)move).a;
            l = __dmul_rn(-w, s0);
            rr = l + w;
            phase = PH_OUT;
            ends = 0;
            step = step2 = 0;
            continue;
        }
        if (phase == PH_OUT) {
            // both ends' cube tests first, then one atomic for the rows they need
            bool okl = false, okr = false;
            double yl0 = 0.0, yl1 = 0.0, yr0 = 0.0, yr1 = 0.0;
            if (!(ends & 1) && row < 0) {
                if (step >= r.cap_steps) { flags |= NS_BIT_SLICE_CAP; ends |= 1; }
                else {
                    yl0 = __dadd_rn(x0, __dmul_rn(l, u0v));
                    yl1 = __dadd_rn(x1, __dmul_rn(l, u1v));
                    okl = __all_sync(0xffffffffu, (!has0 || (yl0 > 0.0 && yl0 < 1.0)) && (!has1 || (yl1 > 0.0 && yl1 < 1.0)));
                    if (!okl) ends |= 1;
                }
            }
            if (!(ends & 2) && row2 < 0) {
                if (step2 >= r.cap_steps) { flags |= NS_BIT_SLICE_CAP; ends |= 2; }
                else {
                    yr0 = __dadd_rn(x0, __dmul_rn(rr, u0v));
                    yr1 = __dadd_rn(x1, __dmul_rn(rr, u1v));
                    okr = __all_sync(0xffffffffu, (!has0 || (yr0 > 0.0 && yr0 < 1.0)) && (!has1 || (yr1 > 0.0 && yr1 < 1.0)));
                    if (!okr) ends |= 2;
                }
            }
            if (okl || okr) {
                int base = 0;
                if (lane == 0) base = atomicAdd(r.batch_ctr, (okl ? 1 : 0) + (okr ? 1 : 0));
                base = __shfl_sync(0xffffffffu, base, 0);
                if (okl) {
                    row = base;
                    emit_theta(r, q, row, has0 ? yl0 : 0.0, has1 ? yl1 : 0.0, lane);
                    ++evals;
                }
                if (okr) {
                    row2 = base + (okl ? 1 : 0);
                    emit_theta(r, q, row2, has0 ? yr0 : 0.0, has1 ? yr1 : 0.0, lane);
                    ++evals;
                }
            }
            if (ends == 3) { phase = PH_SHRINK; step = 0; continue; }
            break;                                  // an end is being evaluated
        }
        if (phase == PH_SHRINK) {
            if (step >= r.cap_steps) {
                flags |= NS_BIT_SLICE_CAP;
                ++move;
                phase = PH_NEWMOVE;
                continue;
            }
            const double us = philox_uniforms(r.seed, P_SHRINK, (uint32_t)step, (uint32_t)it, (uint32_t)c,
                                              (uint32_t)move).a;
            t = __dadd_rn(l, __dmul_rn(us, __dsub_rn(rr, l)));
            if ((row = propose(t)) < 0) {
                if (t < 0.0) l = t; else rr = t;
                ++step;
                continue;
            }
            break;
        }
        break;
    }
    if (has0) { x[lane] = x0; u[lane] = u0v; }
    if (has1) { x[lane + 32] = x1; u[lane + 32] = u1v; }
    if (lane == 0) {
        r.ch_phase[c] = phase | (ends << 8); r.ch_move[c] = move; r.ch_step[c] = step; r.ch_step2[c] = step2;
        r.ch_row[c] = row; r.ch_row2[c] = row2;
        r.ch_evals[c] = evals; r.ch_l[c] = l; r.ch_r[c] = rr; r.ch_t[c] = t; r.ch_L[c] = chL;
        if (flags) atomicOr(&r.sc->status, flags);
        if (n_nonfinite) atomicAdd(&r.sc->nonfinite, n_nonfinite);
        if (phase == PH_DONE) atomicSub(&r.sc->n_active, 1);
    }
}

// One warp per chain of the group [chain0, chain0 + grp_chains), one warp per
// CTA: the chains' FP64 arithmetic (positions, prior transform) spreads over
// the FP64 units of every SM instead of a few.
constexpr int kSliceWarps = 1;
__global__ void __launch_bounds__(32 * kSliceWarps) k_slice_advance(RunDev r) {
    const PriorRegs q = load_prior_regs(r, threadIdx.x & 31);   // problem constants
    pdl_begin();
    // the previous round (the last reader of the other counter) has completed
    if (blockIdx.x == 0 && threadIdx.x == 0 && r.batch_next) *r.batch_next = 0;
    const int c = blockIdx.x * kSliceWarps + (threadIdx.x >> 5);
    if (c >= r.grp_chains) return;
    advance_chain(r, q, r.chain0 + c, threadIdx.x & 31);
}

// All chains of several packed runs: global warp g -> (run, chain) through the
// prefix offsets chain_off[0..n_runs].
__global__ void __launch_bounds__(32 * kSliceWarps) k_slice_advance_multi(const RunDev* __restrict__ runs,
                                                                          const int* __restrict__ chain_off,
                                                                          int n_runs) {
    const int g = blockIdx.x * kSliceWarps + (threadIdx.x >> 5);
    if (g >= chain_off[n_runs]) return;
    int r = 0;
    while (r + 1 < n_runs && chain_off[r + 1] <= g) ++r;
    const RunDev rd = runs[r];
    advance_chain(rd, load_prior_regs(rd, threadIdx.x & 31), g - chain_off[r], threadIdx.x & 31);
}

// A shard's final chain states for the exchange between devices: row c - sh_c0
// of out = (x[0..d), log L, evaluations) of chain c in [sh_c0, sh_c1).
__global__ void k_shard_pack(RunDev r, double* __restrict__ out) {
    const int w = r.d + 2;
    const int nc = r.sh_c1 - r.sh_c0;
    for (int t = blockIdx.x * blockDim.x + threadIdx.x; t < nc * w; t += gridDim.x * blockDim.x) {
        const int i = t / w, j = t % w, c = r.sh_c0 + i;
        out[t] = (j < r.d) ? r.ch_x[(size_t)c * r.d + j] : (j == r.d) ? r.ch_L[c] : (double)r.ch_evals[c];
    }
}

// Every chain's final state (k rows in chain order, as k_shard_pack writes
// them) into the chain arrays, for k_insert.
__global__ void k_shard_unpack(RunDev r, const double* __restrict__ in) {
    const int w = r.d + 2;
    for (int t = blockIdx.x * blockDim.x + threadIdx.x; t < r.k * w; t += gridDim.x * blockDim.x) {
        const int c = t / w, j = t % w;
        const double v = in[t];
        if (j < r.d) r.ch_x[(size_t)c * r.d + j] = v;
        else if (j == r.d) r.ch_L[c] = v;
        else r.ch_evals[c] = (int)v;
    }
}

__global__ void k_insert(RunDev r) {
    __shared__ double red[32];
    __shared__ long long ev_sh;
    const int tid = threadIdx.x, nt = blockDim.x;
    if (tid == 0) ev_sh = 0;
    __syncthreads();
    long long ev = 0;
    for (int c = tid; c < r.k; c += nt) {
        const int s = r.deleted[c];
        r.live_L[s] = r.ch_L[c];
        for (int j = 0; j < r.d; ++j) r.live_x[(size_t)s * r.d + j] = r.ch_x[(size_t)c * r.d + j];
        ev += r.ch_evals[c];
    }
    atomicAdd((unsigned long long*)&ev_sh, (unsigned long long)ev);
    __syncthreads();
    // termination: ln(Z + X mean(L_live)) - ln Z < tol
    // block max
    double mx = -INFINITY;
    for (int i = tid; i < r.n; i += nt) mx = fmax(mx, r.live_L[i]);
    mx = warp_max(mx);
    if ((tid & 31) == 0) red[tid >> 5] = mx;
    __syncthreads();
    if (tid < 32) {
        double v = (tid < (nt + 31) / 32) ? red[tid] : -INFINITY;
        v = warp_max(v);
        if (tid == 0) red[0] = v;
    }
    __syncthreads();
    mx = red[0];
    __syncthreads();
    double s = 0.0;
    if (mx > -INFINITY)
        for (int i = tid; i < r.n; i += nt) s += exp(r.live_L[i] - mx);
    s = block_sum(s, red);
    if (tid == 0) {
        r.sc->evals += ev_sh;
        r.sc->iter += 1;
        const double lz = r.sc->logZ;
        const double lzl = (mx > -INFINITY) ? r.sc->logX + mx + log(s) - log((double)r.n) : -INFINITY;
        r.sc->converged = (lz > -INFINITY) && (lse2(lz, lzl) - lz < r.tol);
    }
}

// ------------------------------------------------------------------ evidence
// The live points added at the end in ascending order with n, n-1, ..., 1 live points.
__global__ void __launch_bounds__(1024) k_final_evidence(RunDev r, double* out /* logZ, logX, H */) {
    extern __shared__ __align__(16) unsigned char smem_raw[];
    double* L = reinterpret_cast<double*>(smem_raw);
    double* tmp = L + r.n;
    __shared__ double red[34];
    for (int j = threadIdx.x; j < r.n; j += blockDim.x) L[j] = r.live_L[r.order[j]];
    double logZ = r.sc->logZ, logX = r.sc->logX, H = r.sc->H;
    __syncthreads();
    evidence_batch(L, tmp, r.n, r.n, logZ, logX, H, red);
    if (threadIdx.x == 0) { out[0] = logZ; out[1] = logX; out[2] = H; }
}

// One block per replay: ln t_i = ln(U_{s,i}) / n_i; ln Z_s = LSE_i(L_i + ln X_{i-1} + ln(1 - t_i)).
__global__ void __launch_bounds__(256) k_err_replays(RunDev r, long long n_dead, double* __restrict__ out) {
    extern __shared__ __align__(16) unsigned char smem_raw[];
    double* red = reinterpret_cast<double*>(smem_raw);     // 128 doubles
    const int s = blockIdx.x;
    auto Lof = [&](long long i) -> double { return (i < n_dead) ? r.dead_L[i] : r.live_L[r.order[i - n_dead]]; };
    auto nof = [&](long long i) -> int { return (i < n_dead) ? r.dead_n[i] : (int)(r.n - (i - n_dead)); };
    auto lnt = [&](long long i) -> double {
        const Draw2 u = philox_uniforms(r.seed, P_ERR, 0, (uint32_t)s, (uint32_t)i, 0);
        return log(u.a) / nof(i);
    };
    const double lz = sequence_logZ(Lof, n_dead + r.n, lnt, red, nullptr);
    if (threadIdx.x == 0) out[s] = lz;
}

}  // namespace gpuns

using namespace gpuns;

struct ns_run {
    const ns_problem* p = nullptr;
    ns_config cfg{};
    int n = 0, k = 0, d = 0, R = 0, n_pad = 0;
    cudaStream_t st = nullptr;
    Workspace ws;
    RunDev rd{};
    Scalars* sc = nullptr;
    Scalars* h_sc = nullptr;          // pinned mirror
    long long dead_cap = 0;
    std::vector<void*> owned;
    cudaStream_t cap_st = nullptr;    // private stream used only to capture the round graph
    cudaGraphExec_t graph = nullptr;
    int graph_rounds = 0;
    long long rounds = 0;
    int last_valid = 0;
    StageProbe probe;                 // optional timing of one stage in round 0 of each graph launch
    double prof_ms = 0.0;
    long long prof_launches = 0, prof_rows = 0;
    // chain groups: group 0 uses rd / ws; group 1 (chains [k0, k)) its own
    // batch, proposals and likelihood workspace, with rounds on a second stream
    int n_groups = 1, k0 = 0;
    int n_shards = 1;             // > 1: this run evolves one shard of the chains (ns_shard_*)
    int shard_pending = 0;        // an iteration's chains evolved, waiting for ns_shard_insert
    int* grp1_ctr = nullptr;      // chain group 1's pair of round batch counters
    Workspace ws1;
    RunDev grd[2]{};
    cudaStream_t cap_st1 = nullptr;
    cudaEvent_t ev_gfork = nullptr, ev_gjoin = nullptr;
};

static int run_alloc(ns_run* r, size_t bytes, void** p) {
    if (cudaMalloc(p, bytes) != cudaSuccess) return NS_ENOMEM;
    r->owned.push_back(*p);
    return NS_OK;
}

static int grow_dead(ns_run* r, long long need) {
    if (need <= r->dead_cap) return NS_OK;
    long long cap = std::max(need, 2 * r->dead_cap + 4 * (long long)r->n);
    double *x, *L;
    int* nl;
    if (cudaMalloc(&x, sizeof(double) * cap * r->d) != cudaSuccess) return NS_ENOMEM;
    if (cudaMalloc(&L, sizeof(double) * cap) != cudaSuccess) { cudaFree(x); return NS_ENOMEM; }
    if (cudaMalloc(&nl, sizeof(int) * cap) != cudaSuccess) { cudaFree(x); cudaFree(L); return NS_ENOMEM; }
    NS_CUDA_TRY(cudaStreamSynchronize(r->st));
    const long long used = r->h_sc->n_dead;
    if (r->rd.dead_x && used > 0) {
        NS_CUDA_TRY(cudaMemcpy(x, r->rd.dead_x, sizeof(double) * used * r->d, cudaMemcpyDeviceToDevice));
        NS_CUDA_TRY(cudaMemcpy(L, r->rd.dead_L, sizeof(double) * used, cudaMemcpyDeviceToDevice));
        NS_CUDA_TRY(cudaMemcpy(nl, r->rd.dead_n, sizeof(int) * used, cudaMemcpyDeviceToDevice));
    }
    cudaFree(r->rd.dead_x); cudaFree(r->rd.dead_L); cudaFree(r->rd.dead_n);
    r->rd.dead_x = x; r->rd.dead_L = L; r->rd.dead_n = nl;
    r->dead_cap = cap;
    if (r->graph) { cudaGraphExecDestroy(r->graph); r->graph = nullptr; }
    return NS_OK;
}

static int sync_scalars(ns_run* r) {
    NS_CUDA_TRY(cudaMemcpyAsync(r->h_sc, r->sc, sizeof(Scalars), cudaMemcpyDeviceToHost, r->st));
    NS_TRY(workspace_err_fetch(&r->ws, r->st));
    if (r->n_groups > 1) NS_TRY(workspace_err_fetch(&r->ws1, r->st));
    NS_CUDA_TRY(cudaStreamSynchronize(r->st));
    if (const int bits = workspace_err_bits(&r->ws) | (r->n_groups > 1 ? workspace_err_bits(&r->ws1) : 0)) {
        r->h_sc->status |= bits;
        return NS_ETIMEOUT;
    }
    return NS_OK;
}

// Round i of a captured launch: the batch counts into counter i & 1 of the
// group's pair, and the slice kernel zeroes the other one for round i + 1
// (no separate reset launch; launches hold an even number of rounds, so each
// starts on counter 0, and every iteration starts with both zero).
static int launch_round(ns_run* r, int g, int i, cudaStream_t st, const StageProbe* probe) {
    Workspace* ws = g ? &r->ws1 : &r->ws;
    int* pair = g ? r->grp1_ctr : r->rd.sc->batch2;
    RunDev rd = r->grd[g];
    rd.batch_ctr = pair + (i & 1);
    rd.batch_next = pair + ((i + 1) & 1);
    int* const saved = ws->d_nrows;
    ws->d_nrows = rd.batch_ctr;
    int s = NS_OK;
    if (launch_pdl(k_slice_advance, dim3((rd.grp_chains + kSliceWarps - 1) / kSliceWarps), dim3(32 * kSliceWarps), 0,
                   st, rd) != cudaSuccess)
        s = NS_ECUDA;
    // up to two proposals per chain (both stepping-out ends)
    if (s == NS_OK) s = run_likelihood(r->p, ws, 2 * rd.grp_chains, ws->logL, nullptr, st, probe);
    ws->d_nrows = saved;
    return s;
}

// Per-group copies of the run state for the round kernels (rebuilt with the
// graph, since the dead-list pointers in rd change when it grows).
static void refresh_groups(ns_run* r) {
    r->grd[0] = r->rd;
    r->grd[0].chain0 = r->rd.sh_c0;
    r->grd[0].grp_chains = r->n_groups > 1 ? r->k0 : r->rd.sh_c1 - r->rd.sh_c0;
    if (r->n_groups > 1) {
        RunDev& g1 = r->grd[1];
        g1 = r->rd;
        g1.chain0 = r->k0;
        g1.grp_chains = r->k - r->k0;
        g1.batch_ctr = r->ws1.d_nrows;
        g1.logL = r->ws1.logL;
        g1.theta_full = r->ws1.theta_full;
        g1.prop = r->rd.prop + (size_t)r->k0 * r->d;   // disjoint rows of the proposal buffer
    }
}

static int build_graph(ns_run* r, int rounds) {
    if (r->graph) { cudaGraphExecDestroy(r->graph); r->graph = nullptr; }
    refresh_groups(r);
    cudaGraph_t g;
    int lo = 0, hi = 0;
    NS_CUDA_TRY(cudaDeviceGetStreamPriorityRange(&lo, &hi));
    if (!r->cap_st) {
        // the round's main chain at the highest priority, so the emulator GEMMs
        // are scheduled ahead of the windows stage running beside them
        NS_CUDA_TRY(cudaStreamCreateWithPriority(&r->cap_st, cudaStreamNonBlocking, hi));
    }
    if (r->n_groups > 1 && !r->cap_st1) {
        NS_CUDA_TRY(cudaStreamCreateWithPriority(&r->cap_st1, cudaStreamNonBlocking, hi));
        NS_CUDA_TRY(cudaEventCreateWithFlags(&r->ev_gfork, cudaEventDisableTiming));
        NS_CUDA_TRY(cudaEventCreateWithFlags(&r->ev_gjoin, cudaEventDisableTiming));
    }
    NS_CUDA_TRY(cudaStreamBeginCapture(r->cap_st, cudaStreamCaptureModeThreadLocal));
    int s = NS_OK;
    if (r->n_groups > 1) {
        // the two groups' rounds are independent chains of kernels on two streams
        if (cudaEventRecord(r->ev_gfork, r->cap_st) != cudaSuccess ||
            cudaStreamWaitEvent(r->cap_st1, r->ev_gfork, 0) != cudaSuccess)
            s = NS_ECUDA;
    }
    for (int i = 0; i < rounds && s == NS_OK; ++i)
        s = launch_round(r, 0, i, r->cap_st, (i == 0 && r->probe.stage != PROBE_NONE) ? &r->probe : nullptr);
    if (r->n_groups > 1) {
        for (int i = 0; i < rounds && s == NS_OK; ++i) s = launch_round(r, 1, i, r->cap_st1, nullptr);
        if (s == NS_OK && (cudaEventRecord(r->ev_gjoin, r->cap_st1) != cudaSuccess ||
                           cudaStreamWaitEvent(r->cap_st, r->ev_gjoin, 0) != cudaSuccess))
            s = NS_ECUDA;
    }
    cudaError_t e = cudaStreamEndCapture(r->cap_st, &g);
    if (s != NS_OK) { if (e == cudaSuccess) cudaGraphDestroy(g); return s; }
    NS_CUDA_TRY(e);
    e = cudaGraphInstantiate(&r->graph, g, cudaGraphInstantiateFlagUseNodePriority);
    cudaGraphDestroy(g);
    NS_CUDA_TRY(e);
    r->graph_rounds = rounds;
    return NS_OK;
}

static void run_release(ns_run* r) {
    if (!r) return;
    if (r->graph) cudaGraphExecDestroy(r->graph);
    if (r->cap_st) cudaStreamDestroy(r->cap_st);
    if (r->probe.ev0) cudaEventDestroy(r->probe.ev0);
    if (r->probe.ev1) cudaEventDestroy(r->probe.ev1);
    if (r->probe.h_rows) cudaFreeHost(r->probe.h_rows);
    cudaFree(r->rd.dead_x); cudaFree(r->rd.dead_L); cudaFree(r->rd.dead_n);
    for (void* q : r->owned) cudaFree(q);
    if (r->h_sc) cudaFreeHost(r->h_sc);
    workspace_free(&r->ws);
    workspace_free(&r->ws1);
    if (r->cap_st1) cudaStreamDestroy(r->cap_st1);
    if (r->ev_gfork) cudaEventDestroy(r->ev_gfork);
    if (r->ev_gjoin) cudaEventDestroy(r->ev_gjoin);
    delete r;
}

static int engine_kernel_attributes() {
    static bool done = false;
    if (done) return NS_OK;
    // live sets up to 4096 points: keys, slots and k weights in shared memory
    NS_CUDA_TRY(cudaFuncSetAttribute(k_sort_delete, cudaFuncAttributeMaxDynamicSharedMemorySize, 96 * 1024));
    NS_CUDA_TRY(cudaFuncSetAttribute(k_final_evidence, cudaFuncAttributeMaxDynamicSharedMemorySize, 96 * 1024));
    done = true;
    return NS_OK;
}

extern "C" int ns_init(const ns_problem* p, const ns_config* cfg, void* stream, ns_run** out) {
    if (!p || !cfg || !out || !p->has_lik) return NS_EINVAL;
    NS_TRY(engine_kernel_attributes());
    *out = nullptr;
    const int n = cfg->n_live, k = cfg->n_delete, d = p->d;
    if (n < 2 || n > 4096 || k < 1 || k >= n || d < 1 || d > 64) return NS_EINVAL;
    if (!(cfg->width > 0) || cfg->step_cap < 1 || !(cfg->tol > 0)) return NS_EINVAL;
    const int G = cfg->n_shards > 1 ? cfg->n_shards : 1;
    if (G > k || cfg->shard < 0 || cfg->shard >= G || (G > 1 && cfg->chain_groups == 2)) return NS_EINVAL;
    ns_run* r = new (std::nothrow) ns_run();
    if (!r) return NS_ENOMEM;
    auto fail = [&](int s) { run_release(r); return s; };
    r->p = p;
    r->cfg = *cfg;
    r->n = n; r->k = k; r->d = d;
    r->R = cfg->repeats > 0 ? cfg->repeats : 5 * d;
    r->st = (cudaStream_t)stream;
    r->n_pad = 1;
    while (r->n_pad < n) r->n_pad <<= 1;
    int s;
    // rounds hold up to two proposals per chain (both stepping-out ends); the
    // initial live set is scored through the same workspace
    const int cap = std::max(n, 2 * k);
    if ((s = workspace_create(p, cap, &r->ws))) return fail(s);
    RunDev& rd = r->rd;
    rd.n = n; rd.k = k; rd.d = d; rd.R = r->R; rd.cap_steps = cfg->step_cap;
    rd.width = cfg->width; rd.tol = cfg->tol; rd.seed = cfg->seed;
    void* v;
#define RA(field, bytes) do { if ((s = run_alloc(r, (bytes), &v))) return fail(s); rd.field = (decltype(rd.field))v; } while (0)
    RA(live_x, sizeof(double) * n * d);
    RA(live_L, sizeof(double) * n);
    RA(order, sizeof(int) * r->n_pad);
    RA(deleted, sizeof(int) * k);
    RA(starts, sizeof(int) * k);
    RA(chol, sizeof(double) * d * d);
    RA(chol32, sizeof(float) * d * d);
    RA(cov, sizeof(double) * d * d);
    RA(mean, sizeof(double) * d);
    RA(dirs, sizeof(double) * (size_t)k * r->R * d);
    RA(ch_x, sizeof(double) * k * d);
    RA(ch_u, sizeof(double) * k * d);
    RA(ch_L, sizeof(double) * k);
    RA(ch_l, sizeof(double) * k);
    RA(ch_r, sizeof(double) * k);
    RA(ch_t, sizeof(double) * k);
    RA(ch_phase, sizeof(int) * k);
    RA(ch_move, sizeof(int) * k);
    RA(ch_step, sizeof(int) * k);
    RA(ch_step2, sizeof(int) * k);
    RA(ch_evals, sizeof(int) * k);
    RA(ch_row, sizeof(int) * k);
    RA(ch_row2, sizeof(int) * k);
    RA(prop, sizeof(double) * cap * d);
    RA(sc, sizeof(Scalars));
#undef RA
    rd.logL = r->ws.logL;
    k_reset_chains<<<(k + 127) / 128, 128, 0, r->st>>>(rd);
    rd.batch_ctr = &rd.sc->batch;
    rd.run_id = 0;
    // a shard evolves the contiguous chains [k s / G, k (s + 1) / G)
    rd.sh_c0 = (int)((long long)k * (G > 1 ? cfg->shard : 0) / G);
    rd.sh_c1 = (int)((long long)k * (G > 1 ? cfg->shard + 1 : 1) / G);
    r->n_shards = G;
    rd.chain0 = rd.sh_c0;
    rd.grp_chains = rd.sh_c1 - rd.sh_c0;
    rd.P = p->P;
    rd.pkind = p->d_pkind;
    rd.pa = p->d_pa;
    rd.pb = p->d_pb;
    rd.fof = p->d_free_of_full;
    rd.prior_f32 = p->precision != NS_PREC_FP64;
    rd.theta_full = r->ws.theta_full;
    r->sc = rd.sc;
    if (cudaMallocHost(&r->h_sc, sizeof(Scalars)) != cudaSuccess) return fail(NS_ENOMEM);
    std::memset(r->h_sc, 0, sizeof(Scalars));
    if (cudaMemsetAsync(rd.sc, 0, sizeof(Scalars), r->st) != cudaSuccess) return fail(NS_ECUDA);
    if ((s = grow_dead(r, 16LL * k + n))) return fail(s);
    // the workspace row count is the round's batch counter
    r->ws.d_nrows = &rd.sc->batch;
    // optionally two groups of chains whose rounds overlap on the GPU (the
    // shear likelihood's tensor-core and FP32 stages then run side by side);
    // one group is the default: on GB300 the 39-d shear rounds measured 109 us
    // with one group of 500 chains against 117 us with two of 250
    const int want = cfg->chain_groups;
    r->n_groups = (k >= 2 && want == 2) ? 2 : 1;
    if (r->n_groups > 1) {
        r->k0 = (k + 1) / 2;
        if ((s = workspace_create(p, 2 * (k - r->k0), &r->ws1))) return fail(s);
        if ((s = run_alloc(r, 2 * sizeof(int), &v))) return fail(s);
        r->grp1_ctr = (int*)v;
        if (cudaMemsetAsync(v, 0, 2 * sizeof(int), r->st) != cudaSuccess) return fail(NS_ECUDA);
    }
    // initial live points
    k_init_points<<<(n + 127) / 128, 128, 0, r->st>>>(n, d, cfg->seed, rd.prop);
    k_set_int<<<1, 1, 0, r->st>>>(&rd.sc->batch, n);
    if (cudaGetLastError() != cudaSuccess) return fail(NS_ECUDA);
    if ((s = launch_cube_to_theta(p, &r->ws, rd.prop, n, r->st))) return fail(s);
    if ((s = run_likelihood(p, &r->ws, n, r->ws.logL, nullptr, r->st))) return fail(s);
    k_init_finish<<<(n + 127) / 128, 128, 0, r->st>>>(rd, r->ws.logL);
    if (cudaGetLastError() != cudaSuccess) return fail(NS_ECUDA);
    if ((s = sync_scalars(r))) return fail(s);
    *out = r;
    return NS_OK;
}

// Rounds per captured graph launch: even, so that the alternating batch
// counters hand over from one launch to the next (launch_round).
static int rounds_per_sync(const ns_run* r) {
    const int R = r->cfg.rounds_per_sync > 0 ? r->cfg.rounds_per_sync : 16;
    return (R + 1) & ~1;
}

// First part of an iteration: deletion and evidence update, live covariance
// and its factor, directions and starts, then likelihood rounds until every
// chain of this run (or of its shard) has made its R slice moves.
static int iteration_evolve(ns_run* r) {
    RunDev& rd = r->rd;
    cudaStream_t st = r->st;
    NS_TRY(grow_dead(r, r->h_sc->n_dead + r->k));
    const size_t sm = (size_t)r->n_pad * (sizeof(double) + sizeof(int)) + sizeof(double) * r->k;
    k_sort_delete<<<1, 1024, sm, st>>>(rd, r->n_pad, r->k, 1);
    NS_CUDA_TRY(cudaGetLastError());
    k_live_mean<<<r->d, 256, 0, st>>>(rd);
    k_live_cov<<<r->d * (r->d + 1) / 2, 256, 0, st>>>(rd, r->cfg.ridge);
    k_cholesky<<<1, 128, 0, st>>>(rd);
    k_directions<<<(unsigned)(((long long)(rd.sh_c1 - rd.sh_c0) * r->R + 7) / 8), 256, 0, st>>>(rd);
    k_chains_start<<<(r->k + 127) / 128, 128, 0, st>>>(rd);
    NS_CUDA_TRY(cudaGetLastError());
    const int R = rounds_per_sync(r);
    if (!r->graph || r->graph_rounds != R) NS_TRY(build_graph(r, R));
    // a chain needs at most repeats * (2 step caps + shrink cap) evaluations
    const long long max_rounds = (long long)r->R * (3LL * r->cfg.step_cap + 2) + 8;
    for (long long done = 0;; done += R) {
        NS_CUDA_TRY(cudaGraphLaunch(r->graph, st));
        r->rounds += R;
        NS_TRY(sync_scalars(r));
        if (r->probe.stage != PROBE_NONE && *r->probe.h_rows > 0) {
            float ms = 0.f;
            NS_CUDA_TRY(cudaEventElapsedTime(&ms, r->probe.ev0, r->probe.ev1));
            r->prof_ms += ms;
            r->prof_launches += 1;
            r->prof_rows += *r->probe.h_rows;
        }
        if (r->h_sc->n_active == 0) break;
        if (done > max_rounds) { r->h_sc->status |= NS_BIT_TIMEOUT; return NS_ETIMEOUT; }
    }
    return NS_OK;
}

// Second part: every chain's final point replaces its deleted slot, the
// evaluation count and the termination test are updated.
static int iteration_insert(ns_run* r) {
    RunDev& rd = r->rd;
    cudaStream_t st = r->st;
    k_insert<<<1, 1024, 0, st>>>(rd);
    NS_CUDA_TRY(cudaGetLastError());
    NS_TRY(sync_scalars(r));
    r->last_valid = 1;
    return NS_OK;
}

static int one_iteration(ns_run* r) {
    NS_TRY(iteration_evolve(r));
    return iteration_insert(r);
}

static void fill_status(const ns_run* r, ns_status* st) {
    if (st) {
        st->iterations = r->h_sc->iter;
        st->evaluations = r->h_sc->evals;
        st->rounds = r->rounds;
        st->converged = r->h_sc->converged;
        st->status_bits = r->h_sc->status;
        st->logZ = r->h_sc->logZ;
        st->logX = r->h_sc->logX;
        st->lstar = r->h_sc->lstar;
        st->nonfinite = r->h_sc->nonfinite;
    }
}

extern "C" int ns_step(ns_run* r, int n_iters, ns_status* st) {
    if (!r || n_iters < 0) return NS_EINVAL;
    if (r->n_shards > 1 && n_iters > 0) return NS_EINVAL;   // sharded runs advance by ns_shard_*
    int s = NS_OK;
    for (int i = 0; i < n_iters; ++i) {
        if (r->h_sc->converged) break;
        if ((s = one_iteration(r)) != NS_OK) break;
    }
    fill_status(r, st);
    return s;
}

extern "C" int ns_shard_evolve(ns_run* r, ns_status* st) {
    if (!r || r->shard_pending) return NS_EINVAL;
    int s = NS_OK;
    if (!r->h_sc->converged) {
        s = iteration_evolve(r);
        if (s == NS_OK) r->shard_pending = 1;
    }
    fill_status(r, st);
    return s;
}

extern "C" int ns_shard_export(const ns_run* r, double* finals_dev) {
    if (!r || !finals_dev || !r->shard_pending) return NS_EINVAL;
    const int rows = r->rd.sh_c1 - r->rd.sh_c0;
    const int blocks = std::max(1, std::min(1024, (rows * (r->d + 2) + 255) / 256));
    k_shard_pack<<<blocks, 256, 0, r->st>>>(r->rd, finals_dev);
    NS_CUDA_TRY(cudaGetLastError());
    return NS_OK;
}

extern "C" int ns_shard_insert(ns_run* r, const double* all_finals_dev, ns_status* st) {
    if (!r || !all_finals_dev || !r->shard_pending) return NS_EINVAL;
    const int blocks = std::max(1, std::min(1024, (r->k * (r->d + 2) + 255) / 256));
    k_shard_unpack<<<blocks, 256, 0, r->st>>>(r->rd, all_finals_dev);
    NS_CUDA_TRY(cudaGetLastError());
    r->shard_pending = 0;
    const int s = iteration_insert(r);
    fill_status(r, st);
    return s;
}

extern "C" int ns_shard_range(const ns_run* r, int* chain_begin, int* chain_end) {
    if (!r) return NS_EINVAL;
    if (chain_begin) *chain_begin = r->rd.sh_c0;
    if (chain_end) *chain_end = r->rd.sh_c1;
    return NS_OK;
}

extern "C" int ns_evidence(const ns_run* rc, int n_replays, double* logZ, double* logZ_err, double* logX,
                           double* H, long long* n_dead) {
    if (!rc) return NS_EINVAL;
    ns_run* r = const_cast<ns_run*>(rc);
    if (n_replays <= 0) n_replays = 200;
    cudaStream_t st = r->st;
    NS_TRY(sync_scalars(r));
    const size_t sm = (size_t)r->n_pad * (sizeof(double) + sizeof(int));
    k_sort_delete<<<1, 1024, sm, st>>>(r->rd, r->n_pad, 0, 0);   // order of the live set only
    NS_CUDA_TRY(cudaGetLastError());
    double* dout;
    if (cudaMalloc(&dout, sizeof(double) * (3 + n_replays)) != cudaSuccess) return NS_ENOMEM;
    k_final_evidence<<<1, 1024, 2 * sizeof(double) * r->n, st>>>(r->rd, dout);
    k_err_replays<<<n_replays, 256, 128 * sizeof(double), st>>>(r->rd, r->h_sc->n_dead, dout + 3);
    std::vector<double> h(3 + n_replays);
    cudaError_t e = cudaGetLastError();
    if (e == cudaSuccess) e = cudaMemcpyAsync(h.data(), dout, sizeof(double) * h.size(), cudaMemcpyDeviceToHost, st);
    if (e == cudaSuccess) e = cudaStreamSynchronize(st);
    cudaFree(dout);
    if (e != cudaSuccess) { ns_set_last_cuda_error(e, "ns_evidence", __FILE__, __LINE__); return NS_ECUDA; }
    double mean = 0.0;
    for (int i = 0; i < n_replays; ++i) mean += h[3 + i];
    mean /= n_replays;
    double var = 0.0;
    for (int i = 0; i < n_replays; ++i) var += (h[3 + i] - mean) * (h[3 + i] - mean);
    var /= std::max(1, n_replays - 1);
    if (logZ) *logZ = h[0];
    if (logX) *logX = h[1];
    if (H) *H = h[2];
    if (logZ_err) *logZ_err = std::sqrt(var);
    if (n_dead) *n_dead = r->h_sc->n_dead + r->n;
    return NS_OK;
}

extern "C" int ns_live_points(const ns_run* r, double* x, double* logL) {
    if (!r) return NS_EINVAL;
    NS_CUDA_TRY(cudaStreamSynchronize(r->st));
    if (x) NS_CUDA_TRY(cudaMemcpy(x, r->rd.live_x, sizeof(double) * r->n * r->d, cudaMemcpyDeviceToHost));
    if (logL) NS_CUDA_TRY(cudaMemcpy(logL, r->rd.live_L, sizeof(double) * r->n, cudaMemcpyDeviceToHost));
    return NS_OK;
}

extern "C" int ns_dead_points(const ns_run* r, long long max_out, double* x, double* logL, int* nl,
                              long long* n_out) {
    if (!r || max_out < 0) return NS_EINVAL;
    NS_CUDA_TRY(cudaStreamSynchronize(r->st));
    const long long m = std::min(max_out, r->h_sc->n_dead);
    if (m > 0) {
        if (x) NS_CUDA_TRY(cudaMemcpy(x, r->rd.dead_x, sizeof(double) * m * r->d, cudaMemcpyDeviceToHost));
        if (logL) NS_CUDA_TRY(cudaMemcpy(logL, r->rd.dead_L, sizeof(double) * m, cudaMemcpyDeviceToHost));
        if (nl) NS_CUDA_TRY(cudaMemcpy(nl, r->rd.dead_n, sizeof(int) * m, cudaMemcpyDeviceToHost));
    }
    if (n_out) *n_out = m;
    return NS_OK;
}

extern "C" int ns_last_iteration(const ns_run* r, double* lstar, int* deleted, int* starts, int* evals) {
    if (!r || !r->last_valid) return NS_EINVAL;
    NS_CUDA_TRY(cudaStreamSynchronize(r->st));
    if (lstar) *lstar = r->h_sc->lstar;
    if (deleted) NS_CUDA_TRY(cudaMemcpy(deleted, r->rd.deleted, sizeof(int) * r->k, cudaMemcpyDeviceToHost));
    if (starts) NS_CUDA_TRY(cudaMemcpy(starts, r->rd.starts, sizeof(int) * r->k, cudaMemcpyDeviceToHost));
    if (evals) NS_CUDA_TRY(cudaMemcpy(evals, r->rd.ch_evals, sizeof(int) * r->k, cudaMemcpyDeviceToHost));
    return NS_OK;
}

extern "C" int ns_profile_stage(ns_run* r, int stage) {
    if (!r || stage < PROBE_NONE || stage > PROBE_WINDOWS) return NS_EINVAL;
    NS_CUDA_TRY(cudaStreamSynchronize(r->st));
    if (stage != PROBE_NONE && !r->probe.ev0) {
        NS_CUDA_TRY(cudaEventCreate(&r->probe.ev0));
        NS_CUDA_TRY(cudaEventCreate(&r->probe.ev1));
        if (cudaMallocHost(&r->probe.h_rows, sizeof(int)) != cudaSuccess) return NS_ENOMEM;
        *r->probe.h_rows = 0;
    }
    r->probe.stage = stage;
    r->prof_ms = 0.0;
    r->prof_launches = 0;
    r->prof_rows = 0;
    if (r->graph) { cudaGraphExecDestroy(r->graph); r->graph = nullptr; }
    return NS_OK;
}

extern "C" int ns_profile_read(const ns_run* r, double* total_ms, long long* launches, long long* rows) {
    if (!r) return NS_EINVAL;
    if (total_ms) *total_ms = r->prof_ms;
    if (launches) *launches = r->prof_launches;
    if (rows) *rows = r->prof_rows;
    return NS_OK;
}

extern "C" int ns_free(ns_run* r) {
    if (!r) return NS_EINVAL;
    cudaStreamSynchronize(r->st);
    run_release(r);
    return NS_OK;
}

// ======================================================================
// Packed runs (row A15): several independent runs of one model (same
// emulator, data and covariance), each with its own priors (so its own
// dimension), live-point count and deletion count.  Each run keeps its own
// state and iteration cycle; their chains' proposals share one batch per
// round, tagged with the run index, so one likelihood launch serves all.
// ======================================================================
namespace gpuns {

}  // namespace gpuns

struct ns_multi {
    int n_runs = 0;
    std::vector<ns_run*> runs;
    const ns_problem* model = nullptr;
    cudaStream_t st = nullptr;
    cudaStream_t cap_st = nullptr;
    Workspace ws;
    int total_chains = 0;
    RunDev* d_runs = nullptr;
    int* d_chain_off = nullptr;
    std::vector<void*> owned;
    cudaGraphExec_t graph = nullptr;
    int graph_rounds = 0;
    long long rounds = 0;
    std::vector<int> state;           // 0 idle (start next iteration), 1 running
};

static void multi_release(ns_multi* m) {
    if (!m) return;
    if (m->graph) cudaGraphExecDestroy(m->graph);
    if (m->cap_st) cudaStreamDestroy(m->cap_st);
    for (ns_run* r : m->runs) run_release(r);
    for (void* q : m->owned) cudaFree(q);
    workspace_free(&m->ws);
    delete m;
}

static int multi_refresh_runs(ns_multi* m) {
    // device copies of every run's state with the packed batch fields
    std::vector<RunDev> h(m->n_runs);
    for (int i = 0; i < m->n_runs; ++i) {
        h[i] = m->runs[i]->rd;
        h[i].batch_ctr = m->ws.d_nrows;
        h[i].theta_full = m->ws.theta_full;
        h[i].run_id = i;
        h[i].logL = m->ws.logL;
    }
    NS_CUDA_TRY(cudaMemcpyAsync(m->d_runs, h.data(), sizeof(RunDev) * m->n_runs, cudaMemcpyHostToDevice, m->st));
    NS_CUDA_TRY(cudaStreamSynchronize(m->st));
    return NS_OK;
}

static int multi_launch_round(ns_multi* m, cudaStream_t st) {
    NS_CUDA_TRY(cudaMemsetAsync(m->ws.d_nrows, 0, sizeof(int), st));
    k_slice_advance_multi<<<(m->total_chains + kSliceWarps - 1) / kSliceWarps, 32 * kSliceWarps, 0, st>>>(
        m->d_runs, m->d_chain_off, m->n_runs);
    NS_CUDA_TRY(cudaGetLastError());
    return run_likelihood(m->model, &m->ws, 2 * m->total_chains, m->ws.logL, nullptr, st);
}

static int multi_build_graph(ns_multi* m, int rounds) {
    if (m->graph) { cudaGraphExecDestroy(m->graph); m->graph = nullptr; }
    if (!m->cap_st) {
        int lo = 0, hi = 0;
        NS_CUDA_TRY(cudaDeviceGetStreamPriorityRange(&lo, &hi));
        NS_CUDA_TRY(cudaStreamCreateWithPriority(&m->cap_st, cudaStreamNonBlocking, hi));
    }
    cudaGraph_t g;
    NS_CUDA_TRY(cudaStreamBeginCapture(m->cap_st, cudaStreamCaptureModeThreadLocal));
    int s = NS_OK;
    for (int i = 0; i < rounds && s == NS_OK; ++i) s = multi_launch_round(m, m->cap_st);
    cudaError_t e = cudaStreamEndCapture(m->cap_st, &g);
    if (s != NS_OK) { if (e == cudaSuccess) cudaGraphDestroy(g); return s; }
    NS_CUDA_TRY(e);
    e = cudaGraphInstantiate(&m->graph, g, cudaGraphInstantiateFlagUseNodePriority);
    cudaGraphDestroy(g);
    NS_CUDA_TRY(e);
    m->graph_rounds = rounds;
    return NS_OK;
}

extern "C" int ns_multi_init(const ns_problem* const* problems, int n_runs, const ns_config* cfgs, void* stream,
                             ns_multi** out) {
    if (!problems || !cfgs || !out || n_runs < 1 || n_runs > 64) return NS_EINVAL;
    *out = nullptr;
    const ns_problem* p0 = problems[0];
    if (!p0) return NS_EINVAL;
    for (int i = 0; i < n_runs; ++i) {
        const ns_problem* p = problems[i];
        if (!p || p->kind != p0->kind || p->precision != p0->precision || p->P != p0->P || p->D != p0->D)
            return NS_EINVAL;
    }
    ns_multi* m = new (std::nothrow) ns_multi();
    if (!m) return NS_ENOMEM;
    auto fail = [&](int s) { multi_release(m); return s; };
    m->n_runs = n_runs;
    m->model = p0;
    m->st = (cudaStream_t)stream;
    std::vector<int> off(n_runs + 1, 0);
    for (int i = 0; i < n_runs; ++i) {
        ns_run* r = nullptr;
        ns_config ci = cfgs[i];
        ci.chain_groups = 1;      // packed runs share one batch instead
        ci.n_shards = 0;          // and are not split across devices
        ci.shard = 0;
        int s = ns_init(problems[i], &ci, stream, &r);
        if (s) return fail(s);
        m->runs.push_back(r);
        off[i + 1] = off[i] + r->k;
    }
    m->total_chains = off[n_runs];
    int s;
    // a round holds up to two proposals per chain (both stepping-out ends)
    if ((s = workspace_create(p0, 2 * m->total_chains, &m->ws))) return fail(s);
    void* v;
    auto alloc = [&](size_t bytes) -> void* {
        void* q = nullptr;
        if (cudaMalloc(&q, bytes) != cudaSuccess) return nullptr;
        m->owned.push_back(q);
        return q;
    };
    m->d_runs = (RunDev*)alloc(sizeof(RunDev) * n_runs);
    m->d_chain_off = (int*)alloc(sizeof(int) * (n_runs + 1));
    if (!m->d_runs || !m->d_chain_off) return fail(NS_ENOMEM);
    (void)v;
    if (cudaMemcpy(m->d_chain_off, off.data(), sizeof(int) * (n_runs + 1), cudaMemcpyHostToDevice) != cudaSuccess)
        return fail(NS_ECUDA);
    m->state.assign(n_runs, 0);
    if ((s = multi_refresh_runs(m))) return fail(s);
    *out = m;
    return NS_OK;
}

static int multi_start_iteration(ns_multi* m, int i) {
    ns_run* r = m->runs[i];
    NS_TRY(grow_dead(r, r->h_sc->n_dead + r->k));
    const size_t sm = (size_t)r->n_pad * (sizeof(double) + sizeof(int)) + sizeof(double) * r->k;
    k_sort_delete<<<1, 1024, sm, m->st>>>(r->rd, r->n_pad, r->k, 1);
    k_live_mean<<<r->d, 256, 0, m->st>>>(r->rd);
    k_live_cov<<<r->d * (r->d + 1) / 2, 256, 0, m->st>>>(r->rd, r->cfg.ridge);
    k_cholesky<<<1, 128, 0, m->st>>>(r->rd);
    k_directions<<<(unsigned)(((long long)(r->rd.sh_c1 - r->rd.sh_c0) * r->R + 7) / 8), 256, 0, m->st>>>(r->rd);
    k_chains_start<<<(r->k + 127) / 128, 128, 0, m->st>>>(r->rd);
    NS_CUDA_TRY(cudaGetLastError());
    return NS_OK;
}

extern "C" int ns_multi_step(ns_multi* m, int n_iters, ns_status* st) {
    if (!m || n_iters < 0) return NS_EINVAL;
    const int nr = m->n_runs;
    std::vector<int> todo(nr);
    for (int i = 0; i < nr; ++i) {
        NS_CUDA_TRY(cudaMemcpyAsync(m->runs[i]->h_sc, m->runs[i]->sc, sizeof(Scalars), cudaMemcpyDeviceToHost, m->st));
    }
    NS_CUDA_TRY(cudaStreamSynchronize(m->st));
    for (int i = 0; i < nr; ++i) todo[i] = m->runs[i]->h_sc->converged ? 0 : n_iters;
    const int R = 16;
    if (!m->graph || m->graph_rounds != R) NS_TRY(multi_build_graph(m, R));
    long long guard = 0;
    long long max_rounds = 0;
    for (ns_run* r : m->runs) max_rounds = std::max(max_rounds, (long long)r->R * (3LL * r->cfg.step_cap + 2) + 8);
    for (;;) {
        bool started = false;
        for (int i = 0; i < nr; ++i)
            if (m->state[i] == 0 && todo[i] > 0) {
                const long long cap_before = m->runs[i]->dead_cap;
                NS_TRY(multi_start_iteration(m, i));
                m->state[i] = 1;
                started = true;
                (void)cap_before;
            }
        if (started) { NS_TRY(multi_refresh_runs(m)); guard = 0; }
        bool any = false;
        for (int i = 0; i < nr; ++i) any = any || (m->state[i] == 1);
        if (!any) break;
        NS_CUDA_TRY(cudaGraphLaunch(m->graph, m->st));
        m->rounds += R;
        guard += R;
        for (int i = 0; i < nr; ++i)
            if (m->state[i] == 1)
                NS_CUDA_TRY(cudaMemcpyAsync(m->runs[i]->h_sc, m->runs[i]->sc, sizeof(Scalars), cudaMemcpyDeviceToHost,
                                            m->st));
        NS_TRY(workspace_err_fetch(&m->ws, m->st));
        NS_CUDA_TRY(cudaStreamSynchronize(m->st));
        if (const int bits = workspace_err_bits(&m->ws)) {
            for (ns_run* r : m->runs) r->h_sc->status |= bits;
            return NS_ETIMEOUT;
        }
        bool finished = false;
        for (int i = 0; i < nr; ++i)
            if (m->state[i] == 1 && m->runs[i]->h_sc->n_active == 0) {
                k_insert<<<1, 1024, 0, m->st>>>(m->runs[i]->rd);
                NS_CUDA_TRY(cudaGetLastError());
                m->state[i] = 2;
                finished = true;
            }
        if (finished) {
            for (int i = 0; i < nr; ++i)
                if (m->state[i] == 2)
                    NS_CUDA_TRY(cudaMemcpyAsync(m->runs[i]->h_sc, m->runs[i]->sc, sizeof(Scalars),
                                                cudaMemcpyDeviceToHost, m->st));
            NS_CUDA_TRY(cudaStreamSynchronize(m->st));
            for (int i = 0; i < nr; ++i)
                if (m->state[i] == 2) {
                    m->state[i] = 0;
                    m->runs[i]->last_valid = 1;
                    todo[i] = m->runs[i]->h_sc->converged ? 0 : todo[i] - 1;
                }
        }
        if (guard > max_rounds) return NS_ETIMEOUT;
    }
    if (st)
        for (int i = 0; i < nr; ++i) {
            const Scalars* h = m->runs[i]->h_sc;
            st[i].iterations = h->iter;
            st[i].evaluations = h->evals;
            st[i].rounds = m->rounds;
            st[i].converged = h->converged;
            st[i].status_bits = h->status;
            st[i].logZ = h->logZ;
            st[i].logX = h->logX;
            st[i].lstar = h->lstar;
            st[i].nonfinite = h->nonfinite;
        }
    return NS_OK;
}

extern "C" int ns_multi_run(const ns_multi* m, int i, ns_run** out) {
    if (!m || !out || i < 0 || i >= m->n_runs) return NS_EINVAL;
    *out = m->runs[i];
    return NS_OK;
}

extern "C" int ns_multi_free(ns_multi* m) {
    if (!m) return NS_EINVAL;
    cudaStreamSynchronize(m->st);
    multi_release(m);
    return NS_OK;
}
