// Shared device/host helpers of the gpuns library (sm_103a).
#pragma once

#include <cuda_runtime.h>
#include <cuda_bf16.h>
#include <stdint.h>
#include <utility>
#include <math.h>

#include "../../include/gpuns.h"

#define NS_CUDA_TRY(expr)                                                    \
    do {                                                                     \
        cudaError_t _e = (expr);                                             \
        if (_e != cudaSuccess) { ns_set_last_cuda_error(_e, #expr, __FILE__, __LINE__); return NS_ECUDA; } \
    } while (0)

#define NS_TRY(...)                                                          \
    do { int _s = (__VA_ARGS__); if (_s != NS_OK) return _s; } while (0)

void ns_set_last_cuda_error(cudaError_t e, const char* what, const char* file, int line);

namespace gpuns {

constexpr double kCkms = 299792.458;          // speed of light [km/s]
constexpr double kCover100 = kCkms / 100.0;   // c / (100 km/s/Mpc) [Mpc]
constexpr double kLn10 = 2.302585092994045684;

// --------------------------------------------------------------------------
// Philox4x32-10 (Salmon et al. 2011, SC'11): ten rounds of two 32x32->64
// multiplies with fixed multipliers, XOR with the other words and the round
// key, then a word permutation; the key advances by two Weyl increments
// between rounds.
// --------------------------------------------------------------------------
struct U4 { uint32_t x, y, z, w; };

__host__ __device__ inline U4 philox4x32_10(U4 c, uint32_t k0, uint32_t k1) {
    const uint32_t M0 = 0xD2511F53u, M1 = 0xCD9E8D57u;
    const uint32_t W0 = 0x9E3779B9u, W1 = 0xBB67AE85u;
#pragma unroll
    for (int r = 0; r < 10; ++r) {
        if (r > 0) { k0 += W0; k1 += W1; }
        uint64_t p0 = (uint64_t)M0 * c.x;
        uint64_t p1 = (uint64_t)M1 * c.z;
        uint32_t hi0 = (uint32_t)(p0 >> 32), lo0 = (uint32_t)p0;
        uint32_t hi1 = (uint32_t)(p1 >> 32), lo1 = (uint32_t)p1;
        U4 n;
        n.x = hi1 ^ c.y ^ k0;
        n.y = lo1;
        n.z = hi0 ^ c.w ^ k1;
        n.w = lo0;
        c = n;
    }
    return c;
}

enum Purpose : uint32_t { P_INIT = 1, P_START = 2, P_DIR = 3, P_STEPOUT = 4, P_SHRINK = 5, P_ERR = 6 };

// 52 random bits -> (2m + 1) 2^-53: exact, strictly inside (0, 1).
__host__ __device__ inline double u01_from(uint32_t hi, uint32_t lo) {
    uint64_t m = ((((uint64_t)hi) << 32) | lo) >> 12;
    return (2.0 * (double)m + 1.0) * 1.1102230246251565404e-16;  // 2^-53
}

struct Draw2 { double a, b; };

__host__ __device__ inline Draw2 philox_uniforms(unsigned long long seed, uint32_t purpose, uint32_t j,
                                                 uint32_t w1, uint32_t w2, uint32_t w3) {
    U4 c{purpose | (j << 8), w1, w2, w3};
    U4 o = philox4x32_10(c, (uint32_t)(seed & 0xffffffffull), (uint32_t)(seed >> 32));
    return Draw2{u01_from(o.x, o.y), u01_from(o.z, o.w)};
}

// --------------------------------------------------------------------------
// Phi^-1(c) of a Gaussian prior (Table 1).  With f32 (reduced-precision
// problems) the quantile is taken in FP32 on the smaller tail probability
// q = min(c, 1 - c) (1 - c is exact in FP64 for c >= 1/2) and mirrored, so a
// coordinate within 2^-25 of 1 does not round to 1.0f, where the FP32
// quantile is +inf; tails below 1e-37 (under FLT_MIN) use the FP64 quantile.
// --------------------------------------------------------------------------
__device__ __forceinline__ double gauss_quantile(double c, bool f32) {
    if (!f32) return normcdfinv(c);
    const double q = (c < 0.5) ? c : 1.0 - c;
    if (q < 1e-37) return normcdfinv(c);
    const double z = (double)normcdfinvf((float)q);
    return (c < 0.5) ? z : -z;
}

// --------------------------------------------------------------------------
// Catmull-Rom weights for taps (-1, 0, 1, 2) at fraction t.
// --------------------------------------------------------------------------
template <typename T>
__host__ __device__ inline void catmull_rom(T t, T w[4]) {
    T t2 = t * t, t3 = t2 * t;
    w[0] = T(0.5) * (-t + T(2) * t2 - t3);
    w[1] = T(0.5) * (T(2) - T(5) * t2 + T(3) * t3);
    w[2] = T(0.5) * (t + T(4) * t2 - T(3) * t3);
    w[3] = T(0.5) * (-t2 + t3);
}

// Fold the ghost taps of a cell [i, i+1] of an n-point axis into real nodes:
// ghost -1 = 2 p0 - p1 and ghost n = 2 p[n-1] - p[n-2] (linear extrapolation).
// Out: four node indices (may repeat, with zero weight) and weights.
template <typename T>
__host__ __device__ inline void fold_taps(int i, int n, const T w_in[4], int idx[4], T w[4]) {
    idx[0] = i - 1; idx[1] = i; idx[2] = i + 1; idx[3] = i + 2;
    w[0] = w_in[0]; w[1] = w_in[1]; w[2] = w_in[2]; w[3] = w_in[3];
    if (i == 0) {            // tap -1 is a ghost
        w[1] += T(2) * w[0];
        w[2] -= w[0];
        w[0] = T(0); idx[0] = 0;
    }
    if (i + 2 >= n) {        // tap n is a ghost (i = n - 2)
        w[2] += T(2) * w[3];
        w[1] -= w[3];
        w[3] = T(0); idx[3] = n - 1;
    }
}

// --------------------------------------------------------------------------
// Warp / block reductions.
// --------------------------------------------------------------------------
template <typename T>
__device__ inline T warp_sum(T v) {
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
    return v;
}

template <typename T>
__device__ inline T warp_max(T v) {
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v = fmax(v, __shfl_xor_sync(0xffffffffu, v, o));
    return v;
}

// Sum over the block; every thread gets the result.  red: >= 32 T of smem.
template <typename T>
__device__ inline T block_sum(T v, T* red) {
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5, nw = (blockDim.x + 31) >> 5;
    v = warp_sum(v);
    __syncthreads();
    if (lane == 0) red[wid] = v;
    __syncthreads();
    T s = (threadIdx.x < nw) ? red[threadIdx.x] : T(0);
    if (wid == 0) s = warp_sum(s);
    if (threadIdx.x == 0) red[0] = s;
    __syncthreads();
    T r = red[0];
    __syncthreads();
    return r;
}

// In-place exclusive prefix sum of x[0..n) in shared memory (any block size).
// red: >= 33 T of smem.  Each thread scans a contiguous chunk sequentially.
template <typename T>
__device__ inline void block_exclusive_scan(T* x, int n, T* red) {
    const int nt = blockDim.x, tid = threadIdx.x;
    const int chunk = (n + nt - 1) / nt;
    const int lo = min(n, tid * chunk), hi = min(n, lo + chunk);
    T s = T(0);
    for (int i = lo; i < hi; ++i) s += x[i];
    // exclusive scan of the per-thread totals across the block
    const int lane = tid & 31, wid = tid >> 5, nw = (nt + 31) >> 5;
    T inc = s;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
        T y = __shfl_up_sync(0xffffffffu, inc, o);
        if (lane >= o) inc += y;
    }
    __syncthreads();
    if (lane == 31) red[wid] = inc;
    __syncthreads();
    if (wid == 0) {
        T v = (lane < nw) ? red[lane] : T(0);
        T vi = v;
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
            T y = __shfl_up_sync(0xffffffffu, vi, o);
            if (lane >= o) vi += y;
        }
        if (lane < nw) red[lane] = vi - v;   // exclusive warp offsets
    }
    __syncthreads();
    T run = red[wid] + inc - s;
    for (int i = lo; i < hi; ++i) { T v = x[i]; x[i] = run; run += v; }
    __syncthreads();
}

// In-place exclusive suffix sum: x[i] <- sum_{j > i} x[j].
template <typename T>
__device__ inline void block_exclusive_suffix_scan(T* x, int n, T* red) {
    const int nt = blockDim.x, tid = threadIdx.x;
    const int chunk = (n + nt - 1) / nt;
    // thread tid owns the reversed chunk: indices n-1-lo .. n-hi
    const int lo = min(n, tid * chunk), hi = min(n, lo + chunk);
    T s = T(0);
    for (int i = lo; i < hi; ++i) s += x[n - 1 - i];
    const int lane = tid & 31, wid = tid >> 5, nw = (nt + 31) >> 5;
    T inc = s;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
        T y = __shfl_up_sync(0xffffffffu, inc, o);
        if (lane >= o) inc += y;
    }
    __syncthreads();
    if (lane == 31) red[wid] = inc;
    __syncthreads();
    if (wid == 0) {
        T v = (lane < nw) ? red[lane] : T(0);
        T vi = v;
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
            T y = __shfl_up_sync(0xffffffffu, vi, o);
            if (lane >= o) vi += y;
        }
        if (lane < nw) red[lane] = vi - v;
    }
    __syncthreads();
    T run = red[wid] + inc - s;
    for (int i = lo; i < hi; ++i) { T v = x[n - 1 - i]; x[n - 1 - i] = run; run += v; }
    __syncthreads();
}

template <typename T> __device__ inline T dexp(T x);
template <> __device__ inline double dexp<double>(double x) { return exp(x); }
template <> __device__ inline float dexp<float>(float x) { return expf(x); }
template <typename T> __device__ inline T dlog(T x);
template <> __device__ inline double dlog<double>(double x) { return log(x); }
template <> __device__ inline float dlog<float>(float x) { return logf(x); }

__global__ void k_set_int(int* p, int v);

// Programmatic dependent launch.  A kernel of the round chain first lets the
// next grid in its stream begin launching (its CTAs then fill SMs as this
// grid's CTAs retire) and then waits until its own predecessor has completed
// and its memory is visible.  Nothing is read or written before the wait, so
// the overlap covers launch latency and tails only.  Both are no-ops for a
// grid launched without the attribute.
__device__ __forceinline__ void pdl_begin() {
    asm volatile("griddepcontrol.launch_dependents;" ::: "memory");
    asm volatile("griddepcontrol.wait;" ::: "memory");
}

// Launch with the programmatic-stream-serialization attribute (see pdl_begin).
template <typename... KArgs, typename... Args>
inline cudaError_t launch_pdl(void (*kernel)(KArgs...), dim3 grid, dim3 block, size_t smem, cudaStream_t st,
                              Args&&... args) {
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = grid;
    cfg.blockDim = block;
    cfg.dynamicSmemBytes = smem;
    cfg.stream = st;
    cudaLaunchAttribute attr[1];
    attr[0].id = cudaLaunchAttributeProgrammaticStreamSerialization;
    attr[0].val.programmaticStreamSerializationAllowed = 1;
    cfg.attrs = attr;
    cfg.numAttrs = 1;
    return cudaLaunchKernelEx(&cfg, kernel, std::forward<Args>(args)...);
}

}  // namespace gpuns
