// Block-wide evidence of a dead-point sequence under a given shrinkage sequence
// (Eq. 1 as the sum of L_i w_i with prior-volume weights
// w_i = X_{i-1} - X_i = X_{i-1} (1 - t_i), ln X_i = sum_{j <= i} ln t_j).
// Shared by the run's simulated-shrinkage error (ns_engine.cu) and the
// allocation-free evidence entry point (noalloc.cu), so both give the same
// replays for the same sequence and Philox key.
#pragma once

#include "common.cuh"

namespace gpuns {

// ln Z = LSE_i(ln L_i + ln X_{i-1} + ln(1 - t_i)) over i < N, with ln L_i = Lof(i)
// and ln t_i = lnt(i) (< 0).  Threads own contiguous chunks of the sequence; the
// running ln X of each chunk comes from a block scan of the chunk totals.  Called
// by every thread of a block of a multiple of 32 threads (<= 256); red: >= 48
// doubles of shared memory.  The result is valid in every thread; *logX_out
// (if given) receives the final ln X (written by thread 0).
template <typename LFn, typename LnT>
__device__ double sequence_logZ(LFn Lof, long long N, LnT lnt, double* red, double* logX_out) {
    const int tid = threadIdx.x, nt = blockDim.x;
    const long long chunk = (N + nt - 1) / nt;
    const long long lo = min(N, (long long)tid * chunk), hi = min(N, lo + chunk);
    double tot = 0.0;
    for (long long i = lo; i < hi; ++i) tot += lnt(i);
    const int lane = tid & 31, wid = tid >> 5, nw = nt >> 5;
    double inc = tot;
    for (int o = 1; o < 32; o <<= 1) { const double y = __shfl_up_sync(0xffffffffu, inc, o); if (lane >= o) inc += y; }
    __syncthreads();
    if (lane == 31) red[wid] = inc;
    __syncthreads();
    if (wid == 0) {
        const double v = (lane < nw) ? red[lane] : 0.0;
        double vi = v;
        for (int o = 1; o < 32; o <<= 1) { const double y = __shfl_up_sync(0xffffffffu, vi, o); if (lane >= o) vi += y; }
        if (lane < nw) red[lane] = vi - v;     // exclusive warp offsets
        if (lane == nw - 1) red[32] = vi;      // total ln X
    }
    __syncthreads();
    double logX = red[wid] + inc - tot;        // ln X before this thread's first point
    if (logX_out && tid == 0) *logX_out = red[32];
    __syncthreads();
    double mx = -INFINITY, acc = 0.0;          // running log-sum-exp (max, scaled sum)
    for (long long i = lo; i < hi; ++i) {
        const double lt = lnt(i);
        const double term = Lof(i) + logX + log(-expm1(lt));
        if (term > mx) { acc = (mx == -INFINITY ? 0.0 : acc * exp(mx - term)) + 1.0; mx = term; }
        else if (term > -INFINITY) acc += exp(term - mx);
        logX += lt;
    }
    double gmx = warp_max(mx);
    if (lane == 0) red[34 + wid] = gmx;
    __syncthreads();
    if (wid == 0) {
        double v = (lane < nw) ? red[34 + lane] : -INFINITY;
        v = warp_max(v);
        if (lane == 0) red[33] = v;
    }
    __syncthreads();
    gmx = red[33];
    __syncthreads();
    double part = (mx > -INFINITY && gmx > -INFINITY) ? acc * exp(mx - gmx) : 0.0;
    part = block_sum(part, red);
    return (gmx > -INFINITY) ? gmx + log(part) : -INFINITY;
}

}  // namespace gpuns
