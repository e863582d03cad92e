// Evidence of a caller-held dead-point sequence without any device allocation.
//
// ns_evidence() allocates a small device buffer for the per-replay log Z values
// of its simulated-shrinkage error estimate.  Some callers cannot allocate
// device memory at the time they need the number: code that records its work
// into a CUDA graph under a strict capture mode (where cudaMalloc is an error),
// or a host framework that owns all device memory through its own pool and
// forbids allocations by libraries it calls.  ns_evidence_noalloc() serves
// them: the caller passes the sequence and an output buffer, and the per-replay
// values go to the file-scope array g_replay_scratch below, which every GPU that
// loads this library holds (kMaxNoallocReplays doubles) until the process exits.
#include <mutex>

#include "likelihood.cuh"

namespace gpuns {

constexpr int kMaxNoallocReplays = 4096;   // 32 KiB of device memory per GPU

// Shared by every call on a device; each call overwrites the slots it uses.
static __device__ __align__(256) double g_replay_scratch[kMaxNoallocReplays];

__device__ inline double nl_lse2(double a, double b) {
    if (a == -INFINITY) return b;
    if (b == -INFINITY) return a;
    const double m = fmax(a, b);
    return m + log(exp(a - m) + exp(b - m));
}

// Block-wide log-sum-exp of sum_i exp(logL_i + ln X_{i-1} + ln(1 - t_i)) with
// ln t_i = lnt(i); threads own contiguous chunks, offsets by a block scan.
template <typename LnT>
__device__ double sequence_logZ(const double* __restrict__ logL, long long N, LnT lnt, double* red,
                                double* logX_out) {
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
        if (lane < nw) red[lane] = vi - v;
        if (lane == nw - 1) red[32] = vi;      // total ln X
    }
    __syncthreads();
    double logX = red[wid] + inc - tot;
    if (logX_out && tid == 0) *logX_out = red[32];
    __syncthreads();
    double mx = -INFINITY, acc = 0.0;
    for (long long i = lo; i < hi; ++i) {
        const double lt = lnt(i);
        const double term = logL[i] + logX + log(-expm1(lt));
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

// One block per replay s: ln t_i = ln(U_{s,i}) / n_i, U from Philox (ERR, s, i, 0).
__global__ void __launch_bounds__(256)
k_noalloc_replays(const double* __restrict__ logL, const int* __restrict__ nlive, long long N,
                  unsigned long long seed, double* __restrict__ scratch) {
    __shared__ double red[80];
    const int s = blockIdx.x;
    auto lnt = [&](long long i) -> double {
        const Draw2 u = philox_uniforms(seed, P_ERR, 0, (uint32_t)s, (uint32_t)i, 0);
        return log(u.a) / nlive[i];
    };
    const double lz = sequence_logZ(logL, N, lnt, red, nullptr);
    if (threadIdx.x == 0) scratch[s] = lz;
}

// out[0] = ln Z with the expected shrinkage ln t_i = -1/n_i, out[1] = standard
// deviation (ddof 1) of the replays in scratch, out[2] = final ln X.
__global__ void __launch_bounds__(256)
k_noalloc_finish(const double* __restrict__ logL, const int* __restrict__ nlive, long long N, int n_replays,
                 const double* __restrict__ scratch, double* __restrict__ out) {
    __shared__ double red[80];
    __shared__ double logX;
    auto lnt = [&](long long i) -> double { return -1.0 / nlive[i]; };
    const double lz = sequence_logZ(logL, N, lnt, red, &logX);
    double m = 0.0;
    for (int s = threadIdx.x; s < n_replays; s += blockDim.x) m += scratch[s];
    m = block_sum(m, red) / n_replays;
    double v = 0.0;
    for (int s = threadIdx.x; s < n_replays; s += blockDim.x) v += (scratch[s] - m) * (scratch[s] - m);
    v = block_sum(v, red) / max(1, n_replays - 1);
    if (threadIdx.x == 0) {
        out[0] = lz;
        out[1] = sqrt(v);
        out[2] = logX;
    }
}

}  // namespace gpuns

using namespace gpuns;

// Device address of g_replay_scratch for each device, looked up once per device
// with that device current (the host-side symbol is only a stand-in).
static double* g_scratch_addr[64] = {nullptr};
static std::mutex g_scratch_mu;

static int scratch_for_current_device(double** out) {
    int dev = 0;
    NS_CUDA_TRY(cudaGetDevice(&dev));
    if (dev < 0 || dev >= 64) return NS_ENOTSUP;
    std::lock_guard<std::mutex> lk(g_scratch_mu);
    if (!g_scratch_addr[dev]) {
        void* p = nullptr;
        NS_CUDA_TRY(cudaGetSymbolAddress(&p, g_replay_scratch));
        g_scratch_addr[dev] = static_cast<double*>(p);
    }
    *out = g_scratch_addr[dev];
    return NS_OK;
}

extern "C" int ns_evidence_noalloc(const double* logL_dev, const int* nlive_dev, long long n,
                                   unsigned long long seed, int n_replays, double* out_dev, void* stream) {
    if (!logL_dev || !nlive_dev || !out_dev || n < 1) return NS_EINVAL;
    if (n_replays <= 0) n_replays = 200;
    if (n_replays < 2 || n_replays > kMaxNoallocReplays) return NS_EINVAL;
    double* scratch = nullptr;
    NS_TRY(scratch_for_current_device(&scratch));
    cudaStream_t st = (cudaStream_t)stream;
    k_noalloc_replays<<<n_replays, 256, 0, st>>>(logL_dev, nlive_dev, n, seed, scratch);
    k_noalloc_finish<<<1, 256, 0, st>>>(logL_dev, nlive_dev, n, n_replays, scratch, out_dev);
    NS_CUDA_TRY(cudaGetLastError());
    return NS_OK;
}
