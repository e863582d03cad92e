// Evidence of a caller-held dead-point sequence without any device allocation.
//
// ns_evidence() allocates a small device buffer for the per-replay log Z values
// of its simulated-shrinkage error estimate.  Some callers cannot allocate
// device memory when they need the number: a host framework that reserves the
// device memory up front for its own caching pool (a library cudaMalloc then
// fails or fragments that pool, and the framework forbids it), or a control
// loop that must not call cudaMalloc / cudaFree because they can synchronise
// the device and stall its other streams.  ns_evidence_noalloc() serves them:
// the caller passes the sequence and an output buffer, and the per-replay values
// go to the file-scope array g_replay_scratch below, which every GPU that loads
// this library holds (kMaxNoallocReplays doubles) until the process exits.
#include <mutex>

#include "evidence_seq.cuh"
#include "likelihood.cuh"

namespace gpuns {

constexpr int kMaxNoallocReplays = 4096;   // 32 KiB of device memory per GPU

// Shared by every call on a device; each call overwrites the slots it uses.
static __device__ __align__(256) double g_replay_scratch[kMaxNoallocReplays];

// One block per replay s: ln t_i = ln(U_{s,i}) / n_i, U from Philox (ERR, s, i, 0).
__global__ void __launch_bounds__(256)
k_noalloc_replays(const double* __restrict__ logL, const int* __restrict__ nlive, long long N,
                  unsigned long long seed, double* __restrict__ scratch) {
    __shared__ double red[80];
    const int s = blockIdx.x;
    auto Lof = [&](long long i) -> double { return logL[i]; };
    auto lnt = [&](long long i) -> double {
        const Draw2 u = philox_uniforms(seed, P_ERR, 0, (uint32_t)s, (uint32_t)i, 0);
        return log(u.a) / nlive[i];
    };
    const double lz = sequence_logZ(Lof, N, lnt, red, nullptr);
    if (threadIdx.x == 0) scratch[s] = lz;
}

// out[0] = ln Z with the expected shrinkage ln t_i = -1/n_i, out[1] = standard
// deviation (ddof 1) of the replays in scratch, out[2] = final ln X.  A live
// count below 1 anywhere in the sequence makes all three outputs NaN.
__global__ void __launch_bounds__(256)
k_noalloc_finish(const double* __restrict__ logL, const int* __restrict__ nlive, long long N, int n_replays,
                 const double* __restrict__ scratch, double* __restrict__ out) {
    __shared__ double red[80];
    __shared__ double logX;
    int bad = 0;
    for (long long i = threadIdx.x; i < N; i += blockDim.x) bad |= (nlive[i] < 1);
    if (__syncthreads_or(bad)) {
        if (threadIdx.x < 3) out[threadIdx.x] = __longlong_as_double(0x7ff8000000000000ll);
        return;
    }
    auto Lof = [&](long long i) -> double { return logL[i]; };
    auto lnt = [&](long long i) -> double { return -1.0 / nlive[i]; };
    const double lz = sequence_logZ(Lof, N, lnt, red, &logX);
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
// with that device current (the host-side symbol is only a stand-in).  The
// cached address belongs to the device's primary context: it is not refreshed
// after a cudaDeviceReset, which this entry point does not support.
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
