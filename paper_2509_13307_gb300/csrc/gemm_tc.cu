// BF16 x BF16 -> FP32 GEMM on the 5th-generation tensor cores (tcgen05) with
// TMA-fed shared-memory staging, used for the emulator's hidden and output
// layers (the dense contractions of the likelihood, Sec. 2.5 / App. A).
//
//   C[M x N] = epi(A[M x K] W[N x K]^T + bias)
//   A: activations, row-major (K-major), bf16;  W: weights [N][K], bf16.
//   epi 0: tanh, stored bf16 (next layer's A);  epi 1: mu + sigma * v, FP32.
//
// One CTA computes a 128 x BN tile.  A ring of STAGES slots guarded by
// full/empty mbarriers holds KPS k-blocks of 64 per slot; warp 0 (one lane)
// loads a slot's A box (128 x 64 x KPS bf16, 128-byte swizzle) and B box
// (BN x 64 x KPS); warp 1 (one lane) issues
// tcgen05.mma.cta_group::1.kind::f16 (M = 128, N = BN, K = 16) into a TMEM
// accumulator and releases ring slots with tcgen05.commit; warp 2 owns the
// TMEM allocation.  All four warps then drain TMEM with tcgen05.ld (warp w
// reads lanes 32w..32w+31 = tile rows), apply the epilogue and store.
// A thread's bulk copies complete one after another (a few hundred cycles
// each on GB300, almost independent of their size), so the operand rate of a
// CTA is set by its copy instructions per byte: with K a multiple of 128 a
// slot holds two k-blocks, each operand's pair loaded by one copy through a
// 3-D view of the row-major matrix ([K/64][rows][64], see
// make_tensor_map_bf16), in two slots (the shared memory of four one-block
// slots, so the CTA still fits beside the concurrent windows stage).
// Every wait is bounded: on timeout the CTA records an error and leaves.
#include <cudaTypedefs.h>

#include "likelihood.cuh"
#include "async_copy.cuh"

namespace gpuns {

namespace tc {

constexpr int BM = 128;
constexpr int BK = 64;                 // 64 bf16 = 128 bytes = one swizzle row

__device__ __forceinline__ void tma_load_2d(uint32_t dst, const CUtensorMap* tm, uint32_t bar, int x, int y) {
    asm volatile(
        "cp.async.bulk.tensor.2d.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1, {%3, %4}], [%2];"
        :: "r"(dst), "l"(reinterpret_cast<uint64_t>(tm)), "r"(bar), "r"(x), "r"(y) : "memory");
}

__device__ __forceinline__ void tma_load_3d(uint32_t dst, const CUtensorMap* tm, uint32_t bar, int x, int y, int z) {
    asm volatile(
        "cp.async.bulk.tensor.3d.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1, {%3, %4, %5}], [%2];"
        :: "r"(dst), "l"(reinterpret_cast<uint64_t>(tm)), "r"(bar), "r"(x), "r"(y), "r"(z) : "memory");
}

// k-blocks [KPS it, KPS (it + 1)) of the box rows starting at r0: a 2-D map
// (x = k offset) for KPS = 1, the 3-D view (z = k-block) otherwise.
template <int KPS>
__device__ __forceinline__ void tma_load_kb(uint32_t dst, const CUtensorMap* tm, uint32_t bar, int it, int r0) {
    if constexpr (KPS == 1) tma_load_2d(dst, tm, bar, it * BK, r0);
    else tma_load_3d(dst, tm, bar, 0, r0, it * KPS);
}

// Shared-memory matrix descriptor: K-major operand, 128-byte swizzle,
// 8-row groups 1024 bytes apart (stride byte offset), descriptor version 1.
__device__ __forceinline__ uint64_t smem_desc(uint32_t addr) {
    uint64_t d = 0;
    d |= (uint64_t)((addr & 0x3FFFF) >> 4);          // start address
    d |= (uint64_t)1 << 16;                          // leading byte offset (unused for swizzled K-major)
    d |= (uint64_t)(1024 >> 4) << 32;                // stride byte offset
    d |= (uint64_t)1 << 46;                          // version
    d |= (uint64_t)2 << 61;                          // 128-byte swizzle
    return d;
}

// Instruction descriptor, kind::f16: D = F32, A = B = BF16, both K-major.
template <int BN>
__host__ __device__ constexpr uint32_t instr_desc() {
    return (1u << 4) | (1u << 7) | (1u << 10) | ((uint32_t)(BN >> 3) << 17) | ((uint32_t)(BM >> 4) << 24);
}

__device__ __forceinline__ void mma_bf16(uint32_t tmem_d, uint64_t a, uint64_t b, uint32_t idesc, uint32_t acc) {
    asm volatile(
        "{\n\t.reg .pred p;\n\t"
        "setp.ne.b32 p, %4, 0;\n\t"
        "tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n\t}"
        :: "r"(tmem_d), "l"(a), "l"(b), "r"(idesc), "r"(acc));
}

__device__ __forceinline__ void mma_commit(uint32_t bar) {
    asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" :: "r"(bar) : "memory");
}

__device__ __forceinline__ void fence_before() { asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory"); }
__device__ __forceinline__ uint32_t cluster_ctarank() {
    uint32_t r;
    asm volatile("mov.u32 %0, %%cluster_ctarank;" : "=r"(r));
    return r;
}
__device__ __forceinline__ void fence_after() { asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory"); }

// 32 consecutive FP32 columns of one TMEM lane per thread.
__device__ __forceinline__ void tmem_ld32(uint32_t taddr, float v[32]) {
    uint32_t r[32];
    asm volatile(
        "tcgen05.ld.sync.aligned.32x32b.x32.b32 "
        "{%0,%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,%14,%15,"
        "%16,%17,%18,%19,%20,%21,%22,%23,%24,%25,%26,%27,%28,%29,%30,%31}, [%32];"
        : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]), "=r"(r[7]),
          "=r"(r[8]), "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]), "=r"(r[13]), "=r"(r[14]), "=r"(r[15]),
          "=r"(r[16]), "=r"(r[17]), "=r"(r[18]), "=r"(r[19]), "=r"(r[20]), "=r"(r[21]), "=r"(r[22]), "=r"(r[23]),
          "=r"(r[24]), "=r"(r[25]), "=r"(r[26]), "=r"(r[27]), "=r"(r[28]), "=r"(r[29]), "=r"(r[30]), "=r"(r[31])
        : "r"(taddr));
    asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
#pragma unroll
    for (int i = 0; i < 32; ++i) v[i] = __uint_as_float(r[i]);
}

// 16 consecutive FP32 columns of one TMEM lane per thread.
__device__ __forceinline__ void tmem_ld16(uint32_t taddr, float v[16]) {
    uint32_t r[16];
    asm volatile(
        "tcgen05.ld.sync.aligned.32x32b.x16.b32 "
        "{%0,%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,%14,%15}, [%16];"
        : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]), "=r"(r[7]),
          "=r"(r[8]), "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]), "=r"(r[13]), "=r"(r[14]), "=r"(r[15])
        : "r"(taddr));
    asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
#pragma unroll
    for (int i = 0; i < 16; ++i) v[i] = __uint_as_float(r[i]);
}

template <int CW>
__device__ __forceinline__ void tmem_ld(uint32_t taddr, float (&v)[CW]) {
    if constexpr (CW == 16) tmem_ld16(taddr, v);
    else tmem_ld32(taddr, v);
}

__device__ __forceinline__ float tanh_fast(float x) {
    float y;
    asm("tanh.approx.f32 %0, %1;" : "=f"(y) : "f"(x));
    return y;
}

template <int BN, int KPS>
struct Cfg {
    // one-block slots: 4 (6 for 128-wide tiles); two-block slots: the same
    // shared memory (2 slots, 3 for 128-wide tiles)
    static constexpr int STAGES = KPS == 1 ? ((BN >= 256) ? 4 : (BN >= 128 ? 6 : 4)) : (BN == 128 ? 3 : 2);
    static constexpr int A_SUB = BM * BK * 2;          // one k-block of A
    static constexpr int B_SUB = BN * BK * 2;          // one k-block of B
    static constexpr int A_BYTES = KPS * A_SUB;
    static constexpr int B_BYTES = KPS * B_SUB;
    static constexpr int STAGE_BYTES = A_BYTES + B_BYTES;
    static constexpr int SMEM = STAGES * STAGE_BYTES + 1024 /*align*/ + 256 /*barriers*/;
    static constexpr uint32_t TMEM_COLS = BN < 32 ? 32 : BN;
    static_assert(STAGE_BYTES % 1024 == 0 && B_SUB % 1024 == 0, "slots and k-blocks keep the 1024-byte swizzle atom");
};

template <int BN, int EPI, int KPS>
__global__ void __launch_bounds__(128, 1)
k_gemm_tc(const __grid_constant__ CUtensorMap tmA, const __grid_constant__ CUtensorMap tmB,
          const float* __restrict__ bias, const float* __restrict__ out_mu, float out_sigma,
          void* __restrict__ Cout, const int* __restrict__ nrows, int N, int K, const float* __restrict__ act_beta,
          int* __restrict__ err) {
    using C = Cfg<BN, KPS>;
    pdl_begin();
    const int M = *nrows;
    const int m0 = blockIdx.y * BM, n0 = blockIdx.x * BN;
    if (m0 >= M) return;

    extern __shared__ __align__(1024) uint8_t smem_raw[];
    const uint32_t raw = smem_u32(smem_raw);
    const uint32_t base = (raw + 1023u) & ~1023u;
    uint8_t* gbase = smem_raw + (base - raw);
    const uint32_t bar0 = base + C::STAGES * C::STAGE_BYTES;        // full[s], empty[s], accf
    auto full_bar = [&](int s) { return bar0 + 8u * s; };
    auto empty_bar = [&](int s) { return bar0 + 8u * (C::STAGES + s); };
    const uint32_t accf = bar0 + 8u * (2 * C::STAGES);
    uint32_t* tmem_slot = reinterpret_cast<uint32_t*>(gbase + C::STAGES * C::STAGE_BYTES + 8 * (2 * C::STAGES + 1));
    __shared__ int s_fail;

    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    if (threadIdx.x == 0) {
        s_fail = 0;
        for (int s = 0; s < C::STAGES; ++s) { mbar_init(full_bar(s), 1); mbar_init(empty_bar(s), 1); }
        mbar_init(accf, 1);
        mbar_init_fence();
    }
    if (warp == 2) {
        asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;"
                     :: "r"(smem_u32(tmem_slot)), "r"(C::TMEM_COLS) : "memory");
        asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
    }
    fence_before();
    __syncthreads();
    fence_after();
    const uint32_t tmem = *tmem_slot;
    // slots of KPS k-blocks; KPS > 1 only when K is a multiple of 64 KPS
    const int n_it = (K + BK * KPS - 1) / (BK * KPS);

    if (warp == 0 && lane == 0) {
        // TMA producer: the A and B boxes of a slot
        for (int it = 0; it < n_it; ++it) {
            const int s = it % C::STAGES;
            if (it >= C::STAGES && !mbar_wait(empty_bar(s), ((it / C::STAGES) & 1) ^ 1)) { s_fail = 1; break; }
            mbar_expect_tx(full_bar(s), C::STAGE_BYTES);
            tma_load_kb<KPS>(base + s * C::STAGE_BYTES, &tmA, full_bar(s), it, m0);
            tma_load_kb<KPS>(base + s * C::STAGE_BYTES + C::A_BYTES, &tmB, full_bar(s), it, n0);
        }
    } else if (warp == 1 && lane == 0) {
        // MMA issuer
        constexpr uint32_t idesc = instr_desc<BN>();
        for (int it = 0; it < n_it; ++it) {
            const int s = it % C::STAGES;
            if (!mbar_wait(full_bar(s), (it / C::STAGES) & 1)) { s_fail = 1; break; }
            fence_after();
            const uint32_t sa = base + s * C::STAGE_BYTES;
#pragma unroll
            for (int j = 0; j < KPS; ++j) {
                const uint64_t da = smem_desc(sa + j * C::A_SUB), db = smem_desc(sa + C::A_BYTES + j * C::B_SUB);
#pragma unroll
                for (int kk = 0; kk < BK / 16; ++kk)
                    mma_bf16(tmem, da + 2 * kk, db + 2 * kk, idesc, (it | j | kk) != 0);
            }
            mma_commit(empty_bar(s));
        }
        mma_commit(accf);
    }
    __syncwarp();

    // Epilogue: all four warps.
    const bool ok = mbar_wait(accf, 0);
    fence_after();
    __syncwarp();
    if (ok && !s_fail) {
        // column chunks of CW accumulators per thread (tile row)
        constexpr int CW = BN < 32 ? BN : 32;
        const int row = m0 + warp * 32 + lane;
        const uint32_t lane_addr = tmem + ((uint32_t)(warp * 32) << 16);
#pragma unroll 1
        for (int c = 0; c < BN / CW; ++c) {
            float v[CW];
            tmem_ld<CW>(lane_addr + c * CW, v);
            const int col0 = n0 + c * CW;
            if (row >= M || col0 >= N) continue;
            if (EPI == 0 || EPI == 2) {
                // hidden layer: tanh (EPI 0) or sigmoid-linear with per-unit
                // (g, beta) = (out_mu, act_beta) (EPI 2); stored bf16
                auto act = [&](float x, int col) {
                    if (EPI == 0) return tanh_fast(x);
                    const float g = __ldg(out_mu + col);
                    return (g + (1.f - g) / (1.f + __expf(-__ldg(act_beta + col) * x))) * x;
                };
                __nv_bfloat16* out = reinterpret_cast<__nv_bfloat16*>(Cout) + (size_t)row * N + col0;
                if (col0 + CW <= N && (N % 8) == 0) {
                    uint32_t pk[CW / 2];
#pragma unroll
                    for (int j = 0; j < CW / 2; ++j) {
                        const float a0 = act(v[2 * j] + __ldg(bias + col0 + 2 * j), col0 + 2 * j);
                        const float a1 = act(v[2 * j + 1] + __ldg(bias + col0 + 2 * j + 1), col0 + 2 * j + 1);
                        __nv_bfloat162 h2 = __floats2bfloat162_rn(a0, a1);
                        pk[j] = *reinterpret_cast<uint32_t*>(&h2);
                    }
                    uint4* o4 = reinterpret_cast<uint4*>(out);
#pragma unroll
                    for (int q = 0; q < CW / 8; ++q)
                        o4[q] = make_uint4(pk[4 * q], pk[4 * q + 1], pk[4 * q + 2], pk[4 * q + 3]);
                } else {
#pragma unroll
                    for (int j = 0; j < CW; ++j)
                        if (col0 + j < N) out[j] = __float2bfloat16_rn(act(v[j] + bias[col0 + j], col0 + j));
                }
            } else {
                float* out = reinterpret_cast<float*>(Cout) + (size_t)row * N + col0;
                if (col0 + CW <= N && (N % 4) == 0) {
                    float4* o4 = reinterpret_cast<float4*>(out);
#pragma unroll
                    for (int q = 0; q < CW / 4; ++q) {
                        float4 r;
                        r.x = __ldg(out_mu + col0 + 4 * q + 0) + out_sigma * (v[4 * q + 0] + __ldg(bias + col0 + 4 * q + 0));
                        r.y = __ldg(out_mu + col0 + 4 * q + 1) + out_sigma * (v[4 * q + 1] + __ldg(bias + col0 + 4 * q + 1));
                        r.z = __ldg(out_mu + col0 + 4 * q + 2) + out_sigma * (v[4 * q + 2] + __ldg(bias + col0 + 4 * q + 2));
                        r.w = __ldg(out_mu + col0 + 4 * q + 3) + out_sigma * (v[4 * q + 3] + __ldg(bias + col0 + 4 * q + 3));
                        o4[q] = r;
                    }
                } else {
#pragma unroll
                    for (int j = 0; j < CW; ++j)
                        if (col0 + j < N) out[j] = out_mu[col0 + j] + out_sigma * (v[j] + bias[col0 + j]);
                }
            }
        }
    }
    if ((!ok || s_fail) && threadIdx.x == 0 && err) atomicOr(err, NS_BIT_TIMEOUT);
    fence_before();
    __syncthreads();
    if (warp == 2) {
        fence_after();
        asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" :: "r"(tmem), "r"(C::TMEM_COLS) : "memory");
    }
}

// Output layer with swapped operands for a small row count: the MMA's M is
// 128 output features (rows of W, the A operand) and its N is BR activation
// rows (the B operand), D^T[f][r] = W[f][:] . X[r][:] in TMEM.  With
// BR = 256 the 39-d output layer (10000 features, <= 500 rows) is one wave of
// CTAs; each thread owns one feature, so mu / bias are loaded once per thread
// and for every row the 32 lanes of a warp store 32 consecutive features.
template <int BR>
struct CfgS {
    static constexpr int STAGES = 2;   // 96 KB: leaves room for other kernels' CTAs on the SM
    static constexpr int A_BYTES = 128 * BK * 2;
    static constexpr int B_BYTES = BR * BK * 2;
    static constexpr int STAGE_BYTES = A_BYTES + B_BYTES;
    static constexpr int SMEM = STAGES * STAGE_BYTES + 1024 + 256;
    static constexpr uint32_t TMEM_COLS = BR;
};

template <int BR>
__global__ void __launch_bounds__(128, 1)
k_gemm_tc_swap(const __grid_constant__ CUtensorMap tmW, const __grid_constant__ CUtensorMap tmX,
               const float* __restrict__ bias, const float* __restrict__ out_mu, float out_sigma,
               float* __restrict__ Cout, const int* __restrict__ nrows, int N, int K, int* __restrict__ err) {
    using C = CfgS<BR>;
    pdl_begin();
    const int M = *nrows;
    const int f0 = blockIdx.x * 128, r0 = blockIdx.y * BR;
    if (r0 >= M) return;

    extern __shared__ __align__(1024) uint8_t smem_raw[];
    const uint32_t raw = smem_u32(smem_raw);
    const uint32_t base = (raw + 1023u) & ~1023u;
    uint8_t* gbase = smem_raw + (base - raw);
    const uint32_t bar0 = base + C::STAGES * C::STAGE_BYTES;
    auto full_bar = [&](int s) { return bar0 + 8u * s; };
    auto empty_bar = [&](int s) { return bar0 + 8u * (C::STAGES + s); };
    const uint32_t accf = bar0 + 8u * (2 * C::STAGES);
    uint32_t* tmem_slot = reinterpret_cast<uint32_t*>(gbase + C::STAGES * C::STAGE_BYTES + 8 * (2 * C::STAGES + 1));
    __shared__ int s_fail;

    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    if (threadIdx.x == 0) {
        s_fail = 0;
        for (int s = 0; s < C::STAGES; ++s) { mbar_init(full_bar(s), 1); mbar_init(empty_bar(s), 1); }
        mbar_init(accf, 1);
        mbar_init_fence();
    }
    if (warp == 2) {
        asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;"
                     :: "r"(smem_u32(tmem_slot)), "r"(C::TMEM_COLS) : "memory");
        asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
    }
    fence_before();
    __syncthreads();
    fence_after();
    const uint32_t tmem = *tmem_slot;
    const int nk = (K + BK - 1) / BK;

    if (warp == 0 && lane == 0) {
        for (int kb = 0; kb < nk; ++kb) {
            const int s = kb % C::STAGES;
            if (kb >= C::STAGES && !mbar_wait(empty_bar(s), ((kb / C::STAGES) & 1) ^ 1)) { s_fail = 1; break; }
            const uint32_t sa = base + s * C::STAGE_BYTES;
            mbar_expect_tx(full_bar(s), C::STAGE_BYTES);
            tma_load_2d(sa, &tmW, full_bar(s), kb * BK, f0);
            tma_load_2d(sa + C::A_BYTES, &tmX, full_bar(s), kb * BK, r0);
        }
    } else if (warp == 1 && lane == 0) {
        // M = 128 features, N = BR rows
        constexpr uint32_t idesc = (1u << 4) | (1u << 7) | (1u << 10) | ((uint32_t)(BR >> 3) << 17) |
                                   ((uint32_t)(128 >> 4) << 24);
        for (int kb = 0; kb < nk; ++kb) {
            const int s = kb % C::STAGES;
            if (!mbar_wait(full_bar(s), (kb / C::STAGES) & 1)) { s_fail = 1; break; }
            fence_after();
            const uint32_t sa = base + s * C::STAGE_BYTES;
            const uint64_t da = smem_desc(sa), db = smem_desc(sa + C::A_BYTES);
#pragma unroll
            for (int kk = 0; kk < BK / 16; ++kk)
                mma_bf16(tmem, da + 2 * kk, db + 2 * kk, idesc, (kb | kk) != 0);
            mma_commit(empty_bar(s));
        }
        mma_commit(accf);
    }
    __syncwarp();

    const bool ok = mbar_wait(accf, 0);
    fence_after();
    __syncwarp();
    if (ok && !s_fail) {
        const int f = f0 + warp * 32 + lane;
        const bool valid = f < N;
        const float mu_f = valid ? __ldg(out_mu + f) : 0.f;
        const float b_f = valid ? __ldg(bias + f) : 0.f;
        const uint32_t lane_addr = tmem + ((uint32_t)(warp * 32) << 16);
#pragma unroll 1
        for (int c = 0; c < BR / 32; ++c) {
            if (r0 + c * 32 >= M) break;
            float v[32];
            tmem_ld32(lane_addr + c * 32, v);
            if (!valid) continue;
#pragma unroll
            for (int j = 0; j < 32; ++j) {
                const int r = r0 + c * 32 + j;
                if (r < M) Cout[(size_t)r * N + f] = mu_f + out_sigma * (v[j] + b_f);
            }
        }
    }
    if ((!ok || s_fail) && threadIdx.x == 0 && err) atomicOr(err, NS_BIT_TIMEOUT);
    fence_before();
    __syncthreads();
    if (warp == 2) {
        fence_after();
        asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" :: "r"(tmem), "r"(C::TMEM_COLS) : "memory");
    }
}

// ------------------------------------------------------------------ split-BF16 GEMM
// FP32-accurate products on the bf16 tensor path, for the adjoint: the A
// operand is held as two bf16 matrices whose sum is the FP32 value
// (hi = bf16(a), lo = bf16(a - hi), ~2^-17 relative), B is exact in bf16 (the
// emulator's weights), and every k-block issues MMA(A_hi, B) and MMA(A_lo, B)
// into one FP32 accumulator.  One CTA computes a 128 x BN tile; TMA ring of
// STAGES slots holding A_hi | A_lo | B boxes; warp roles as in k_gemm_tc.
// Epilogues (thread = tile row):
//   SPL_TANH   h = tanh(acc + b) -> (hi, lo) pair                    [forward hidden]
//   SPL_OUT    mu + sigma (acc + b) -> FP32                          [forward output]
//   SPL_DTANH  g = acc (1 - h^2), h = aux_hi + aux_lo -> (hi, lo)    [backward hidden]
//   SPL_DTANH32 the same -> FP32                                      [backward, first hidden layer]
template <int BN>
struct CfgSplit {
    static constexpr int STAGES = (BN >= 256) ? 3 : 4;
    static constexpr int A_BYTES = BM * BK * 2;
    static constexpr int B_BYTES = BN * BK * 2;
    static constexpr int STAGE_BYTES = 2 * A_BYTES + B_BYTES;
    static constexpr int SMEM = STAGES * STAGE_BYTES + 1024 + 256;
    static constexpr uint32_t TMEM_COLS = BN < 32 ? 32 : BN;
};

__device__ __forceinline__ void split_store32(const float (&v)[32], __nv_bfloat16* hi, __nv_bfloat16* lo, int nvalid,
                                              bool vec) {
    if (vec) {
        uint32_t ph[16], pl[16];
#pragma unroll
        for (int j = 0; j < 16; ++j) {
            const __nv_bfloat162 h2 = __floats2bfloat162_rn(v[2 * j], v[2 * j + 1]);
            const float2 hf = __bfloat1622float2(h2);
            const __nv_bfloat162 l2 = __floats2bfloat162_rn(v[2 * j] - hf.x, v[2 * j + 1] - hf.y);
            ph[j] = *reinterpret_cast<const uint32_t*>(&h2);
            pl[j] = *reinterpret_cast<const uint32_t*>(&l2);
        }
        uint4* oh = reinterpret_cast<uint4*>(hi);
        uint4* ol = reinterpret_cast<uint4*>(lo);
#pragma unroll
        for (int q = 0; q < 4; ++q) {
            oh[q] = make_uint4(ph[4 * q], ph[4 * q + 1], ph[4 * q + 2], ph[4 * q + 3]);
            ol[q] = make_uint4(pl[4 * q], pl[4 * q + 1], pl[4 * q + 2], pl[4 * q + 3]);
        }
    } else {
#pragma unroll
        for (int j = 0; j < 32; ++j)
            if (j < nvalid) {
                const __nv_bfloat16 h = __float2bfloat16_rn(v[j]);
                hi[j] = h;
                lo[j] = __float2bfloat16_rn(v[j] - __bfloat162float(h));
            }
    }
}

template <int BN, int EPI>
__global__ void __launch_bounds__(128, 1)
k_gemm_split(const __grid_constant__ CUtensorMap tmAhi, const __grid_constant__ CUtensorMap tmAlo,
             const __grid_constant__ CUtensorMap tmB, const float* __restrict__ bias, const float* __restrict__ out_mu,
             float out_sigma, void* __restrict__ Cout, __nv_bfloat16* __restrict__ Clo,
             const __nv_bfloat16* __restrict__ aux_hi, const __nv_bfloat16* __restrict__ aux_lo,
             const int* __restrict__ nrows, int N, int K, int* __restrict__ err) {
    using C = CfgSplit<BN>;
    pdl_begin();
    const int M = *nrows;
    const int m0 = blockIdx.y * BM, n0 = blockIdx.x * BN;
    if (m0 >= M) return;

    extern __shared__ __align__(1024) uint8_t smem_raw[];
    const uint32_t raw = smem_u32(smem_raw);
    const uint32_t base = (raw + 1023u) & ~1023u;
    uint8_t* gbase = smem_raw + (base - raw);
    const uint32_t bar0 = base + C::STAGES * C::STAGE_BYTES;
    auto full_bar = [&](int s) { return bar0 + 8u * s; };
    auto empty_bar = [&](int s) { return bar0 + 8u * (C::STAGES + s); };
    const uint32_t accf = bar0 + 8u * (2 * C::STAGES);
    uint32_t* tmem_slot = reinterpret_cast<uint32_t*>(gbase + C::STAGES * C::STAGE_BYTES + 8 * (2 * C::STAGES + 1));
    __shared__ int s_fail;

    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    if (threadIdx.x == 0) {
        s_fail = 0;
        for (int s = 0; s < C::STAGES; ++s) { mbar_init(full_bar(s), 1); mbar_init(empty_bar(s), 1); }
        mbar_init(accf, 1);
        mbar_init_fence();
    }
    if (warp == 2) {
        asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;"
                     :: "r"(smem_u32(tmem_slot)), "r"(C::TMEM_COLS) : "memory");
        asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
    }
    fence_before();
    __syncthreads();
    fence_after();
    const uint32_t tmem = *tmem_slot;
    const int nk = (K + BK - 1) / BK;

    if (warp == 0 && lane == 0) {
        for (int kb = 0; kb < nk; ++kb) {
            const int s = kb % C::STAGES;
            if (kb >= C::STAGES && !mbar_wait(empty_bar(s), ((kb / C::STAGES) & 1) ^ 1)) { s_fail = 1; break; }
            const uint32_t sa = base + s * C::STAGE_BYTES;
            mbar_expect_tx(full_bar(s), C::STAGE_BYTES);
            tma_load_2d(sa, &tmAhi, full_bar(s), kb * BK, m0);
            tma_load_2d(sa + C::A_BYTES, &tmAlo, full_bar(s), kb * BK, m0);
            tma_load_2d(sa + 2 * C::A_BYTES, &tmB, full_bar(s), kb * BK, n0);
        }
    } else if (warp == 1 && lane == 0) {
        constexpr uint32_t idesc = instr_desc<BN>();
        for (int kb = 0; kb < nk; ++kb) {
            const int s = kb % C::STAGES;
            if (!mbar_wait(full_bar(s), (kb / C::STAGES) & 1)) { s_fail = 1; break; }
            fence_after();
            const uint32_t sa = base + s * C::STAGE_BYTES;
            const uint64_t dh = smem_desc(sa), dl = smem_desc(sa + C::A_BYTES), db = smem_desc(sa + 2 * C::A_BYTES);
#pragma unroll
            for (int kk = 0; kk < BK / 16; ++kk) {
                mma_bf16(tmem, dh + 2 * kk, db + 2 * kk, idesc, (kb | kk) != 0);
                mma_bf16(tmem, dl + 2 * kk, db + 2 * kk, idesc, 1u);
            }
            mma_commit(empty_bar(s));
        }
        mma_commit(accf);
    }
    __syncwarp();

    const bool ok = mbar_wait(accf, 0);
    fence_after();
    __syncwarp();
    if (ok && !s_fail) {
        const int row = m0 + warp * 32 + lane;
        const uint32_t lane_addr = tmem + ((uint32_t)(warp * 32) << 16);
#pragma unroll 1
        for (int c = 0; c < BN / 32; ++c) {
            float v[32];
            tmem_ld32(lane_addr + c * 32, v);
            const int col0 = n0 + c * 32;
            if (row >= M || col0 >= N) continue;
            const int nvalid = min(32, N - col0);
            const bool vec = nvalid == 32 && (N % 8) == 0;
            const size_t off = (size_t)row * N + col0;
            if (EPI == SPL_OUT) {
                float* out = reinterpret_cast<float*>(Cout) + off;
#pragma unroll
                for (int j = 0; j < 32; ++j)
                    if (j < nvalid) out[j] = out_mu[col0 + j] + out_sigma * (v[j] + bias[col0 + j]);
                continue;
            }
            if (EPI == SPL_TANH) {
#pragma unroll
                for (int j = 0; j < 32; ++j) v[j] = (j < nvalid) ? tanhf(v[j] + bias[col0 + j]) : 0.f;
            } else {
#pragma unroll
                for (int j = 0; j < 32; ++j) {
                    if (j < nvalid) {
                        const float h = __bfloat162float(aux_hi[off + j]) + __bfloat162float(aux_lo[off + j]);
                        v[j] *= 1.f - h * h;
                    }
                }
            }
            if (EPI == SPL_DTANH32) {
                float* out = reinterpret_cast<float*>(Cout) + off;
#pragma unroll
                for (int j = 0; j < 32; ++j)
                    if (j < nvalid) out[j] = v[j];
            } else {
                split_store32(v, reinterpret_cast<__nv_bfloat16*>(Cout) + off, Clo + off, nvalid, vec);
            }
        }
    }
    if ((!ok || s_fail) && threadIdx.x == 0 && err) atomicOr(err, NS_BIT_TIMEOUT);
    fence_before();
    __syncthreads();
    if (warp == 2) {
        fence_after();
        asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" :: "r"(tmem), "r"(C::TMEM_COLS) : "memory");
    }
}

template <int BN>
static int launch_split_bn(const CUtensorMap* tmAhi, const CUtensorMap* tmAlo, const CUtensorMap* tmB,
                           const float* bias, const float* mu, float sigma, void* C, __nv_bfloat16* Clo,
                           const __nv_bfloat16* aux_hi, const __nv_bfloat16* aux_lo, const int* nrows, int grid_rows,
                           int N, int K, int epi, int* err, cudaStream_t st) {
    using CF = CfgSplit<BN>;
    static bool attr = false;
    if (!attr) {
        NS_CUDA_TRY(cudaFuncSetAttribute(k_gemm_split<BN, SPL_TANH>, cudaFuncAttributeMaxDynamicSharedMemorySize, CF::SMEM));
        NS_CUDA_TRY(cudaFuncSetAttribute(k_gemm_split<BN, SPL_OUT>, cudaFuncAttributeMaxDynamicSharedMemorySize, CF::SMEM));
        NS_CUDA_TRY(cudaFuncSetAttribute(k_gemm_split<BN, SPL_DTANH>, cudaFuncAttributeMaxDynamicSharedMemorySize, CF::SMEM));
        NS_CUDA_TRY(cudaFuncSetAttribute(k_gemm_split<BN, SPL_DTANH32>, cudaFuncAttributeMaxDynamicSharedMemorySize, CF::SMEM));
        attr = true;
    }
    dim3 grid((N + BN - 1) / BN, (grid_rows + BM - 1) / BM);
    auto kern = epi == SPL_TANH ? k_gemm_split<BN, SPL_TANH> : epi == SPL_OUT ? k_gemm_split<BN, SPL_OUT>
              : epi == SPL_DTANH ? k_gemm_split<BN, SPL_DTANH> : k_gemm_split<BN, SPL_DTANH32>;
    NS_CUDA_TRY(launch_pdl(kern, grid, dim3(128), (size_t)CF::SMEM, st, *tmAhi, *tmAlo, *tmB, bias, mu, sigma, C, Clo,
                           aux_hi, aux_lo, nrows, N, K, err));
    return NS_OK;
}

template <int BN, int KPS>
static int launch_bn_kps(const CUtensorMap* tmA, const CUtensorMap* tmB, const float* bias, const float* mu,
                         float sigma, void* Cout, const int* nrows, int grid_rows, int N, int K, int epi,
                         const float* beta, int* err, cudaStream_t st) {
    using C = Cfg<BN, KPS>;
    static bool attr = false;
    if (!attr) {
        NS_CUDA_TRY(cudaFuncSetAttribute(k_gemm_tc<BN, 0, KPS>, cudaFuncAttributeMaxDynamicSharedMemorySize, C::SMEM));
        NS_CUDA_TRY(cudaFuncSetAttribute(k_gemm_tc<BN, 1, KPS>, cudaFuncAttributeMaxDynamicSharedMemorySize, C::SMEM));
        NS_CUDA_TRY(cudaFuncSetAttribute(k_gemm_tc<BN, 2, KPS>, cudaFuncAttributeMaxDynamicSharedMemorySize, C::SMEM));
        attr = true;
    }
    dim3 grid((N + BN - 1) / BN, (grid_rows + BM - 1) / BM);
    auto kern = (epi == TC_EPI_TANH) ? k_gemm_tc<BN, 0, KPS>
              : (epi == TC_EPI_OUT) ? k_gemm_tc<BN, 1, KPS> : k_gemm_tc<BN, 2, KPS>;
    NS_CUDA_TRY(launch_pdl(kern, grid, dim3(128), (size_t)C::SMEM, st, *tmA, *tmB, bias, mu, sigma, Cout, nrows, N,
                           K, beta, err));
    return NS_OK;
}

template <int BN>
static int launch_bn(const CUtensorMap* tmA, const CUtensorMap* tmB, const float* bias, const float* mu,
                     float sigma, void* Cout, const int* nrows, int grid_rows, int N, int K, int epi,
                     const float* beta, int* err, cudaStream_t st) {
    if (gemm_tc_kps(K) == 2)
        return launch_bn_kps<BN, 2>(tmA, tmB, bias, mu, sigma, Cout, nrows, grid_rows, N, K, epi, beta, err, st);
    return launch_bn_kps<BN, 1>(tmA, tmB, bias, mu, sigma, Cout, nrows, grid_rows, N, K, epi, beta, err, st);
}


// ------------------------------------------------------------------ fused emulator stack
// The input layer and every hidden layer of a BF16 emulator whose hidden
// widths all equal H = 128 CS (CS <= 8), in one kernel.  A thread-block
// cluster of CS CTAs takes a tile of FR = 64 rows; CTA q owns features
// [128 q, 128 q + 128) of every layer.  The tile's activations (FR x H bf16)
// stay in each CTA's shared memory as the MMA's B operand (K-major, 128-byte
// swizzle, k-block after k-block); the CTA's weight slice (128 x H) streams
// through a two-slot TMA ring (two k-blocks per copy) and
// tcgen05.mma.cta_group::1 (M = 128 features, N = FR rows) accumulates
// D^T = W_q A^T in TMEM.  The epilogue (tanh, bf16) writes the CTA's output
// slice (FR x 128) to a staging tile in the same swizzled layout, and one
// thread pushes it into every CTA's activation buffer with
// cp.async.bulk.shared::cluster, completing on the receiver's A_ready barrier;
// the last layer's slice goes to global memory by a TMA store instead.  A
// slice may be pushed only when every CTA of the cluster has finished the
// layer (its MMAs read the buffer being overwritten): each CTA arrives on
// every peer's `ready` barrier (release, cluster scope) after its epilogue,
// and the pushers wait on their own (acquire); lane p of warp 0 arrives on and
// pushes to peer p, so the CS arrivals and copies are issued in parallel.  The
// input layer (K0 <= 32 inputs, FP32 on CUDA cores, the arithmetic of
// k_emu_input) fills the first staging tile.  Warps 0-7: input layer and
// epilogues (warp w reads TMEM lanes 32 (w % 4) .. + 31 = features, rows
// 32 (w / 4) .. + 31); warp 8 lane 0: weight producer (all layers, ahead of
// the MMAs); warp 9: TMEM owner and MMA issuer.  Every wait is bounded; after a timeout
// the CTA records NS_BIT_TIMEOUT, skips its MMAs and keeps the protocol's
// arrivals, and all threads of the cluster meet at a final cluster barrier
// before TMEM is freed and the CTAs exit.
constexpr int FR = 64;                   // rows per cluster tile
constexpr int F_SLICE = 128;             // features per CTA
constexpr int F_SLOT = 2 * F_SLICE * BK * 2;   // ring slot: two k-blocks of the weight slice (32 KB)
constexpr int F_STAGING = FR * F_SLICE * 2;    // the CTA's output slice (16 KB)
constexpr int F_KIN = 32;                // largest input count of the fused input layer
constexpr int F_EPI = 256;              // input-layer / epilogue threads (8 warps)
constexpr int F_THREADS = F_EPI + 64;

struct FusedMaps {
    CUtensorMap w[kFusedMaxHidden + 1];  // [l] for hidden layers l = 1 .. n_h: box 128 rows x (2 x 64) k
    CUtensorMap out;                     // the last layer's activations: box FR rows x (2 x 64) k
};
struct FusedArgs {
    const double* theta;                 // rows x P
    int P, K0, n_h;
    const int* inputs;
    const double* center;
    const double* inv_scale;
    const float* W0;                     // H x K0
    const float* b0;
    const float* bh[kFusedMaxHidden + 1];// hidden biases, [l] for l = 1 .. n_h
    const int* nrows;
    int* err;
};

__device__ __forceinline__ uint32_t mapa_u32(uint32_t addr, uint32_t rank) {
    uint32_t r;
    asm volatile("mapa.shared::cluster.u32 %0, %1, %2;" : "=r"(r) : "r"(addr), "r"(rank));
    return r;
}
__device__ __forceinline__ void mbar_arrive_remote(uint32_t cluster_bar) {
    asm volatile("mbarrier.arrive.release.cluster.shared::cluster.b64 _, [%0];" :: "r"(cluster_bar) : "memory");
}
__device__ __forceinline__ bool mbar_try_wait_cluster(uint32_t bar, uint32_t parity) {
    uint32_t ok;
    asm volatile(
        "{\n\t.reg .pred p;\n\t"
        "mbarrier.try_wait.parity.acquire.cluster.shared::cta.b64 p, [%1], %2;\n\t"
        "selp.u32 %0, 1, 0, p;\n\t}"
        : "=r"(ok) : "r"(bar), "r"(parity) : "memory");
    return ok != 0;
}
// bounded wait with cluster-scope acquire (peers' arrivals)
__device__ __forceinline__ bool mbar_wait_cluster(uint32_t bar, uint32_t parity) {
    if (mbar_try_wait_cluster(bar, parity)) return true;
    const uint64_t t0 = globaltimer();
    for (uint32_t i = 1;; ++i) {
        if (mbar_try_wait_cluster(bar, parity)) return true;
        if ((i & 255u) == 0) {
            __nanosleep(64);
            if (globaltimer() - t0 > kWaitNs) return false;
        }
    }
}
// shared::cta -> shared::cluster bulk copy (a peer's buffer), completing on the peer's barrier
__device__ __forceinline__ void bulk_s2cluster(uint32_t dst_cluster, uint32_t src, uint32_t bytes,
                                               uint32_t bar_cluster) {
    asm volatile(
        "cp.async.bulk.shared::cluster.shared::cta.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];"
        :: "r"(dst_cluster), "r"(src), "r"(bytes), "r"(bar_cluster) : "memory");
}
__device__ __forceinline__ void tma_store_3d(const CUtensorMap* tm, uint32_t src, int x, int y, int z) {
    asm volatile("cp.async.bulk.tensor.3d.global.shared::cta.bulk_group [%0, {%2, %3, %4}], [%1];"
                 :: "l"(reinterpret_cast<uint64_t>(tm)), "r"(src), "r"(x), "r"(y), "r"(z) : "memory");
}
__device__ __forceinline__ void bulk_commit() { asm volatile("cp.async.bulk.commit_group;" ::: "memory"); }
__device__ __forceinline__ void bulk_wait_read0() { asm volatile("cp.async.bulk.wait_group.read 0;" ::: "memory"); }
__device__ __forceinline__ void bulk_wait0() { asm volatile("cp.async.bulk.wait_group 0;" ::: "memory"); }
__device__ __forceinline__ void fence_proxy_async_smem() { asm volatile("fence.proxy.async.shared::cta;" ::: "memory"); }
__device__ __forceinline__ void named_sync_epi() { asm volatile("bar.sync 1, 256;" ::: "memory"); }
__device__ __forceinline__ void cluster_sync_all() {
    asm volatile("barrier.cluster.arrive.release.aligned;\n\tbarrier.cluster.wait.acquire.aligned;" ::: "memory");
}

// byte offset of element (row r, k) of a k-block tile of FR rows x 64 k, 128-byte swizzle
__device__ __forceinline__ uint32_t swz_off(int r, int k) {
    return (uint32_t)(r * 128 + ((((k >> 3) ^ (r & 7)) & 7) << 4) + ((k & 7) << 1));
}

template <int CS>
__global__ void __launch_bounds__(F_THREADS, 1)
k_emu_fused(const __grid_constant__ FusedMaps maps, const FusedArgs args) {
    constexpr int H = F_SLICE * CS;
    constexpr int A_BYTES = FR * H * 2;              // the tile's activations, H / 64 k-blocks of FR x 64
    constexpr int NKB2 = H / (2 * BK);               // ring slots per layer
    pdl_begin();
    const int M = *args.nrows;
    const int r0 = blockIdx.y * FR;
    if (r0 >= M) return;                             // the whole cluster (same row tile) leaves together
    const uint32_t q = cluster_ctarank();

    extern __shared__ __align__(1024) uint8_t smem_raw[];
    const uint32_t raw = smem_u32(smem_raw);
    const uint32_t base = (raw + 1023u) & ~1023u;
    uint8_t* gbase = smem_raw + (base - raw);
    const uint32_t sA = base;                        // A_BYTES
    const uint32_t sRing = base + A_BYTES;           // 2 x F_SLOT
    const uint32_t sS = sRing + 2 * F_SLOT;          // F_STAGING
    uint8_t* gS = gbase + (A_BYTES + 2 * F_SLOT);
    const uint32_t bar0 = sS + F_STAGING;
    auto full_bar = [&](int s) { return bar0 + 8u * s; };
    auto empty_bar = [&](int s) { return bar0 + 16u + 8u * s; };
    const uint32_t accf = bar0 + 32u, a_ready = bar0 + 40u, ready = bar0 + 48u;
    uint32_t* tmem_slot = reinterpret_cast<uint32_t*>(gbase + (A_BYTES + 2 * F_SLOT + F_STAGING) + 64);
    __shared__ float xin[FR][F_KIN];
    __shared__ int s_fail;

    const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
    if (tid == 0) {
        s_fail = 0;
        for (int s = 0; s < 2; ++s) { mbar_init(full_bar(s), 1); mbar_init(empty_bar(s), 1); }
        mbar_init(accf, 1);
        mbar_init(a_ready, 1);
        mbar_init(ready, CS);                        // one arrival from every CTA of the cluster per layer
        mbar_init_fence();
    }
    if (warp == 9) {
        asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;"
                     :: "r"(smem_u32(tmem_slot)), "r"(64) : "memory");
        asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
    }
    fence_before();
    __syncthreads();
    fence_after();
    // every CTA's barriers are initialised before any peer arrives on them
    cluster_sync_all();
    const uint32_t tmem = *tmem_slot;
    const int n_h = args.n_h;

    if (warp == 8) {
        if (lane == 0) {
            // weight producer: slots of two k-blocks of the CTA's 128-feature slice, all layers in order
            int g = 0;
            for (int l = 1; l <= n_h; ++l)
                for (int kb2 = 0; kb2 < NKB2; ++kb2, ++g) {
                    const int s = g & 1;
                    if (g >= 2 && !mbar_wait(empty_bar(s), ((g >> 1) & 1) ^ 1)) { s_fail = 1; break; }
                    mbar_expect_tx(full_bar(s), F_SLOT);
                    tma_load_3d(sRing + s * F_SLOT, &maps.w[l], full_bar(s), 0, (int)q * F_SLICE, 2 * kb2);
                }
        }
        __syncwarp();
    } else if (warp == 9) {
        if (lane == 0) {
            // MMA issuer: layer l waits for its activations (phase l - 1), then the ring
            constexpr uint32_t idesc = (1u << 4) | (1u << 7) | (1u << 10) | ((uint32_t)(FR >> 3) << 17) |
                                       ((uint32_t)(F_SLICE >> 4) << 24);
            int g = 0;
            bool ok = true;
            for (int l = 1; l <= n_h; ++l) {
                ok = ok && mbar_wait(a_ready, (l - 1) & 1);
                fence_after();
                for (int kb2 = 0; kb2 < NKB2; ++kb2, ++g) {
                    const int s = g & 1;
                    ok = ok && mbar_wait(full_bar(s), (g >> 1) & 1);
                    fence_after();
                    if (ok) {
#pragma unroll
                        for (int j = 0; j < 2; ++j) {
                            const uint64_t dw = smem_desc(sRing + s * F_SLOT + j * (F_SLICE * BK * 2));
                            const uint64_t da = smem_desc(sA + (2 * kb2 + j) * (FR * BK * 2));
#pragma unroll
                            for (int kk = 0; kk < BK / 16; ++kk)
                                mma_bf16(tmem, dw + 2 * kk, da + 2 * kk, idesc, (kb2 | j | kk) != 0);
                        }
                    }
                    mma_commit(empty_bar(s));        // frees the slot (or releases it unused after a failure)
                }
                mma_commit(accf);
            }
            if (!ok) s_fail = 1;
        }
        __syncwarp();
    } else {
        // warps 0-7: thread tid owns feature 128 q + e (TMEM lane e) for rows
        // [32 h, 32 h + 32), h = tid / 128
        const int e = tid & (F_SLICE - 1), h = tid >> 7;
        auto write_slice = [&](int r, float v) {
            *reinterpret_cast<__nv_bfloat16*>(gS + (e >> 6) * (FR * BK * 2) + swz_off(r, e & 63)) =
                __float2bfloat16_rn(v);
        };
        // hand the staged slice of layer l to every CTA (or, after the last layer, to global memory)
        auto boundary = [&](int l) {
            fence_proxy_async_smem();
            fence_before();
            named_sync_epi();
            if (warp == 0) {
                // the next layer's activations: CS slices arriving from the peers
                if (lane == 0 && l < n_h) mbar_expect_tx(a_ready, A_BYTES);
                __syncwarp();
                if (lane < CS) mbar_arrive_remote(mapa_u32(ready, (uint32_t)lane));
                bool okw = true;
                if (lane == 0) okw = mbar_wait_cluster(ready, l & 1);
                okw = __shfl_sync(0xffffffffu, okw ? 1 : 0, 0) != 0;
                if (!okw && lane == 0) s_fail = 1;
                if (l < n_h) {
                    if (lane < CS)
                        bulk_s2cluster(mapa_u32(sA + q * (2 * FR * BK * 2), (uint32_t)lane), sS, F_STAGING,
                                       mapa_u32(a_ready, (uint32_t)lane));
                    if (lane < CS) { bulk_commit(); bulk_wait_read0(); }
                } else if (lane == 0) {
                    tma_store_3d(&maps.out, sS, 0, r0, 2 * (int)q);
                    bulk_commit();
                    bulk_wait0();
                }
                __syncwarp();
            }
            named_sync_epi();
        };
        // input layer: x = (theta[inputs] - center) * inv_scale (FP64, then FP32), h = tanh(W0 x + b0)
        const int K0 = args.K0;
        for (int i = tid; i < FR * K0; i += F_EPI) {
            const int r = i / K0, j = i - r * K0;
            float xv = 0.f;
            if (r0 + r < M) {
                const double v = args.theta[(size_t)(r0 + r) * args.P + args.inputs[j]] - args.center[j];
                xv = (float)(v * args.inv_scale[j]);
            }
            xin[r][j] = xv;
        }
        named_sync_epi();
        {
            const int n = (int)q * F_SLICE + e;
            float w[F_KIN];
#pragma unroll
            for (int j = 0; j < F_KIN; ++j) w[j] = j < K0 ? args.W0[(size_t)n * K0 + j] : 0.f;
            const float bn = args.b0[n];
            for (int r = 32 * h; r < 32 * h + 32; ++r) {
                float acc = bn;
#pragma unroll
                for (int j = 0; j < F_KIN; ++j)
                    if (j < K0) acc = fmaf(w[j], xin[r][j], acc);
                write_slice(r, tanhf(acc));
            }
        }
        boundary(0);
        const uint32_t lane_addr = tmem + ((uint32_t)((warp & 3) * 32) << 16) + 32 * h;
        for (int l = 1; l <= n_h; ++l) {
            const bool ok = mbar_wait(accf, (l - 1) & 1);
            fence_after();
            if (!ok) s_fail = 1;
            const float b = args.bh[l][(int)q * F_SLICE + e];
            float v[32];
            tmem_ld32(lane_addr, v);
#pragma unroll
            for (int j = 0; j < 32; ++j) write_slice(32 * h + j, tanh_fast(v[j] + b));
            boundary(l);
        }
    }
    // every thread of the cluster meets here: no CTA leaves while a peer may
    // still push into its shared memory or arrive on its barriers
    fence_before();
    __syncwarp();
    cluster_sync_all();
    if (s_fail && tid == 0 && args.err) atomicOr(args.err, NS_BIT_TIMEOUT);
    if (warp == 9) {
        fence_after();
        asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" :: "r"(tmem), "r"(64) : "memory");
    }
}

template <int CS>
static int launch_fused_cs(const FusedMaps& maps, const FusedArgs& args, int grid_rows, cudaStream_t st) {
    constexpr int H = F_SLICE * CS;
    constexpr size_t SMEM = (size_t)FR * H * 2 + 2 * F_SLOT + F_STAGING + 1024 /*align*/ + 256 /*barriers*/;
    static bool attr = false;
    if (!attr) {
        NS_CUDA_TRY(cudaFuncSetAttribute(k_emu_fused<CS>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)SMEM));
        attr = true;
    }
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = dim3(CS, (grid_rows + FR - 1) / FR);
    cfg.blockDim = dim3(F_THREADS);
    cfg.dynamicSmemBytes = SMEM;
    cfg.stream = st;
    cudaLaunchAttribute attr2[2];
    attr2[0].id = cudaLaunchAttributeClusterDimension;
    attr2[0].val.clusterDim.x = CS;
    attr2[0].val.clusterDim.y = 1;
    attr2[0].val.clusterDim.z = 1;
    attr2[1].id = cudaLaunchAttributeProgrammaticStreamSerialization;
    attr2[1].val.programmaticStreamSerializationAllowed = 1;
    cfg.attrs = attr2;
    cfg.numAttrs = 2;
    NS_CUDA_TRY(cudaLaunchKernelEx(&cfg, k_emu_fused<CS>, maps, args));
    return NS_OK;
}

}  // namespace tc

int launch_gemm_tc(const CUtensorMap* tmA, const CUtensorMap* tmB, int tile_n, const float* bias,
                   const float* out_mu, float out_sigma, void* C, const int* d_nrows, int grid_rows, int N, int K,
                   int epi, const float* act_beta, int* d_err, cudaStream_t st) {
    if (grid_rows <= 0) return NS_OK;
    switch (tile_n) {
        case 16: return tc::launch_bn<16>(tmA, tmB, bias, out_mu, out_sigma, C, d_nrows, grid_rows, N, K, epi, act_beta, d_err, st);
        case 32: return tc::launch_bn<32>(tmA, tmB, bias, out_mu, out_sigma, C, d_nrows, grid_rows, N, K, epi, act_beta, d_err, st);
        case 64: return tc::launch_bn<64>(tmA, tmB, bias, out_mu, out_sigma, C, d_nrows, grid_rows, N, K, epi, act_beta, d_err, st);
        case 128: return tc::launch_bn<128>(tmA, tmB, bias, out_mu, out_sigma, C, d_nrows, grid_rows, N, K, epi, act_beta, d_err, st);
        case 256: return tc::launch_bn<256>(tmA, tmB, bias, out_mu, out_sigma, C, d_nrows, grid_rows, N, K, epi, act_beta, d_err, st);
        default: return NS_EINVAL;
    }
}

int launch_gemm_tc_out_swap(const CUtensorMap* tmW, const CUtensorMap* tmX, const float* bias, const float* out_mu,
                            float out_sigma, float* C, const int* d_nrows, int grid_rows, int N, int K, int* d_err,
                            cudaStream_t st) {
    if (grid_rows <= 0) return NS_OK;
    constexpr int BR = kSwapRows;
    using CS = tc::CfgS<BR>;
    static bool attr = false;
    if (!attr) {
        NS_CUDA_TRY(cudaFuncSetAttribute(tc::k_gemm_tc_swap<BR>, cudaFuncAttributeMaxDynamicSharedMemorySize, CS::SMEM));
        attr = true;
    }
    dim3 grid((N + 127) / 128, (grid_rows + BR - 1) / BR);
    NS_CUDA_TRY(launch_pdl(tc::k_gemm_tc_swap<BR>, grid, dim3(128), (size_t)CS::SMEM, st, *tmW, *tmX, bias, out_mu,
                           out_sigma, C, d_nrows, N, K, d_err));
    return NS_OK;
}

int launch_emu_fused(const ns_problem* p, const Workspace* ws, int grid_rows, cudaStream_t st) {
    if (grid_rows <= 0) return NS_OK;
    const int n_h = p->n_layers - 2;
    if (p->fused_cs < 1 || n_h < 1 || n_h > kFusedMaxHidden) return NS_EINVAL;
    tc::FusedMaps maps;
    for (int l = 1; l <= n_h; ++l) maps.w[l] = p->tmF[l];
    maps.out = ws->tmF_out;
    tc::FusedArgs a{};
    a.theta = ws->theta_full;
    a.P = p->P;
    a.K0 = p->dims[0];
    a.n_h = n_h;
    a.inputs = p->d_inputs;
    a.center = p->d_in_center;
    a.inv_scale = p->d_in_inv_scale;
    a.W0 = (const float*)p->d_W[0];
    a.b0 = (const float*)p->d_b[0];
    for (int l = 1; l <= n_h; ++l) a.bh[l] = (const float*)p->d_b[l];
    a.nrows = ws->d_nrows;
    a.err = ws->d_err;
    switch (p->fused_cs) {
        case 4: return tc::launch_fused_cs<4>(maps, a, grid_rows, st);
        case 8: return tc::launch_fused_cs<8>(maps, a, grid_rows, st);
        default: return NS_ENOTSUP;
    }
}

int launch_gemm_split(const CUtensorMap* tmAhi, const CUtensorMap* tmAlo, const CUtensorMap* tmB, int tile_n,
                      const float* bias, const float* out_mu, float out_sigma, void* C, __nv_bfloat16* C_lo,
                      const __nv_bfloat16* aux_hi, const __nv_bfloat16* aux_lo, const int* d_nrows, int grid_rows,
                      int N, int K, int epi, int* d_err, cudaStream_t st) {
    if (grid_rows <= 0) return NS_OK;
    if (epi < SPL_TANH || epi > SPL_DTANH32) return NS_EINVAL;
    if ((epi == SPL_TANH || epi == SPL_DTANH) && !C_lo) return NS_EINVAL;
    if ((epi == SPL_DTANH || epi == SPL_DTANH32) && (!aux_hi || !aux_lo)) return NS_EINVAL;
    switch (tile_n) {
        case 64: return tc::launch_split_bn<64>(tmAhi, tmAlo, tmB, bias, out_mu, out_sigma, C, C_lo, aux_hi, aux_lo,
                                                d_nrows, grid_rows, N, K, epi, d_err, st);
        case 128: return tc::launch_split_bn<128>(tmAhi, tmAlo, tmB, bias, out_mu, out_sigma, C, C_lo, aux_hi, aux_lo,
                                                  d_nrows, grid_rows, N, K, epi, d_err, st);
        case 256: return tc::launch_split_bn<256>(tmAhi, tmAlo, tmB, bias, out_mu, out_sigma, C, C_lo, aux_hi, aux_lo,
                                                  d_nrows, grid_rows, N, K, epi, d_err, st);
        default: return NS_EINVAL;
    }
}

int gemm_tc_supported(int N, int K) {
    // rows of A and W must be 16-byte aligned for TMA (K multiple of 8 bf16)
    return (K % 8 == 0) && (N % 8 == 0) && K >= 16;
}

static PFN_cuTensorMapEncodeTiled_v12000 get_encode() {
    static PFN_cuTensorMapEncodeTiled_v12000 fn = nullptr;
    if (!fn) {
        void* p = nullptr;
        cudaDriverEntryPointQueryResult q;
        if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &p, 12000, cudaEnableDefault, &q) ==
                cudaSuccess && q == cudaDriverEntryPointSuccess)
            fn = reinterpret_cast<PFN_cuTensorMapEncodeTiled_v12000>(p);
    }
    return fn;
}

int gemm_tc_kps(int K) { return (K % (2 * tc::BK) == 0) ? 2 : 1; }

// bf16 tensor map over a row-major rows x K matrix, 128-byte swizzle.
// kps = 1: 2-D map, box = box_rows x 64.  kps > 1 (K a multiple of 64 kps):
// the 3-D view [K/64][rows][64] (strides: a row K * 2 bytes, a k-block 128
// bytes), box = kps k-blocks of box_rows x 64, landing in shared memory as kps
// consecutive box_rows x 64 tiles.
int make_tensor_map_bf16(CUtensorMap* tm, const void* base, int rows, int K, int box_rows, int kps) {
    auto enc = get_encode();
    if (!enc) return NS_ECUDA;
    if ((reinterpret_cast<uintptr_t>(base) & 15) || (K * 2) % 16) return NS_EINVAL;
    CUresult r;
    if (kps == 1) {
        cuuint64_t dims[2] = {(cuuint64_t)K, (cuuint64_t)rows};
        cuuint64_t strides[1] = {(cuuint64_t)K * 2};
        cuuint32_t box[2] = {(cuuint32_t)tc::BK, (cuuint32_t)box_rows};
        cuuint32_t estr[2] = {1, 1};
        r = enc(tm, CU_TENSOR_MAP_DATA_TYPE_BFLOAT16, 2, const_cast<void*>(base), dims, strides, box, estr,
                CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_128B, CU_TENSOR_MAP_L2_PROMOTION_L2_256B,
                CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
    } else {
        if (kps < 1 || K % (tc::BK * kps)) return NS_EINVAL;
        cuuint64_t dims[3] = {(cuuint64_t)tc::BK, (cuuint64_t)rows, (cuuint64_t)(K / tc::BK)};
        cuuint64_t strides[2] = {(cuuint64_t)K * 2, (cuuint64_t)tc::BK * 2};
        cuuint32_t box[3] = {(cuuint32_t)tc::BK, (cuuint32_t)box_rows, (cuuint32_t)kps};
        cuuint32_t estr[3] = {1, 1, 1};
        r = enc(tm, CU_TENSOR_MAP_DATA_TYPE_BFLOAT16, 3, const_cast<void*>(base), dims, strides, box, estr,
                CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_128B, CU_TENSOR_MAP_L2_PROMOTION_L2_256B,
                CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
    }
    return r == CUDA_SUCCESS ? NS_OK : NS_EINVAL;
}

}  // namespace gpuns
