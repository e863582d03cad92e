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
