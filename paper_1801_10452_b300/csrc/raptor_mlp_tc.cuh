// raptor_mlp_tc.cuh -- inference of the surrogate network on the 5th-generation tensor cores
// (tcgen05): BF16 operands in shared memory, FP32 accumulators in tensor memory (TMEM).
//
// The two 256 x 256 hidden layers are the only dense contraction of the rendering path.
// Two persistent kernels, one per hidden layer, each holding its layer's BF16 weight matrix
// (128 KB) resident in shared memory for the whole launch:
//   k_mlp_tc12: layer 1 (4 -> 256, FP32 on the CUDA cores, SiLU) written as the A operand,
//               layer 2 by tcgen05.mma (M = 128 rows, N = 256, K = 16 per instruction),
//               bias + SiLU read back from TMEM, BF16 h2 stored to global memory in the
//               operand layout (one contiguous 64 KB block per 128-row tile);
//   k_mlp_tc34: h2 tile loaded by one bulk copy, layer 3 by tcgen05.mma, bias + SiLU from
//               TMEM, and the 256 -> NOUT output layer in FP32 on the CUDA cores (8 outputs
//               for the state network, 16 for the crossing network).
// The arithmetic is that of the training forward pass (raptor_surrogate.cuh): BF16
// activations and weights, FP32 accumulation, FP32 thin layers, SiLU.
//
// Operand layout (both A = activations [128 rows][256 k] and B = weights [256 n][256 k],
// K-major, no swizzle): 8 x 8 BF16 core matrices of 128 contiguous bytes (8 rows of 16 B);
// core matrices adjacent in k are kTcLbo = 128 B apart, 8-row groups kTcSbo = 4096 B apart.
// One MMA instruction consumes k = 16, i.e. two core matrices along k: its descriptors start
// 256 B further for each k-step.
//
// Each kernel holds two accumulators in TMEM (512 columns; one CTA per SM, which its shared
// memory enforces): while the tensor cores run tile t's MMAs into one, the CUDA cores read
// tile t-1's result out of the other (bias, SiLU, stores), so the MMAs leave the critical
// path.  Every wait on an mbarrier is bounded (kTcWaitNs); a wait that runs out sets *err,
// and the kernel releases its TMEM and returns.
#pragma once

#include <cuda_bf16.h>
#include <stdint.h>

#include "raptor_surrogate.cuh"

namespace raptor {

constexpr int kTcRows = 128;                                  // rows per tile = TMEM lanes
constexpr int kTcThreads = 512;                              // 16 warps: 4 per TMEM lane group
constexpr int kTcQuarters = kTcThreads / kTcRows;            // column quarters (64 columns each)
constexpr uint32_t kTcTileBytes = kTcRows * kHid * 2;         // 64 KB of BF16 activations
constexpr uint32_t kTcWBytes = kHid * kHid * 2;               // 128 KB: one BF16 weight matrix
constexpr uint32_t kTcLbo = 128, kTcSbo = (kHid / 8) * 128;   // core-matrix strides (k, rows)
constexpr uint32_t kTcAcc = 256;                              // TMEM columns of one FP32 256-wide accumulator
constexpr uint32_t kTcCols = 2 * kTcAcc;                      // two accumulators: a tile's MMAs overlap the
                                                              // previous tile's epilogue
constexpr unsigned long long kTcWaitNs = 2000000000ull;       // 2 s

// Byte offset of element (row, k) of a [rows][256] BF16 operand in the layout above.
__host__ __device__ constexpr uint32_t tc_off(int row, int k) {
    return (uint32_t)(row >> 3) * kTcSbo + (uint32_t)(k >> 3) * kTcLbo + (uint32_t)(row & 7) * 16u + (uint32_t)(k & 7) * 2u;
}

// Instruction descriptor of tcgen05.mma kind::f16: FP32 accumulator (bits 4-5 = 1), BF16 A
// and B (bits 7-9, 10-12 = 1), both K-major (bits 15, 16 = 0), N >> 3 in bits 17-22,
// M >> 4 in bits 24-28.
constexpr uint32_t kTcIdesc = (1u << 4) | (1u << 7) | (1u << 10) | ((uint32_t)(256 >> 3) << 17) | ((uint32_t)(128 >> 4) << 24);

struct TcCtl {
    unsigned long long wbar;  // weights landed
    unsigned long long abar;  // activation tile landed (k_mlp_tc34)
    unsigned long long mbar;  // MMAs of a tile complete
    uint32_t tmem;            // TMEM base address written by tcgen05.alloc
    int abort;
};

__device__ __forceinline__ uint32_t tc_smem(const void* p) { return (uint32_t)__cvta_generic_to_shared(p); }

__device__ __forceinline__ unsigned long long tc_now_ns() {
    unsigned long long t;
    asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
    return t;
}

__device__ __forceinline__ void tc_mbar_init(unsigned long long* bar, uint32_t count) {
    asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(tc_smem(bar)), "r"(count) : "memory");
}

__device__ __forceinline__ void tc_mbar_init_fence() { asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory"); }

__device__ __forceinline__ void tc_mbar_expect_tx(unsigned long long* bar, uint32_t bytes) {
    asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(tc_smem(bar)), "r"(bytes) : "memory");
}

__device__ __forceinline__ bool tc_mbar_try(unsigned long long* bar, uint32_t parity) {
    uint32_t ok;
    asm volatile(
        "{\n .reg .pred p;\n mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n selp.u32 %0, 1, 0, p;\n}\n"
        : "=r"(ok)
        : "r"(tc_smem(bar)), "r"(parity)
        : "memory");
    return ok != 0;
}

// Wait for the phase with the given parity to complete; false after kTcWaitNs.
__device__ __forceinline__ bool tc_mbar_wait(unsigned long long* bar, uint32_t parity) {
    if (tc_mbar_try(bar, parity)) return true;
    const unsigned long long t0 = tc_now_ns();
    for (;;) {
        if (tc_mbar_try(bar, parity)) return true;
        if (tc_now_ns() - t0 > kTcWaitNs) return false;
    }
}

// Bulk copy global -> shared (16-byte aligned, size a multiple of 16), completing on `bar`.
__device__ __forceinline__ void tc_bulk_g2s(void* dst, const void* src, uint32_t bytes, unsigned long long* bar) {
    asm volatile("cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];" ::"r"(tc_smem(dst)),
                 "l"(src), "r"(bytes), "r"(tc_smem(bar))
                 : "memory");
}

__device__ __forceinline__ void tc_fence_before() { asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory"); }
__device__ __forceinline__ void tc_fence_after() { asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory"); }
// Thread writes to shared memory made visible to the tensor core (async proxy).
__device__ __forceinline__ void tc_fence_proxy() { asm volatile("fence.proxy.async.shared::cta;" ::: "memory"); }

// Block-wide barrier that also orders tcgen05 operations across it.
__device__ __forceinline__ void tc_sync() {
    tc_fence_before();
    __syncthreads();
    tc_fence_after();
}

// TMEM allocation (one warp, converged).
__device__ __forceinline__ void tc_tmem_alloc(uint32_t* slot, uint32_t cols) {
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(tc_smem(slot)), "r"(cols) : "memory");
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
}
__device__ __forceinline__ void tc_tmem_free(uint32_t taddr, uint32_t cols) {
    asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(taddr), "r"(cols) : "memory");
}

// Shared-memory matrix descriptor: start address, leading (k) and stride (row-group) byte
// offsets, each >> 4; bits 46-48 = 0b001; base offset 0; no swizzle.
__device__ __forceinline__ uint64_t tc_desc(uint32_t saddr, uint32_t lbo, uint32_t sbo) {
    return (uint64_t)((saddr & 0x3FFFFu) >> 4) | ((uint64_t)((lbo & 0x3FFFFu) >> 4) << 16) |
           ((uint64_t)((sbo & 0x3FFFFu) >> 4) << 32) | (1ull << 46);
}

// D[tmem] (+)= A[smem] B[smem]^T for one k-step; issued by one thread.
__device__ __forceinline__ void tc_mma(uint32_t d_tmem, uint64_t adesc, uint64_t bdesc, uint32_t idesc, uint32_t accumulate) {
    asm volatile(
        "{\n .reg .pred p;\n setp.ne.b32 p, %4, 0;\n tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n}\n" ::"r"(d_tmem),
        "l"(adesc), "l"(bdesc), "r"(idesc), "r"(accumulate)
        : "memory");
}

// Arrive on `bar` once every MMA issued so far by this thread has completed.
__device__ __forceinline__ void tc_commit(unsigned long long* bar) {
    asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(tc_smem(bar)) : "memory");
}

// 32 consecutive FP32 columns of this thread's TMEM lane (warp w reads lanes 32 (w % 4) ..;
// warps w, w + 4, w + 8, w + 12 share those lanes and split the columns in quarters).
__device__ __forceinline__ void tc_ld32(uint32_t taddr, uint32_t v[32]) {
    asm volatile(
        "tcgen05.ld.sync.aligned.32x32b.x32.b32 {%0,%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,%14,%15,%16,%17,%18,%19,%20,%21,"
        "%22,%23,%24,%25,%26,%27,%28,%29,%30,%31}, [%32];"
        : "=r"(v[0]), "=r"(v[1]), "=r"(v[2]), "=r"(v[3]), "=r"(v[4]), "=r"(v[5]), "=r"(v[6]), "=r"(v[7]), "=r"(v[8]), "=r"(v[9]),
          "=r"(v[10]), "=r"(v[11]), "=r"(v[12]), "=r"(v[13]), "=r"(v[14]), "=r"(v[15]), "=r"(v[16]), "=r"(v[17]), "=r"(v[18]),
          "=r"(v[19]), "=r"(v[20]), "=r"(v[21]), "=r"(v[22]), "=r"(v[23]), "=r"(v[24]), "=r"(v[25]), "=r"(v[26]), "=r"(v[27]),
          "=r"(v[28]), "=r"(v[29]), "=r"(v[30]), "=r"(v[31])
        : "r"(taddr));
    asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
}

__device__ __forceinline__ uint32_t tc_pack_bf16(float lo, float hi) {
    const __nv_bfloat162 h = __floats2bfloat162_rn(lo, hi);
    return *reinterpret_cast<const uint32_t*>(&h);
}

// Issue the 16 k-steps of one 128 x 256 x 256 layer and commit them to `bar`.
__device__ __forceinline__ void tc_issue_layer(uint32_t tmem, const uint8_t* sA, const uint8_t* sW, unsigned long long* bar) {
    const uint32_t a0 = tc_smem(sA), b0 = tc_smem(sW);
#pragma unroll 1
    for (int s = 0; s < kHid / 16; ++s)
        tc_mma(tmem, tc_desc(a0 + 256u * s, kTcLbo, kTcSbo), tc_desc(b0 + 256u * s, kTcLbo, kTcSbo), kTcIdesc, s > 0 ? 1u : 0u);
    tc_commit(bar);
}

// Weights of layers 2 and 3 in the operand layout: wu[l][tc_off(n, k) / 2] = bf16(W[n][k]).
__global__ void k_tc_pack(const float* __restrict__ P, __nv_bfloat16* __restrict__ wu) {
    for (int e = blockIdx.x * blockDim.x + threadIdx.x; e < 2 * kHid * kHid; e += gridDim.x * blockDim.x) {
        const int l = e / (kHid * kHid), r = e - l * kHid * kHid;
        const int nn = r / kHid, k = r - nn * kHid;
        const float w = P[(l == 0 ? MlpLayout::W2 : MlpLayout::W3) + r];
        wu[(size_t)l * kHid * kHid + tc_off(nn, k) / 2] = __float2bfloat16(w);
    }
}

// Shared-memory plan of the two kernels (after aligning the dynamic base to 1024 B).
// Output layer of NOUT outputs: its FP32 weights and biases, and the partial sums of the
// four column quarters for 8 outputs at a time ([4][128][8]; NOUT / 8 rounds).
constexpr uint32_t kTc12Params = (kHid * kIn + 2 * kHid + 8) * 4;          // w1, b1, b2, norm
template <int NOUT>
constexpr uint32_t tc34_params() { return (kHid + NOUT * kHid + NOUT + kTcQuarters * kTcRows * 8) * 4; }
constexpr uint32_t kTc34Params = tc34_params<kOut>();  // b3, w4, b4, partial sums
constexpr uint32_t kTc12Smem = 1024 + kTcWBytes + kTcTileBytes + kTc12Params + sizeof(TcCtl);
template <int NOUT>
constexpr uint32_t tc34_smem() { return 1024 + kTcWBytes + kTcTileBytes + tc34_params<NOUT>() + sizeof(TcCtl); }
constexpr uint32_t kTc34Smem = tc34_smem<kOut>();
static_assert(tc34_smem<16>() <= 232448, "the 16-output plan fits in one CTA's shared memory");

__device__ __forceinline__ uint8_t* tc_align(uint8_t* p) {
    return reinterpret_cast<uint8_t*>((reinterpret_cast<uintptr_t>(p) + 1023) & ~uintptr_t(1023));
}

// Common prologue: TMEM allocation by warp 0, barrier initialisation by thread 0.
__device__ __forceinline__ void tc_prologue(TcCtl* ctl) {
    if ((threadIdx.x >> 5) == 0) tc_tmem_alloc(&ctl->tmem, kTcCols);
    if (threadIdx.x == 0) {
        tc_mbar_init(&ctl->wbar, 1);
        tc_mbar_init(&ctl->abar, 1);
        tc_mbar_init(&ctl->mbar, 1);
        ctl->abort = 0;
        tc_mbar_init_fence();
    }
}

// Common epilogue: every bulk copy into this CTA's shared memory has landed and the MMAs
// last issued have completed (bounded waits; they are outstanding only after an aborted
// loop), then TMEM is released.
__device__ __forceinline__ void tc_teardown(TcCtl* ctl, bool w_pending, bool m_out, uint32_t m_phase, int* err) {
    if (threadIdx.x == 0 && w_pending && !tc_mbar_wait(&ctl->wbar, 0)) ctl->abort = 1;
    if (threadIdx.x == 0 && m_out && !tc_mbar_wait(&ctl->mbar, m_phase)) ctl->abort = 1;
    tc_sync();
    if ((threadIdx.x >> 5) == 0) tc_tmem_free(ctl->tmem, kTcCols);
    if (threadIdx.x == 0 && ctl->abort) atomicExch(err, 1);
}

// Layers 1 and 2.  x: [n][4] raw inputs; h2: [tiles][64 KB] in the operand layout.
template <int NOUT = kOut>
__global__ void __launch_bounds__(kTcThreads, 1) k_mlp_tc12(const float* __restrict__ P, const __nv_bfloat16* __restrict__ wu2,
                                                            const float* __restrict__ x, long long n,
                                                            __nv_bfloat16* __restrict__ h2, int* __restrict__ err) {
    extern __shared__ uint8_t tc_smem_raw[];
    uint8_t* sW = tc_align(tc_smem_raw);
    uint8_t* sA = sW + kTcWBytes;
    float* sw1 = reinterpret_cast<float*>(sA + kTcTileBytes);
    float* sb1 = sw1 + kHid * kIn;
    float* sb2 = sb1 + kHid;
    float* snorm = sb2 + kHid;
    TcCtl* ctl = reinterpret_cast<TcCtl*>(snorm + 8);
    const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
    const long long n_tiles = (n + kTcRows - 1) / kTcRows;

    tc_prologue(ctl);
    for (int i = tid; i < kHid * kIn; i += kTcThreads) sw1[i] = P[MlpLayout::W1 + i];
    for (int i = tid; i < kHid; i += kTcThreads) {
        sb1[i] = P[MlpLayout::B1 + i];
        sb2[i] = P[MlpLayout::B2 + i];
    }
    if (tid < 8) snorm[tid] = P[MlpLayoutT<NOUT>::NORM + tid];
    tc_sync();
    const uint32_t tmem = ctl->tmem;
    if (tid == 0) {
        tc_mbar_expect_tx(&ctl->wbar, kTcWBytes);
        for (int c = 0; c < 8; ++c) tc_bulk_g2s(sW + c * (kTcWBytes / 8), reinterpret_cast<const uint8_t*>(wu2) + c * (kTcWBytes / 8), kTcWBytes / 8, &ctl->wbar);
    }
    bool w_pending = true;
    uint32_t mphase = 0;
    bool m_out = false;   // thread 0: MMAs issued whose completion no wait has seen yet,
    uint32_t m_phase = 0;  // and the barrier phase their commit completes
    const int row = tid & (kTcRows - 1), quarter = tid >> 7;   // layer 1: (row, column quarter)
    const int er = 32 * (warp & 3) + lane, c0 = 64 * quarter;  // epilogue: TMEM lane, columns
    // Iteration k: wait for tile k-1's MMAs (they have read the A tile), layer 1 of tile k into
    // the A tile, tile k's MMAs into accumulator k % 2, then tile k-1's epilogue from the other
    // accumulator while those MMAs run.  The loop runs one extra iteration for the last
    // epilogue.
    long long prev = -1;  // the tile whose MMAs the previous iteration issued
    uint32_t buf = 0;     // accumulator of this iteration's tile
    // raw inputs of this thread's row in the next tile, loaded a tile ahead (their latency
    // hides behind the epilogue)
    float xr[kIn];
    auto load_inputs = [&](long long tt) {
        const long long m = tt * kTcRows + row;
#pragma unroll
        for (int c = 0; c < kIn; ++c) xr[c] = (tt < n_tiles && m < n) ? x[m * kIn + c] : 0.f;
    };
    load_inputs(blockIdx.x);
    for (long long t = blockIdx.x;; t += gridDim.x) {
        const bool have = t < n_tiles;
        if (prev >= 0) {
            if (tc_mbar_wait(&ctl->mbar, mphase)) m_out = false;
            else ctl->abort = 1;
            mphase ^= 1u;
            __syncthreads();
            if (ctl->abort) break;
            tc_fence_after();
        }
        if (have) {
            // layer 1 (FP32): z1 = W1 x_n + b1, h1 = silu(z1) as BF16 into the A operand
            const long long m = t * kTcRows + row;
            float xn[kIn];
#pragma unroll
            for (int c = 0; c < kIn; ++c) xn[c] = m < n ? (xr[c] - snorm[4 + c]) * snorm[c] : 0.f;
#pragma unroll 2
            for (int j0 = quarter * 64; j0 < quarter * 64 + 64; j0 += 8) {
                uint32_t pk[4];
#pragma unroll
                for (int u = 0; u < 4; ++u) {
                    float z[2];
#pragma unroll
                    for (int q = 0; q < 2; ++q) {
                        const int j = j0 + 2 * u + q;
                        float acc = sb1[j];
#pragma unroll
                        for (int c = 0; c < kIn; ++c) acc += sw1[j * kIn + c] * xn[c];
                        z[q] = silu(acc);
                    }
                    pk[u] = tc_pack_bf16(z[0], z[1]);
                }
                *reinterpret_cast<uint4*>(sA + tc_off(row, j0)) = make_uint4(pk[0], pk[1], pk[2], pk[3]);
            }
            tc_fence_proxy();
            tc_sync();
            // layer 2 on the tensor cores
            if (tid == 0) {
                if (w_pending) {
                    if (tc_mbar_wait(&ctl->wbar, 0)) w_pending = false;
                    else ctl->abort = 1;
                }
                if (!ctl->abort) {
                    tc_issue_layer(tmem + kTcAcc * buf, sA, sW, &ctl->mbar);
                    m_out = true;
                    m_phase = mphase;
                }
            }
            load_inputs(t + gridDim.x);
            __syncthreads();
            if (ctl->abort) break;
        }
        if (prev >= 0) {
            // bias + SiLU of tile prev from the other accumulator -> BF16 h2 in the operand layout
            uint8_t* dst = reinterpret_cast<uint8_t*>(h2) + (size_t)prev * kTcTileBytes;
            const uint32_t acc = tmem + kTcAcc * (buf ^ 1u) + ((uint32_t)(32 * (warp & 3)) << 16);
#pragma unroll 1
            for (int cc = 0; cc < 2; ++cc) {
                uint32_t v[32];
                tc_ld32(acc + (uint32_t)(c0 + 32 * cc), v);
#pragma unroll
                for (int u = 0; u < 4; ++u) {
                    uint32_t pk[4];
#pragma unroll
                    for (int q = 0; q < 4; ++q) {
                        const int col = c0 + 32 * cc + 8 * u + 2 * q;
                        pk[q] = tc_pack_bf16(silu(__uint_as_float(v[8 * u + 2 * q]) + sb2[col]),
                                             silu(__uint_as_float(v[8 * u + 2 * q + 1]) + sb2[col + 1]));
                    }
                    *reinterpret_cast<uint4*>(dst + tc_off(er, c0 + 32 * cc + 8 * u)) = make_uint4(pk[0], pk[1], pk[2], pk[3]);
                }
            }
            // every read of this accumulator is done before the MMAs two tiles on overwrite it
            tc_sync();
        }
        if (!have) break;
        prev = t;
        buf ^= 1u;
    }
    tc_teardown(ctl, w_pending, m_out, m_phase, err);
}

// Layers 3 and 4.  h2 as written by k_mlp_tc12; out: [n][NOUT] normalised outputs.
template <int NOUT>
__device__ __forceinline__ void mlp_tc34_body(const float* __restrict__ P, const __nv_bfloat16* __restrict__ wu3,
                                              const __nv_bfloat16* __restrict__ h2, long long n, float* __restrict__ out,
                                              int* __restrict__ err) {
    extern __shared__ uint8_t tc_smem_raw[];
    uint8_t* sW = tc_align(tc_smem_raw);
    uint8_t* sA = sW + kTcWBytes;
    float* sb3 = reinterpret_cast<float*>(sA + kTcTileBytes);
    float* sw4 = sb3 + kHid;
    float* sb4 = sw4 + NOUT * kHid;
    float* sred = sb4 + NOUT;   // [4][128][8] partial sums of the column quarters, 8 outputs a round
    TcCtl* ctl = reinterpret_cast<TcCtl*>(sred + kTcQuarters * kTcRows * 8);
    static_assert(NOUT % 8 == 0, "outputs are reduced 8 at a time");
    const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
    const long long n_tiles = (n + kTcRows - 1) / kTcRows;

    tc_prologue(ctl);
    for (int i = tid; i < kHid; i += kTcThreads) sb3[i] = P[MlpLayoutT<NOUT>::B3 + i];
    for (int i = tid; i < NOUT * kHid; i += kTcThreads) sw4[i] = P[MlpLayoutT<NOUT>::W4 + i];
    if (tid < NOUT) sb4[tid] = P[MlpLayoutT<NOUT>::B4 + tid];
    tc_sync();
    const uint32_t tmem = ctl->tmem;
    if (tid == 0) {
        tc_mbar_expect_tx(&ctl->wbar, kTcWBytes);
        for (int c = 0; c < 8; ++c) tc_bulk_g2s(sW + c * (kTcWBytes / 8), reinterpret_cast<const uint8_t*>(wu3) + c * (kTcWBytes / 8), kTcWBytes / 8, &ctl->wbar);
        if (blockIdx.x < n_tiles) {
            tc_mbar_expect_tx(&ctl->abar, kTcTileBytes);
            tc_bulk_g2s(sA, reinterpret_cast<const uint8_t*>(h2) + (size_t)blockIdx.x * kTcTileBytes, kTcTileBytes, &ctl->abar);
        }
    }
    bool w_pending = true, a_pending = blockIdx.x < n_tiles;
    uint32_t mphase = 0, aphase = 0;
    bool m_out = false;    // thread 0: MMAs issued whose completion no wait has seen yet,
    uint32_t m_phase = 0;  // and the barrier phase their commit completes
    const int er = 32 * (warp & 3) + lane, quarter = warp >> 2, c0 = 64 * quarter;
    // Tile t's MMAs write accumulator buf; the next tile's activations are fetched as soon as
    // they have read the A tile, and its MMAs (into the other accumulator) are issued once the
    // copy has landed, before this tile's cross-quarter reduction: they run while this tile's
    // epilogue finishes and the next one starts.  The first tile's MMAs are issued here.
    uint32_t buf = 0;
    for (long long t = blockIdx.x; t < n_tiles; t += gridDim.x) {
        const bool has_next = t + gridDim.x < n_tiles;
        if (tid == 0 && t == blockIdx.x) {
            if (w_pending) {
                if (tc_mbar_wait(&ctl->wbar, 0)) w_pending = false;
                else ctl->abort = 1;
            }
            if (!ctl->abort) {
                if (tc_mbar_wait(&ctl->abar, aphase)) {
                    a_pending = false;
                    aphase ^= 1u;
                } else {
                    ctl->abort = 1;
                }
            }
            if (!ctl->abort) {
                tc_fence_after();
                tc_issue_layer(tmem + kTcAcc * buf, sA, sW, &ctl->mbar);
                m_out = true;
                m_phase = mphase;
            }
        }
        __syncthreads();
        if (ctl->abort) break;
        if (tc_mbar_wait(&ctl->mbar, mphase)) m_out = false;
        else ctl->abort = 1;
        mphase ^= 1u;
        __syncthreads();
        if (ctl->abort) break;
        tc_fence_after();
        // the MMAs have read the tile: fetch the next one while this one's epilogue runs
        if (tid == 0 && has_next) {
            tc_mbar_expect_tx(&ctl->abar, kTcTileBytes);
            tc_bulk_g2s(sA, reinterpret_cast<const uint8_t*>(h2) + (size_t)(t + gridDim.x) * kTcTileBytes, kTcTileBytes, &ctl->abar);
            a_pending = true;
        }
        // bias + SiLU (rounded to BF16 as in training), then the FP32 output layer
        float acc[NOUT];
#pragma unroll
        for (int o = 0; o < NOUT; ++o) acc[o] = 0.f;
#pragma unroll 1
        for (int cc = 0; cc < 2; ++cc) {
            uint32_t v[32];
            tc_ld32(tmem + kTcAcc * buf + ((uint32_t)(32 * (warp & 3)) << 16) + (uint32_t)(c0 + 32 * cc), v);
#pragma unroll
            for (int q = 0; q < 32; ++q) {
                const int col = c0 + 32 * cc + q;
                const float h = __bfloat162float(__float2bfloat16(silu(__uint_as_float(v[q]) + sb3[col])));
#pragma unroll
                for (int o = 0; o < NOUT; ++o) acc[o] += sw4[o * kHid + col] * h;
            }
        }
        // the next tile's MMAs into the other accumulator (its last reads ended with the
        // previous tile's reduction barriers)
        if (tid == 0 && has_next && !ctl->abort) {
            if (tc_mbar_wait(&ctl->abar, aphase)) {
                a_pending = false;
                aphase ^= 1u;
                tc_fence_after();
                tc_issue_layer(tmem + kTcAcc * (buf ^ 1u), sA, sW, &ctl->mbar);
                m_out = true;
                m_phase = mphase;
            } else {
                ctl->abort = 1;
            }
        }
        // the row's sum over the four quarters, 8 outputs a round: every quarter writes its
        // partial sums, then each thread adds up two of the 8 outputs (quarter order 0-3) and
        // stores them with their biases
#pragma unroll
        for (int g = 0; g < NOUT; g += 8) {
            float4* w4 = reinterpret_cast<float4*>(sred + (quarter * kTcRows + er) * 8);
            w4[0] = make_float4(acc[g + 0], acc[g + 1], acc[g + 2], acc[g + 3]);
            w4[1] = make_float4(acc[g + 4], acc[g + 5], acc[g + 6], acc[g + 7]);
            tc_sync();
            const long long m = t * kTcRows + er;
            if (m < n) {
                const int o = 2 * quarter;
                float2 r = *reinterpret_cast<const float2*>(sred + er * 8 + o);
#pragma unroll
                for (int qq = 1; qq < kTcQuarters; ++qq) {
                    const float2 pq = *reinterpret_cast<const float2*>(sred + (qq * kTcRows + er) * 8 + o);
                    r.x += pq.x;
                    r.y += pq.y;
                }
                *reinterpret_cast<float2*>(out + m * NOUT + g + o) = make_float2(r.x + sb4[g + o], r.y + sb4[g + o + 1]);
            }
            tc_sync();
        }
        buf ^= 1u;
    }
    // an activation copy issued for a tile this CTA will not process cannot exist (the next
    // tile is fetched only if it is processed), but an aborted loop may leave one in flight
    if (tid == 0 && a_pending && !tc_mbar_wait(&ctl->abar, aphase)) ctl->abort = 1;
    tc_teardown(ctl, w_pending, m_out, m_phase, err);
}

template <int NOUT = kOut>
__global__ void __launch_bounds__(kTcThreads, 1) k_mlp_tc34(const float* __restrict__ P, const __nv_bfloat16* __restrict__ wu3,
                                                            const __nv_bfloat16* __restrict__ h2, long long n,
                                                            float* __restrict__ out, int* __restrict__ err) {
    mlp_tc34_body<NOUT>(P, wu3, h2, n, out, err);
}

// The state network's layers 3-4 (k_mlp_tc34_state; the crossing network's 16 outputs use
// k_mlp_tc34<16>) run beside the near-critical rays' FP32 kernel (one
// 128-thread block of 104 registers on most SMs while the network runs): capped at 96
// registers a thread (512 x 96 + 128 x 104 fit the SM's 64 K) a CTA shares the SM with that
// block instead of waiting for it to finish, at the price of a few spills.
__global__ void __maxnreg__(96) k_mlp_tc34_state(const float* __restrict__ P, const __nv_bfloat16* __restrict__ wu3,
                                                 const __nv_bfloat16* __restrict__ h2, long long n, float* __restrict__ out,
                                                 int* __restrict__ err) {
    mlp_tc34_body<kOut>(P, wu3, h2, n, out, err);
}

}  // namespace raptor
