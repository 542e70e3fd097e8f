// hfs_fno_tc.cuh -- the surrogate's row-streaming GEMMs on the fifth-generation
// tensor cores (tcgen05, sm_100 family): C = op(A) op(B) with the epilogues of
// GemmArgs, for op(A) = A row-major with K in {64, 128} and N in {64, 128},
// the shapes of the pointwise layers and projections (M = batch x grid rows,
// the widths small).
//
// A persistent CTA of 128 threads keeps op(B) (N x K, at most 32 KB) in shared
// memory for the whole launch and streams 128-row tiles of A through a
// two-stage ring of 16-byte asynchronous copies; one thread issues the K / 16
// MMAs of a tile (M = 128, N, K = 16, BF16 operands from shared memory, FP32
// accumulator in one of two tensor-memory buffers) and commits them to that
// buffer's mbarrier, so that tile j + 1's products and tile j + 2's copies
// are in flight while the warps read tile j's accumulator back (tcgen05.ld)
// and apply the epilogue.  Both operands are
// stored K-major without swizzle: core matrices of 8 rows x 16 bytes, the
// core matrices adjacent in K 128 bytes apart (leading byte offset) and the
// 8-row groups K x 16 bytes apart (stride byte offset).  The one wait, for
// the MMAs, is bounded; when it runs out the CTA stops writing results, sets
// the status word, waits once more for its MMAs and frees its tensor memory.
#pragma once

#include "hfs_fno_kernels.cuh"
#include "hfs_tc.cuh"

namespace hfs {
namespace fno {

constexpr int TC_M = 128;

// byte offset of element (row, k) of a K-major BF16 tile of KT columns
template <int KT> __device__ __forceinline__ uint32_t cm_off(int row, int k)
{
    return (uint32_t)((((row >> 3) * (KT / 8) + (k >> 3)) * 64 + (row & 7) * 8 + (k & 7)) * 2);
}

// instruction descriptor, kind::f16: D F32 (bits 4-5 = 1), A and B BF16
// (bits 7-9, 10-12 = 1), both K-major, N >> 3 at bit 17, M >> 4 at bit 24
template <int NT> __host__ __device__ constexpr uint32_t idesc_bf16()
{
    return (1u << 4) | (1u << 7) | (1u << 10) | ((uint32_t)(NT >> 3) << 17) | ((uint32_t)(TC_M >> 4) << 24);
}

__device__ __forceinline__ void mma_bf16_ss(uint32_t d, uint64_t adesc, uint64_t bdesc, uint32_t idesc, bool acc)
{
    asm volatile(
        "{\n.reg .pred p;\nsetp.ne.u32 p, %4, 0;\n"
        "tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n}" ::"r"(d),
        "l"(adesc), "l"(bdesc), "r"(idesc), "r"((uint32_t)acc)
        : "memory");
}

template <int COLS> __device__ __forceinline__ void tmem_alloc(uint32_t *slot)
{
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(tc::smem_addr(slot)),
                 "r"(COLS)
                 : "memory");
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
}
template <int COLS> __device__ __forceinline__ void tmem_dealloc(uint32_t taddr)
{
    asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(taddr), "r"(COLS) : "memory");
}

// The epilogue of GemmArgs for a warp's 32 rows m0 .. m0 + 31 and 32
// columns n0 ..: each thread has read its row's accumulators (tcgen05.ld);
// they pass through a padded shared-memory square (conflict-free both ways)
// so that eight lanes then cover one row's 32 columns with 16-byte accesses
// (four rows per warp instruction, whole 128-byte lines of C, pre and add),
// eight such row groups in flight per lane.
__device__ __forceinline__ void epilogue_warp(const GemmArgs &g, int b, int m0, int n0, const uint32_t (&r)[32],
                                              float *sq)
{
    const int lane = threadIdx.x & 31;
#pragma unroll
    for (int j = 0; j < 32; ++j) sq[lane * 33 + j] = __uint_as_float(r[j]);
    __syncwarp();
    const int rs = lane >> 3, cq = (lane & 7) * 4, n = n0 + cq;
    const float4 bias = g.bias ? *reinterpret_cast<const float4 *>(g.bias + n) : make_float4(0.f, 0.f, 0.f, 0.f);
#pragma unroll
    for (int it = 0; it < 8; ++it) {
        const int i = it * 4 + rs, m = m0 + i;
        if (m >= g.M) continue;
        const float *q = sq + i * 33 + cq;
        float4 v = make_float4(g.alpha * q[0] + bias.x, g.alpha * q[1] + bias.y, g.alpha * q[2] + bias.z,
                               g.alpha * q[3] + bias.w);
        const int64_t oc = (int64_t)b * g.sC + (int64_t)m * g.ldc + n;
        if (g.beta) {
            const float4 c = *reinterpret_cast<const float4 *>(g.C + oc);
            v.x += c.x, v.y += c.y, v.z += c.z, v.w += c.w;
        }
        if (g.add) {
            const float4 c = *reinterpret_cast<const float4 *>(g.add + (int64_t)b * g.sAdd + (int64_t)m * g.ldadd + n);
            v.x += c.x, v.y += c.y, v.z += c.z, v.w += c.w;
        }
        if (g.pre) *reinterpret_cast<float4 *>(g.pre + (int64_t)b * g.sP + (int64_t)m * g.ldp + n) = v;
        if (g.gelu) v = make_float4(gelu_f(v.x), gelu_f(v.y), gelu_f(v.z), gelu_f(v.w));
        if (g.C) *reinterpret_cast<float4 *>(g.C + oc) = v;
        if (g.Cb) {
            __nv_bfloat162 h[2] = {__floats2bfloat162_rn(v.x, v.y), __floats2bfloat162_rn(v.z, v.w)};
            *reinterpret_cast<uint2 *>(g.Cb + (int64_t)b * g.sCb + (int64_t)m * g.ldcb + n) =
                *reinterpret_cast<const uint2 *>(h);
        }
    }
    __syncwarp();
}

constexpr int TC_EPI_BYTES = 4 * 32 * 33 * 4;  // one padded 32 x 32 FP32 square per warp
template <int NT, int KT> constexpr int tc_smem_need() { return NT * KT * 2 + 2 * TC_M * KT * 2 + TC_EPI_BYTES; }
// dynamic shared memory requested per CTA: at least what it uses, and enough
// that no more CTAs share an SM than its 512 tensor-memory columns hold (two
// accumulators of NT columns each)
template <int NT, int KT> constexpr int tc_smem_bytes()
{
    return tc_smem_need<NT, KT>() > 228 * 1024 / (512 / (2 * NT) + 1) ? tc_smem_need<NT, KT>()
                                                                     : 228 * 1024 / (512 / (2 * NT) + 1) + 1024;
}

template <bool TB, int NT, int KT> __global__ void __launch_bounds__(128) gemm_bf16_tc_kernel(const GemmArgs g)
{
    constexpr uint32_t B_BYTES = NT * KT * 2, A_BYTES = TC_M * KT * 2;
    constexpr int COLS = 2 * NT;  // two accumulators: tile j + 1's products while tile j's are read
    extern __shared__ __align__(1024) unsigned char smem[];
    unsigned char *sB = smem;
    unsigned char *sA = smem + B_BYTES;  // two stages
    float *sq = reinterpret_cast<float *>(sA + 2 * A_BYTES) + (threadIdx.x >> 5) * 32 * 33;
    __shared__ __align__(8) uint64_t mbar[2];
    __shared__ uint32_t tmem_slot;
    const int tid = threadIdx.x, warp = tid >> 5;
    const int b = blockIdx.y;
    const bf16 *A = g.A + (int64_t)b * g.sA;
    const bf16 *B = g.B + (int64_t)b * g.sB;
    // op(B) as NT rows of KT (K-major): 16-byte vectors along its contiguous
    // dimension, all loads issued before the first store
    {
        constexpr int BV = NT * KT / 8 / 128;  // vectors per thread
        uint4 x[BV];
#pragma unroll
        for (int q = 0; q < BV; ++q) {
            const int v = tid + 128 * q;
            x[q] = TB ? *reinterpret_cast<const uint4 *>(B + (int64_t)(v / (KT / 8)) * g.ldb + (v % (KT / 8)) * 8)
                      : *reinterpret_cast<const uint4 *>(B + (int64_t)(v / (NT / 8)) * g.ldb + (v % (NT / 8)) * 8);
        }
#pragma unroll
        for (int q = 0; q < BV; ++q) {
            const int v = tid + 128 * q;
            if (TB) {
                *reinterpret_cast<uint4 *>(sB + cm_off<KT>(v / (KT / 8), (v % (KT / 8)) * 8)) = x[q];
            } else {
                const int k = v / (NT / 8), n0 = (v % (NT / 8)) * 8;
                const bf16 *e = reinterpret_cast<const bf16 *>(&x[q]);
#pragma unroll
                for (int i = 0; i < 8; ++i) *reinterpret_cast<bf16 *>(sB + cm_off<KT>(n0 + i, k)) = e[i];
            }
        }
    }
    if (warp == 0) tmem_alloc<COLS>(&tmem_slot);
    if (tid == 0) {
        tc::mbar_init(tc::smem_addr(&mbar[0]));
        tc::mbar_init(tc::smem_addr(&mbar[1]));
    }
    const int ntiles = (g.M + TC_M - 1) / TC_M;
    // this CTA's tiles: blockIdx.x + j gridDim.x, j < cnt (the grid has at most ntiles CTAs)
    const int cnt = (ntiles - (int)blockIdx.x + (int)gridDim.x - 1) / (int)gridDim.x;
    auto load_a = [&](int stage, int j) {
        const int m0 = ((int)blockIdx.x + j * (int)gridDim.x) * TC_M;
        unsigned char *dst = sA + stage * A_BYTES;
#pragma unroll 4
        for (int c = tid; c < TC_M * KT / 8; c += 128) {
            const int r = c / (KT / 8), kc = (c % (KT / 8)) * 8, row = m0 + r;
            const bool ok = row < g.M;
            cp16(reinterpret_cast<bf16 *>(dst + cm_off<KT>(r, kc)), ok ? A + (int64_t)row * g.lda + kc : A, ok);
        }
    };
    load_a(0, 0);
    asm volatile("cp.async.commit_group;" ::: "memory");
    if (cnt > 1) load_a(1, 1);
    asm volatile("cp.async.commit_group;" ::: "memory");
    tc::fence_before_sync();
    __syncthreads();  // the allocation's address and the barriers' initialisation
    tc::fence_after_sync();
    const uint32_t tmem = tmem_slot;
    const uint32_t lane_base = (uint32_t)(warp * 32) << 16;
    // the K / 16 products of tile j (A stage j & 1) into accumulator j & 1, by one thread
    auto issue = [&](int j) {
        tc::fence_after_sync();
        const uint32_t a0 = tc::smem_addr(sA + (j & 1) * A_BYTES), b0 = tc::smem_addr(sB);
        const uint32_t d = tmem + (uint32_t)((j & 1) * NT);
#pragma unroll
        for (int kk = 0; kk < KT / 16; ++kk)
            mma_bf16_ss(d, tc::smem_desc(a0 + 256 * kk, 128, KT * 16), tc::smem_desc(b0 + 256 * kk, 128, KT * 16),
                        idesc_bf16<NT>(), kk > 0);
        tc::commit(tc::smem_addr(&mbar[j & 1]));
    };
    asm volatile("cp.async.wait_group 1;" ::: "memory");
    asm volatile("fence.proxy.async.shared::cta;" ::: "memory");  // copies and B's stores, for the tensor core
    __syncthreads();
    if (tid == 0) issue(0);
    bool ok = true;
    int issued = 1;  // tiles whose products have been issued
    for (int j = 0; j < cnt; ++j) {
        // tile j + 1's products, once its copies have landed
        if (j + 1 < cnt) {
            asm volatile("cp.async.wait_group 0;" ::: "memory");
            asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
            __syncthreads();
            if (tid == 0) issue(j + 1);
            issued = j + 2;
        }
        if (!tc::mbar_wait(tc::smem_addr(&mbar[j & 1]), (uint32_t)(j >> 1) & 1u)) ok = false;
        ok = __all_sync(0xffffffffu, ok);  // the epilogue below is warp-cooperative
        // A stage j & 1 is free: tile j + 2's copies
        if (ok && j + 2 < cnt) load_a(j & 1, j + 2);
        asm volatile("cp.async.commit_group;" ::: "memory");
        tc::fence_after_sync();
        const int m0 = ((int)blockIdx.x + j * (int)gridDim.x) * TC_M + warp * 32;
#pragma unroll
        for (int c0 = 0; c0 < NT; c0 += 32) {
            uint32_t r[32];
            tc::ld32(tmem + lane_base + (uint32_t)((j & 1) * NT + c0), r);
            if (ok && m0 < g.M) epilogue_warp(g, b, m0, c0, r, sq);
        }
        tc::fence_before_sync();
        // accumulator j & 1 read before tile j + 2's products overwrite it; a
        // timed-out wait anywhere ends the CTA's loop
        if (!__syncthreads_and(ok)) {
            // the products still in flight finish before the memory is reused
            for (int q = j; q < issued; ++q) (void)tc::mbar_wait(tc::smem_addr(&mbar[q & 1]), (uint32_t)(q >> 1) & 1u);
            break;
        }
    }
    asm volatile("cp.async.wait_group 0;" ::: "memory");
    if (!ok && tid == 0 && g.status) atomicOr(g.status, 1u);
    tc::fence_before_sync();
    __syncthreads();
    if (warp == 0) tmem_dealloc<COLS>(tmem);
}

// shapes the tensor-core form takes: op(A) row-major, A's and B's pointers,
// leading dimensions and batch strides in 16-byte units, the outputs aligned
// for the epilogue's vector accesses, K and N of 64 or 128, no split-K, and
// rows enough to fill the GPU
inline bool gemm_tc_ok(const GemmArgs &g, bool ta)
{
    auto a16 = [](const void *p) { return ((uintptr_t)p & 15) == 0; };
    if (ta || g.splitk != 1 || g.M < 8192) return false;
    if (!((g.K == 64 || g.K == 128) && (g.N == 64 || g.N == 128))) return false;
    if (!a16(g.A) || g.lda % 8 || g.sA % 8) return false;
    if (!a16(g.B) || g.ldb % 8 || g.sB % 8) return false;
    // the epilogue's 16-byte accesses (8 bytes for the BF16 copy)
    if (g.C && (!a16(g.C) || g.ldc % 4 || g.sC % 4)) return false;
    if (g.pre && (!a16(g.pre) || g.ldp % 4 || g.sP % 4)) return false;
    if (g.add && (!a16(g.add) || g.ldadd % 4 || g.sAdd % 4)) return false;
    if (g.bias && !a16(g.bias)) return false;
    if (g.Cb && (((uintptr_t)g.Cb & 7) || g.ldcb % 4 || g.sCb % 4)) return false;
    return true;
}

}  // namespace fno
}  // namespace hfs
