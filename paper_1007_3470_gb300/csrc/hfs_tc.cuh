// hfs_tc.cuh -- a length-16 DFT on the fifth-generation tensor cores
// (tcgen05, sm_100 family), for the first radix-16 pass of the 3D z-pass
// (the transform F_N of Eq. GP1ODE_T along z).
//
// A CTA of 256 threads, each holding the 16 complex inputs of one radix-16
// butterfly in registers, computes all 256 butterflies as one real matrix
// product  D (256 x 32) = A (256 x 32) . W^T (32 x 32):  row m of A is thread
// m's 16 inputs as interleaved (re, im) reals, W is the real form of the
// complex 16 x 16 DFT matrix, row m of D the 16 outputs.  Precision: FP32
// operands split as x = hi + lo with hi, lo TF32 (cvt.rna), three products
// hi.hi + hi.lo + lo.hi accumulated in FP32 by the tensor core (3xTF32).
//
// Data path: each thread writes its row of A_hi and A_lo straight into
// tensor memory (tcgen05.st, its own lane), one elected thread issues the
// MMAs (A from tensor memory, W from shared memory through a matrix
// descriptor), tcgen05.commit arrives on an mbarrier, and each thread reads
// its row of D back (tcgen05.ld).  Tensor-memory lanes: warp w of the CTA
// accesses lanes 32 (w mod 4) .. + 31, so rows 0..127 (warps 0-3) and
// 128..255 (warps 4-7) are two M = 128 blocks kept in separate columns.
//
// Columns of the allocation (256): A_hi [0, 64), A_lo [64, 128), the hi.hi
// products D [128, 192) and the cross terms hi.lo + lo.hi X [192, 256);
// block b of each at +32 b; the thread adds its rows of X and D in FP32.  W is stored K-major without swizzle: core
// matrices of 8 rows x 16 bytes, adjacent K chunks 128 bytes apart (leading
// byte offset), adjacent 8-row groups 1024 bytes apart (stride byte offset).
#pragma once

#include "hfs_internal.cuh"

namespace hfs {
namespace tc {

constexpr uint32_t kCols = 256;
constexpr uint32_t kColAhi = 0, kColAlo = 64, kColD = 128, kColX = 192;
constexpr uint32_t kWBytes = 32 * 32 * 4;  // one 32 x 32 TF32 matrix
// bounded waits: try_wait returns after a hardware time slice, so this is
// far beyond any MMA batch
constexpr int kWaitLimit = 1 << 22;

__device__ __forceinline__ uint32_t smem_addr(const void *p) { return (uint32_t)__cvta_generic_to_shared(p); }

__device__ __forceinline__ uint32_t to_tf32(float x)
{
    uint32_t r;
    asm("cvt.rna.tf32.f32 %0, %1;" : "=r"(r) : "f"(x));
    return r;
}

// shared-memory matrix descriptor: start address, leading / stride byte
// offsets (16-byte units), descriptor version 1 (bits 46-48), no swizzle
__device__ __forceinline__ uint64_t smem_desc(uint32_t addr, uint32_t lbo, uint32_t sbo)
{
    return (uint64_t)((addr & 0x3FFFFu) >> 4) | ((uint64_t)(lbo >> 4) << 16) | ((uint64_t)(sbo >> 4) << 32) |
           (1ull << 46);
}

// instruction descriptor, kind::tf32: D F32 (bits 4-5 = 1), A and B TF32
// (bits 7-9, 10-12 = 2), both K-major, N >> 3 at bit 17, M >> 4 at bit 24
__host__ __device__ constexpr uint32_t idesc_tf32(int M, int N)
{
    return (1u << 4) | (2u << 7) | (2u << 10) | ((uint32_t)(N >> 3) << 17) | ((uint32_t)(M >> 4) << 24);
}

// byte offset of element (row, k) of a K-major 32 x 32 TF32 matrix in the
// layout above
__host__ __device__ constexpr uint32_t w_offset(int row, int k)
{
    return (uint32_t)((row >> 3) * 1024 + (k >> 2) * 128 + (row & 7) * 16 + (k & 3) * 4);
}

__device__ __forceinline__ void fence_before_sync() { asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory"); }
__device__ __forceinline__ void fence_after_sync() { asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory"); }

// whole warp: allocate kCols columns, address written to *slot
__device__ __forceinline__ void alloc(uint32_t *slot)
{
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(smem_addr(slot)),
                 "r"(kCols)
                 : "memory");
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
}
__device__ __forceinline__ void dealloc(uint32_t taddr)
{
    asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(taddr), "r"(kCols) : "memory");
}

__device__ __forceinline__ void st32(uint32_t taddr, const uint32_t (&r)[32])
{
    asm volatile(
        "tcgen05.st.sync.aligned.32x32b.x32.b32 [%0], {%1, %2, %3, %4, %5, %6, %7, %8, %9, %10, %11, %12, %13, %14, "
        "%15, %16, %17, %18, %19, %20, %21, %22, %23, %24, %25, %26, %27, %28, %29, %30, %31, %32};" ::"r"(taddr),
        "r"(r[0]), "r"(r[1]), "r"(r[2]), "r"(r[3]), "r"(r[4]), "r"(r[5]), "r"(r[6]), "r"(r[7]), "r"(r[8]),
        "r"(r[9]), "r"(r[10]), "r"(r[11]), "r"(r[12]), "r"(r[13]), "r"(r[14]), "r"(r[15]), "r"(r[16]), "r"(r[17]),
        "r"(r[18]), "r"(r[19]), "r"(r[20]), "r"(r[21]), "r"(r[22]), "r"(r[23]), "r"(r[24]), "r"(r[25]), "r"(r[26]),
        "r"(r[27]), "r"(r[28]), "r"(r[29]), "r"(r[30]), "r"(r[31])
        : "memory");
}

__device__ __forceinline__ void ld32(uint32_t taddr, uint32_t (&r)[32])
{
    asm volatile(
        "tcgen05.ld.sync.aligned.32x32b.x32.b32 {%0, %1, %2, %3, %4, %5, %6, %7, %8, %9, %10, %11, %12, %13, %14, "
        "%15, %16, %17, %18, %19, %20, %21, %22, %23, %24, %25, %26, %27, %28, %29, %30, %31}, [%32];"
        : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]), "=r"(r[7]),
          "=r"(r[8]), "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]), "=r"(r[13]), "=r"(r[14]), "=r"(r[15]),
          "=r"(r[16]), "=r"(r[17]), "=r"(r[18]), "=r"(r[19]), "=r"(r[20]), "=r"(r[21]), "=r"(r[22]), "=r"(r[23]),
          "=r"(r[24]), "=r"(r[25]), "=r"(r[26]), "=r"(r[27]), "=r"(r[28]), "=r"(r[29]), "=r"(r[30]), "=r"(r[31])
        : "r"(taddr)
        : "memory");
    asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
}

// D[taddr_d] (+)= A[taddr_a] . B[desc]  (M = 128, N = 32, K = 8, TF32)
__device__ __forceinline__ void mma_tf32(uint32_t d, uint32_t a, uint64_t bdesc, bool accumulate)
{
    asm volatile(
        "{\n.reg .pred p;\nsetp.ne.u32 p, %4, 0;\n"
        "tcgen05.mma.cta_group::1.kind::tf32 [%0], [%1], %2, %3, p;\n}" ::"r"(d),
        "r"(a), "l"(bdesc), "r"(idesc_tf32(128, 32)), "r"((uint32_t)accumulate)
        : "memory");
}

__device__ __forceinline__ void commit(uint32_t mbar)
{
    asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(mbar)
                 : "memory");
}

__device__ __forceinline__ void mbar_init(uint32_t mbar)
{
    asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(mbar) : "memory");
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
}

// bounded wait for the phase with the given parity; false when it ran out
__device__ __forceinline__ bool mbar_wait(uint32_t mbar, uint32_t parity)
{
    for (int it = 0; it < kWaitLimit; ++it) {
        uint32_t done;
        asm volatile(
            "{\n.reg .pred p;\nmbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\nselp.u32 %0, 1, 0, p;\n}"
            : "=r"(done)
            : "r"(mbar), "r"(parity)
            : "memory");
        if (done) return true;
    }
    return false;
}

// State of the tensor-core DFT inside one CTA.
struct Dft16 {
    uint32_t tmem;     // allocation base (lane 0, column 0)
    uint32_t whi, wlo; // shared addresses of W_hi, W_lo
    uint32_t mbar;     // shared address of the completion barrier
    uint32_t phase;    // parity of the next completion
};

// cos(q pi / 8) for any integer q >= 0
__device__ __forceinline__ double cos_pi8(int q)
{
    constexpr double c1 = 0.92387953251128675613, c2 = 0.70710678118654752440, c3 = 0.38268343236508977173;
    const int r = q & 15;
    const int m = r > 8 ? 16 - r : r;  // cos is even: fold to 0..8
    const double v = m == 0 ? 1.0 : m == 1 ? c1 : m == 2 ? c2 : m == 3 ? c3 : 0.0;
    const double w = m == 8 ? 1.0 : m == 7 ? c1 : m == 6 ? c2 : m == 5 ? c3 : 0.0;
    return m <= 4 ? v : -w;
}

// Fill W (forward DFT-16 in real form, K-major) as hi + lo TF32 parts; all
// threads of the CTA, before the first dft16 (followed by a CTA barrier).
__device__ __forceinline__ void fill_w(unsigned char *whi, unsigned char *wlo)
{
    for (int i = threadIdx.x; i < 32 * 32; i += blockDim.x) {
        const int n = i >> 5, k = i & 31;  // W row n (output real), column k (input real)
        const int ko = n >> 1, ki = k >> 1;
        // cos and sin of q pi / 8 from the five distinct magnitudes (no FP64
        // sine per entry: the table is rebuilt by every CTA)
        const int q = (ko * ki) & 15;
        const double cs = cos_pi8(q), sn = cos_pi8(q + 12);
        // Re X = sum (ar cos + ai sin), Im X = sum (-ar sin + ai cos)
        const double w = (n & 1) == 0 ? ((k & 1) == 0 ? cs : sn) : ((k & 1) == 0 ? -sn : cs);
        const uint32_t hi = to_tf32((float)w);
        const uint32_t lo = to_tf32((float)(w - (double)__uint_as_float(hi)));
        *reinterpret_cast<uint32_t *>(whi + w_offset(n, k)) = hi;
        *reinterpret_cast<uint32_t *>(wlo + w_offset(n, k)) = lo;
    }
    // generic-proxy writes read later by the tensor core (async proxy)
    asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
}

// In-place DFT of the thread's 16 values: X_k = sum_r a_r exp(-+2 pi i r k / 16)
// (INV: +, through conj(DFT(conj a))).  Every thread of the 256-thread CTA
// calls it together.  Returns false when the completion wait ran out (the
// caller records the error; the values are then unspecified).
template <bool INV> __device__ __forceinline__ bool dft16(cpx<float> (&a)[16], Dft16 &s)
{
    const int warp = threadIdx.x >> 5;
    const uint32_t lane_base = (uint32_t)((warp & 3) * 32) << 16;
    const uint32_t blk = (uint32_t)(warp >> 2) * 32;  // column offset of this thread's M block
    {
        uint32_t hi[32], lo[32];
#pragma unroll
        for (int r = 0; r < 16; ++r) {
            const float x = a[r].x, y = INV ? -a[r].y : a[r].y;
            hi[2 * r] = to_tf32(x);
            hi[2 * r + 1] = to_tf32(y);
            lo[2 * r] = to_tf32(x - __uint_as_float(hi[2 * r]));
            lo[2 * r + 1] = to_tf32(y - __uint_as_float(hi[2 * r + 1]));
        }
        st32(s.tmem + lane_base + kColAhi + blk, hi);
        st32(s.tmem + lane_base + kColAlo + blk, lo);
        asm volatile("tcgen05.wait::st.sync.aligned;" ::: "memory");
    }
    fence_before_sync();
    __syncthreads();
    if (threadIdx.x == 0) {
        fence_after_sync();
        // four independent accumulator chains (block b x {hi.hi, cross terms}),
        // interleaved so that consecutive MMAs do not wait on one another
#pragma unroll
        for (int k = 0; k < 4; ++k) {
#pragma unroll
            for (int b = 0; b < 2; ++b) {
                const uint32_t ahi = s.tmem + kColAhi + 32 * b + 8 * k, alo = s.tmem + kColAlo + 32 * b + 8 * k;
                mma_tf32(s.tmem + kColD + 32 * b, ahi, smem_desc(s.whi + 256 * k, 128, 1024), k > 0);
                mma_tf32(s.tmem + kColX + 32 * b, alo, smem_desc(s.whi + 256 * k, 128, 1024), k > 0);
            }
        }
#pragma unroll
        for (int k = 0; k < 4; ++k) {
#pragma unroll
            for (int b = 0; b < 2; ++b)
                mma_tf32(s.tmem + kColX + 32 * b, s.tmem + kColAhi + 32 * b + 8 * k,
                         smem_desc(s.wlo + 256 * k, 128, 1024), true);
        }
        commit(s.mbar);
    }
    bool ok = mbar_wait(s.mbar, s.phase);
    if (!ok) ok = mbar_wait(s.mbar, s.phase) && false;  // let the MMAs in flight finish before going on
    s.phase ^= 1u;
    fence_after_sync();
    uint32_t d[32];
    ld32(s.tmem + lane_base + kColX + blk, d);
#pragma unroll
    for (int k = 0; k < 16; ++k) a[k] = {__uint_as_float(d[2 * k]), __uint_as_float(d[2 * k + 1])};
    ld32(s.tmem + lane_base + kColD + blk, d);
#pragma unroll
    for (int k = 0; k < 16; ++k) {
        // hi.hi plus the cross terms, in FP32
        a[k].x = __uint_as_float(d[2 * k]) + a[k].x;
        a[k].y = __uint_as_float(d[2 * k + 1]) + a[k].y;
        if (INV) a[k].y = -a[k].y;
    }
    return ok;
}

}  // namespace tc
}  // namespace hfs
