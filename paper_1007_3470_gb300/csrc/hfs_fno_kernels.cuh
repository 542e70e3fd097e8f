// hfs_fno_kernels.cuh -- device kernels of the Fourier-neural-operator
// surrogate: a batched BF16 tensor-core GEMM with FP32 accumulation and fused
// epilogues, and the elementwise, reduction, loss and Adam kernels around it.
#pragma once

#include <cuda_bf16.h>
#include <stdint.h>

namespace hfs {
namespace fno {

typedef __nv_bfloat16 bf16;

// C[b] = alpha * op(A[b]) op(B[b]) (+ beta C[b]) (+ bias[n]) (+ add[b]) -> [pre] -> GELU? -> C, Cb
//   op(A)(m, k) = TA ? A[k lda + m] : A[m lda + k]
//   op(B)(k, n) = TB ? B[n ldb + k] : B[k ldb + n]
// splitk > 1: each z-slice reduces a K range and atomically adds alpha*acc
// into C (no other epilogue; C zeroed by the caller).
struct GemmArgs {
    int M, N, K;
    const bf16 *A;
    int64_t lda, sA;
    const bf16 *B;
    int64_t ldb, sB;
    float *C;
    int64_t ldc, sC;
    bf16 *Cb;
    int64_t ldcb, sCb;
    float *pre;
    int64_t ldp, sP;
    const float *bias;
    const float *add;
    int64_t ldadd, sAdd;
    float alpha;
    int beta, gelu, splitk, batch;
    unsigned *status;  // bit 0 set when a bounded device wait ran out (tensor-core form)
};

constexpr int GT_M = 64, GT_N = 64, GT_K = 32, GT_LD = 40;  // smem rows padded to 40 bf16 (80 B)

__device__ __forceinline__ float gelu_f(float z) { return 0.5f * z * (1.0f + erff(z * 0.70710678118654752f)); }
__device__ __forceinline__ float gelu_grad_f(float z)
{
    return 0.5f * (1.0f + erff(z * 0.70710678118654752f)) + z * expf(-0.5f * z * z) * 0.39894228040143268f;
}

__device__ __forceinline__ void ldsm_x4(unsigned (&r)[4], const bf16 *p)
{
    const unsigned a = (unsigned)__cvta_generic_to_shared(p);
    asm volatile("ldmatrix.sync.aligned.m8n8.x4.shared.b16 {%0,%1,%2,%3}, [%4];"
                 : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3])
                 : "r"(a));
}
__device__ __forceinline__ void ldsm_x2(unsigned (&r)[2], const bf16 *p)
{
    const unsigned a = (unsigned)__cvta_generic_to_shared(p);
    asm volatile("ldmatrix.sync.aligned.m8n8.x2.shared.b16 {%0,%1}, [%2];" : "=r"(r[0]), "=r"(r[1]) : "r"(a));
}
__device__ __forceinline__ void mma_bf16(float (&c)[4], const unsigned (&a)[4], const unsigned (&b)[2])
{
    asm volatile(
        "mma.sync.aligned.m16n8k16.row.col.f32.bf16.bf16.f32 {%0,%1,%2,%3}, {%4,%5,%6,%7}, {%8,%9}, "
        "{%0,%1,%2,%3};"
        : "+f"(c[0]), "+f"(c[1]), "+f"(c[2]), "+f"(c[3])
        : "r"(a[0]), "r"(a[1]), "r"(a[2]), "r"(a[3]), "r"(b[0]), "r"(b[1]));
}

// Load a ROWS x 32 (k) tile into smem as [row][k], from a matrix whose rows
// (m or n) are either k-contiguous (KCONT) or row-contiguous (the transposed
// storage).  Out-of-range elements are zero.
template <bool KCONT>
__device__ __forceinline__ void load_tile(bf16 (*s)[GT_LD], const bf16 *g, int64_t ld, int row0, int rows, int k0,
                                          int kend)
{
    const bf16 zero = __float2bfloat16(0.0f);
    if constexpr (KCONT) {
        // 64 rows x 4 chunks of 8 k
        for (int c = threadIdx.x; c < 64 * 4; c += blockDim.x) {
            const int r = c >> 2, kc = (c & 3) * 8;
            const int row = row0 + r, k = k0 + kc;
            const bf16 *src = g + (int64_t)row * ld + k;
            if (row < rows && k + 8 <= kend && ((uintptr_t)src & 15) == 0) {
                *reinterpret_cast<uint4 *>(&s[r][kc]) = *reinterpret_cast<const uint4 *>(src);
            } else {
#pragma unroll
                for (int i = 0; i < 8; ++i) s[r][kc + i] = (row < rows && k + i < kend) ? src[i] : zero;
            }
        }
    } else {
        // 32 k x 8 chunks of 8 rows
        for (int c = threadIdx.x; c < 32 * 8; c += blockDim.x) {
            const int kk = c >> 3, rc = (c & 7) * 8;
            const int k = k0 + kk, row = row0 + rc;
            const bf16 *src = g + (int64_t)k * ld + row;
            if (k < kend && row + 8 <= rows && ((uintptr_t)src & 15) == 0) {
                const uint4 v = *reinterpret_cast<const uint4 *>(src);
                const bf16 *e = reinterpret_cast<const bf16 *>(&v);
#pragma unroll
                for (int i = 0; i < 8; ++i) s[rc + i][kk] = e[i];
            } else {
#pragma unroll
                for (int i = 0; i < 8; ++i) s[rc + i][kk] = (k < kend && row + i < rows) ? src[i] : zero;
            }
        }
    }
}

template <bool TA, bool TB> __global__ void __launch_bounds__(128) gemm_bf16_kernel(const GemmArgs g)
{
    __shared__ __align__(16) bf16 As[GT_M][GT_LD];
    __shared__ __align__(16) bf16 Bs[GT_N][GT_LD];
    const int n0 = blockIdx.x * GT_N, m0 = blockIdx.y * GT_M;
    const int b = blockIdx.z / g.splitk, kz = blockIdx.z % g.splitk;
    const int kper = ((g.K + g.splitk - 1) / g.splitk + GT_K - 1) / GT_K * GT_K;
    const int kbeg = kz * kper, kend = min(g.K, kbeg + kper);
    const bf16 *A = g.A + (int64_t)b * g.sA;
    const bf16 *B = g.B + (int64_t)b * g.sB;
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int wm = (warp >> 1) * 32, wn = (warp & 1) * 32;
    float acc[2][4][4];
#pragma unroll
    for (int i = 0; i < 2; ++i)
#pragma unroll
        for (int j = 0; j < 4; ++j)
#pragma unroll
            for (int q = 0; q < 4; ++q) acc[i][j][q] = 0.0f;
    for (int k0 = kbeg; k0 < kend; k0 += GT_K) {
        load_tile<!TA>(As, A, g.lda, m0, g.M, k0, kend);
        load_tile<TB>(Bs, B, g.ldb, n0, g.N, k0, kend);
        __syncthreads();
#pragma unroll
        for (int kk = 0; kk < GT_K; kk += 16) {
            unsigned af[2][4], bfr[4][2];
#pragma unroll
            for (int mi = 0; mi < 2; ++mi) ldsm_x4(af[mi], &As[wm + mi * 16 + (lane & 15)][kk + (lane >> 4) * 8]);
#pragma unroll
            for (int ni = 0; ni < 4; ++ni) ldsm_x2(bfr[ni], &Bs[wn + ni * 8 + (lane & 7)][kk + ((lane >> 3) & 1) * 8]);
#pragma unroll
            for (int mi = 0; mi < 2; ++mi)
#pragma unroll
                for (int ni = 0; ni < 4; ++ni) mma_bf16(acc[mi][ni], af[mi], bfr[ni]);
        }
        __syncthreads();
    }
    // epilogue
#pragma unroll
    for (int mi = 0; mi < 2; ++mi)
#pragma unroll
        for (int ni = 0; ni < 4; ++ni)
#pragma unroll
            for (int q = 0; q < 4; ++q) {
                const int m = m0 + wm + mi * 16 + (lane >> 2) + ((q >> 1) << 3);
                const int n = n0 + wn + ni * 8 + (lane & 3) * 2 + (q & 1);
                if (m >= g.M || n >= g.N) continue;
                float v = g.alpha * acc[mi][ni][q];
                if (g.splitk > 1) {
                    atomicAdd(g.C + (int64_t)b * g.sC + (int64_t)m * g.ldc + n, v);
                    continue;
                }
                if (g.beta) v += g.C[(int64_t)b * g.sC + (int64_t)m * g.ldc + n];
                if (g.bias) v += g.bias[n];
                if (g.add) v += g.add[(int64_t)b * g.sAdd + (int64_t)m * g.ldadd + n];
                if (g.pre) g.pre[(int64_t)b * g.sP + (int64_t)m * g.ldp + n] = v;
                if (g.gelu) v = gelu_f(v);
                if (g.C) g.C[(int64_t)b * g.sC + (int64_t)m * g.ldc + n] = v;
                if (g.Cb) g.Cb[(int64_t)b * g.sCb + (int64_t)m * g.ldcb + n] = __float2bfloat16(v);
            }
}

// ---------------------------------------------------------------------------
// Pipelined form of the same GEMM (same arguments, tiles and epilogue): the
// tiles of op(A) and op(B) stream into a three-stage shared-memory ring by
// 16-byte asynchronous copies (cp.async, zero-filled outside the matrix), so
// the loads of tile k + 2 overlap the MMAs of tile k; an operand stored with
// its contiguous dimension along m or n stays in that layout in shared
// memory and is read with ldmatrix.trans (no element-wise transposition).
// Eligible when every 16-byte chunk is all in or all out of range: leading
// dimensions, batch strides and base addresses in whole 8-element chunks,
// and the chunked extents (K; M for a transposed A; N for a row-major B)
// multiples of 8 (gemm_pipe_ok).
// ---------------------------------------------------------------------------
constexpr int GP_STAGES = 3, GP_LDT = 72;  // transposed tiles: [32 k][64 + 8]

__device__ __forceinline__ void ldsm_x4_t(unsigned (&r)[4], const bf16 *p)
{
    const unsigned a = (unsigned)__cvta_generic_to_shared(p);
    asm volatile("ldmatrix.sync.aligned.m8n8.x4.trans.shared.b16 {%0,%1,%2,%3}, [%4];"
                 : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3])
                 : "r"(a));
}
__device__ __forceinline__ void ldsm_x2_t(unsigned (&r)[2], const bf16 *p)
{
    const unsigned a = (unsigned)__cvta_generic_to_shared(p);
    asm volatile("ldmatrix.sync.aligned.m8n8.x2.trans.shared.b16 {%0,%1}, [%2];" : "=r"(r[0]), "=r"(r[1]) : "r"(a));
}
// 16-byte asynchronous copy; an invalid chunk is zero-filled (source size 0)
__device__ __forceinline__ void cp16(bf16 *dst, const bf16 *src, bool valid)
{
    const unsigned d = (unsigned)__cvta_generic_to_shared(dst);
    asm volatile("cp.async.cg.shared.global [%0], [%1], 16, %2;" ::"r"(d), "l"(src), "r"(valid ? 16 : 0) : "memory");
}

inline bool gemm_pipe_ok(const GemmArgs &g, bool ta, bool tb)
{
    auto al = [](const void *p) { return ((uintptr_t)p & 15) == 0; };
    if (!al(g.A) || !al(g.B) || g.lda % 8 || g.ldb % 8 || g.sA % 8 || g.sB % 8) return false;
    if (g.K % 8) return false;
    if (ta && g.M % 8) return false;
    if (!tb && g.N % 8) return false;
    return true;
}

template <bool TA, bool TB> __global__ void __launch_bounds__(128) gemm_bf16_pipe_kernel(const GemmArgs g)
{
    constexpr int A_EL = TA ? GT_K * GP_LDT : GT_M * GT_LD;
    constexpr int B_EL = TB ? GT_N * GT_LD : GT_K * GP_LDT;
    __shared__ __align__(128) bf16 sA[GP_STAGES][A_EL];
    __shared__ __align__(128) bf16 sB[GP_STAGES][B_EL];
    const int n0 = blockIdx.x * GT_N, m0 = blockIdx.y * GT_M;
    const int b = blockIdx.z / g.splitk, kz = blockIdx.z % g.splitk;
    const int kper = ((g.K + g.splitk - 1) / g.splitk + GT_K - 1) / GT_K * GT_K;
    const int kbeg = kz * kper, kend = min(g.K, kbeg + kper);
    const int nk = kend > kbeg ? (kend - kbeg + GT_K - 1) / GT_K : 0;
    const bf16 *A = g.A + (int64_t)b * g.sA;
    const bf16 *B = g.B + (int64_t)b * g.sB;
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int wm = (warp >> 1) * 32, wn = (warp & 1) * 32;

    auto load_stage = [&](int st, int k0) {
        // 256 chunks of 8 elements per operand tile, two per thread
#pragma unroll
        for (int c = threadIdx.x; c < 256; c += 128) {
            if constexpr (!TA) {
                const int r = c >> 2, kc = (c & 3) * 8, row = m0 + r, k = k0 + kc;
                const bool ok = row < g.M && k + 8 <= kend;
                cp16(&sA[st][r * GT_LD + kc], ok ? A + (int64_t)row * g.lda + k : A, ok);
            } else {
                const int kk = c >> 3, mc = (c & 7) * 8, k = k0 + kk, m = m0 + mc;
                const bool ok = k < kend && m < g.M;
                cp16(&sA[st][kk * GP_LDT + mc], ok ? A + (int64_t)k * g.lda + m : A, ok);
            }
            if constexpr (TB) {
                const int r = c >> 2, kc = (c & 3) * 8, row = n0 + r, k = k0 + kc;
                const bool ok = row < g.N && k + 8 <= kend;
                cp16(&sB[st][r * GT_LD + kc], ok ? B + (int64_t)row * g.ldb + k : B, ok);
            } else {
                const int kk = c >> 3, nc = (c & 7) * 8, k = k0 + kk, n = n0 + nc;
                const bool ok = k < kend && n < g.N;
                cp16(&sB[st][kk * GP_LDT + nc], ok ? B + (int64_t)k * g.ldb + n : B, ok);
            }
        }
    };

    float acc[2][4][4];
#pragma unroll
    for (int i = 0; i < 2; ++i)
#pragma unroll
        for (int j = 0; j < 4; ++j)
#pragma unroll
            for (int q = 0; q < 4; ++q) acc[i][j][q] = 0.0f;
#pragma unroll
    for (int s = 0; s < GP_STAGES - 1; ++s) {
        if (s < nk) load_stage(s, kbeg + s * GT_K);
        asm volatile("cp.async.commit_group;" ::: "memory");
    }
    for (int kt = 0; kt < nk; ++kt) {
        asm volatile("cp.async.wait_group %0;" ::"n"(GP_STAGES - 2) : "memory");
        __syncthreads();  // tile kt visible to all; stage (kt - 1) % S no longer read
        if (kt + GP_STAGES - 1 < nk) load_stage((kt + GP_STAGES - 1) % GP_STAGES, kbeg + (kt + GP_STAGES - 1) * GT_K);
        asm volatile("cp.async.commit_group;" ::: "memory");
        const bf16 *a_s = sA[kt % GP_STAGES];
        const bf16 *b_s = sB[kt % GP_STAGES];
#pragma unroll
        for (int kk = 0; kk < GT_K; kk += 16) {
            unsigned af[2][4], bfr[4][2];
#pragma unroll
            for (int mi = 0; mi < 2; ++mi) {
                if constexpr (!TA)
                    ldsm_x4(af[mi], a_s + (wm + mi * 16 + (lane & 15)) * GT_LD + kk + (lane >> 4) * 8);
                else
                    ldsm_x4_t(af[mi], a_s + (kk + (lane & 7) + ((lane >> 4) & 1) * 8) * GP_LDT + wm + mi * 16 +
                                          ((lane >> 3) & 1) * 8);
            }
#pragma unroll
            for (int ni = 0; ni < 4; ++ni) {
                if constexpr (TB)
                    ldsm_x2(bfr[ni], b_s + (wn + ni * 8 + (lane & 7)) * GT_LD + kk + ((lane >> 3) & 1) * 8);
                else
                    ldsm_x2_t(bfr[ni], b_s + (kk + (lane & 7) + ((lane >> 3) & 1) * 8) * GP_LDT + wn + ni * 8);
            }
#pragma unroll
            for (int mi = 0; mi < 2; ++mi)
#pragma unroll
                for (int ni = 0; ni < 4; ++ni) mma_bf16(acc[mi][ni], af[mi], bfr[ni]);
        }
    }
    asm volatile("cp.async.wait_group 0;" ::: "memory");
    // epilogue (as gemm_bf16_kernel), the two adjacent columns (n, n + 1) of
    // an accumulator pair stored together when every output allows it
    auto even = [](int64_t v) { return (v & 1) == 0; };
    auto al8 = [](const void *p) { return ((uintptr_t)p & 7) == 0; };
    const bool vec = g.splitk == 1 && even(g.N) && (!g.C || (al8(g.C) && even(g.ldc) && even(g.sC))) &&
                     (!g.Cb || ((((uintptr_t)g.Cb & 3) == 0) && even(g.ldcb) && even(g.sCb))) &&
                     (!g.pre || (al8(g.pre) && even(g.ldp) && even(g.sP))) &&
                     (!g.add || (al8(g.add) && even(g.ldadd) && even(g.sAdd))) && (!g.bias || al8(g.bias));
#pragma unroll
    for (int mi = 0; mi < 2; ++mi)
#pragma unroll
        for (int ni = 0; ni < 4; ++ni)
#pragma unroll
            for (int h = 0; h < 2; ++h) {
                const int m = m0 + wm + mi * 16 + (lane >> 2) + h * 8;
                const int n = n0 + wn + ni * 8 + (lane & 3) * 2;
                if (m >= g.M || n >= g.N) continue;
                float2 v = make_float2(g.alpha * acc[mi][ni][2 * h], g.alpha * acc[mi][ni][2 * h + 1]);
                if (vec) {
                    const int64_t oc = (int64_t)b * g.sC + (int64_t)m * g.ldc + n;
                    if (g.beta) {
                        const float2 c0 = *reinterpret_cast<const float2 *>(g.C + oc);
                        v.x += c0.x;
                        v.y += c0.y;
                    }
                    if (g.bias) {
                        const float2 bb = *reinterpret_cast<const float2 *>(g.bias + n);
                        v.x += bb.x;
                        v.y += bb.y;
                    }
                    if (g.add) {
                        const float2 ad =
                            *reinterpret_cast<const float2 *>(g.add + (int64_t)b * g.sAdd + (int64_t)m * g.ldadd + n);
                        v.x += ad.x;
                        v.y += ad.y;
                    }
                    if (g.pre) *reinterpret_cast<float2 *>(g.pre + (int64_t)b * g.sP + (int64_t)m * g.ldp + n) = v;
                    if (g.gelu) v = make_float2(gelu_f(v.x), gelu_f(v.y));
                    if (g.C) *reinterpret_cast<float2 *>(g.C + oc) = v;
                    if (g.Cb)
                        *reinterpret_cast<__nv_bfloat162 *>(g.Cb + (int64_t)b * g.sCb + (int64_t)m * g.ldcb + n) =
                            __floats2bfloat162_rn(v.x, v.y);
                    continue;
                }
#pragma unroll
                for (int q = 0; q < 2; ++q) {
                    const int nq = n + q;
                    if (nq >= g.N) continue;
                    float w = q ? v.y : v.x;
                    if (g.splitk > 1) {
                        atomicAdd(g.C + (int64_t)b * g.sC + (int64_t)m * g.ldc + nq, w);
                        continue;
                    }
                    if (g.beta) w += g.C[(int64_t)b * g.sC + (int64_t)m * g.ldc + nq];
                    if (g.bias) w += g.bias[nq];
                    if (g.add) w += g.add[(int64_t)b * g.sAdd + (int64_t)m * g.ldadd + nq];
                    if (g.pre) g.pre[(int64_t)b * g.sP + (int64_t)m * g.ldp + nq] = w;
                    if (g.gelu) w = gelu_f(w);
                    if (g.C) g.C[(int64_t)b * g.sC + (int64_t)m * g.ldc + nq] = w;
                    if (g.Cb) g.Cb[(int64_t)b * g.sCb + (int64_t)m * g.ldcb + nq] = __float2bfloat16(w);
                }
            }
}

// ---------------------------------------------------------------------------
// elementwise and reductions
// ---------------------------------------------------------------------------

// x [rows][cin] FP32 -> out [rows][ldo] BF16, zero-padded columns
__global__ void to_bf16_pad_kernel(const float *x, int64_t rows, int cin, bf16 *out, int ldo)
{
    const int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (i >= rows * ldo) return;
    const int64_t r = i / ldo;
    const int c = (int)(i - r * ldo);
    out[i] = __float2bfloat16(c < cin ? x[r * cin + c] : 0.0f);
}

__global__ void to_bf16_kernel(const float *x, bf16 *out, int64_t n)
{
    const int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (i < n) out[i] = __float2bfloat16(x[i]);
}

// dZ = dH * gelu'(pre) (or dH when apply == 0); FP32 and BF16 outputs
__global__ void gelu_bwd_kernel(const float *dH, const float *pre, int apply, float *dZ, bf16 *dZb, int64_t n)
{
    const int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (i >= n) return;
    const float v = apply ? dH[i] * gelu_grad_f(pre[i]) : dH[i];
    if (dZ) dZ[i] = v;
    if (dZb) dZb[i] = __float2bfloat16(v);
}

// out[c] += sum_r A[r][c]  (rows split over the grid; FP32 atomics)
__global__ void colsum_kernel(const float *A, int64_t rows, int cols, float *out)
{
    const int c = threadIdx.x;  // blockDim.x == cols (<= 1024)
    const int64_t per = (rows + gridDim.x - 1) / gridDim.x;
    const int64_t r0 = blockIdx.x * per, r1 = min(rows, r0 + per);
    float s = 0.0f;
    for (int64_t r = r0; r < r1; ++r) s += A[r * cols + c];
    if (c < cols) atomicAdd(out + c, s);
}

// per-sample sums of |O - Y|^2 and |Y|^2 (one block per sample)
__global__ void loss_sums_kernel(const float *O, const float *Y, int64_t per_sample, float *sums)
{
    __shared__ float red[2][256];
    const int64_t b = blockIdx.x;
    float num = 0.0f, den = 0.0f;
    for (int64_t i = threadIdx.x; i < per_sample; i += blockDim.x) {
        const float d = O[b * per_sample + i] - Y[b * per_sample + i];
        const float y = Y[b * per_sample + i];
        num += d * d;
        den += y * y;
    }
    red[0][threadIdx.x] = num;
    red[1][threadIdx.x] = den;
    __syncthreads();
    for (int s = blockDim.x / 2; s > 0; s >>= 1) {
        if ((int)threadIdx.x < s) {
            red[0][threadIdx.x] += red[0][threadIdx.x + s];
            red[1][threadIdx.x] += red[1][threadIdx.x + s];
        }
        __syncthreads();
    }
    if (threadIdx.x == 0) {
        sums[2 * b] = red[0][0];
        sums[2 * b + 1] = red[1][0];
    }
}

// loss = mean_b sqrt(num_b / den_b); dO = (O - Y) / (sqrt(num_b den_b) B)
__global__ void loss_grad_kernel(const float *O, const float *Y, const float *sums, int64_t per_sample, int batch,
                                 float *dO, bf16 *dOb)
{
    const int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (i >= per_sample * batch) return;
    const int64_t b = i / per_sample;
    const float nd = sqrtf(sums[2 * b] * sums[2 * b + 1]);
    const float v = (nd > 0.0f) ? (O[i] - Y[i]) / (nd * (float)batch) : 0.0f;
    dO[i] = v;
    dOb[i] = __float2bfloat16(v);
}

// one block of 256 threads
__global__ void loss_value_kernel(const float *sums, int batch, float *loss)
{
    __shared__ float red[256];
    float s = 0.0f;
    for (int b = threadIdx.x; b < batch; b += blockDim.x) s += sqrtf(sums[2 * b] / sums[2 * b + 1]);
    red[threadIdx.x] = s;
    __syncthreads();
    for (int k = blockDim.x / 2; k > 0; k >>= 1) {
        if ((int)threadIdx.x < k) red[threadIdx.x] += red[threadIdx.x + k];
        __syncthreads();
    }
    if (threadIdx.x == 0) *loss = red[0] / (float)batch;
}

__global__ void adam_kernel(float *p, const float *g, float *m, float *v, int64_t n, float lr, float b1, float b2,
                            float eps, float c1, float c2)
{
    const int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (i >= n) return;
    const float gi = g[i];
    const float mi = b1 * m[i] + (1.0f - b1) * gi;
    const float vi = b2 * v[i] + (1.0f - b2) * gi * gi;
    m[i] = mi;
    v[i] = vi;
    p[i] -= lr * (mi / c1) / (sqrtf(vi / c2) + eps);
}

// complex mixing weights as real blocks: R1[k] = [Rre | Rim], R2[k] = [-Rim | Rre] ([C][2C])
__global__ void mixing_weights_kernel(const float *Rre, const float *Rim, int M, int C, bf16 *R1, bf16 *R2)
{
    const int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (i >= (int64_t)M * C * 2 * C) return;
    const int64_t k = i / (C * 2 * C);
    const int64_t r = (i / (2 * C)) % C;
    const int col = (int)(i % (2 * C));
    const int64_t src = (k * C + r) * C + (col % C);
    const float re = Rre[src], im = Rim[src];
    R1[i] = __float2bfloat16(col < C ? re : im);
    R2[i] = __float2bfloat16(col < C ? -im : re);
}

// gradients of Rre, Rim from those of R1, R2
__global__ void mixing_grad_kernel(const float *dR1, const float *dR2, int M, int C, float *gRre, float *gRim)
{
    const int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (i >= (int64_t)M * C * C) return;
    const int64_t k = i / (C * C), r = (i / C) % C, c = i % C;
    const int64_t row = (k * C + r) * 2 * C;
    gRre[i] = dR1[row + c] + dR2[row + C + c];
    gRim[i] = dR1[row + C + c] - dR2[row + c];
}

// DFT matrices: F2 [2M][L] (cos rows, then -sin rows); Gre, Gim [L][M]
__global__ void dft_consts_kernel(int L, int M, bf16 *F2, bf16 *Gre, bf16 *Gim)
{
    const int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (i >= (int64_t)L * M) return;
    const int k = (int)(i / L), x = (int)(i % L);
    double s, c;
    sincospi(2.0 * (double)((int64_t)k * x % L) / (double)L, &s, &c);
    F2[(int64_t)k * L + x] = __float2bfloat16((float)c);
    F2[(int64_t)(M + k) * L + x] = __float2bfloat16((float)-s);
    const double w = (k == 0) ? 1.0 : 2.0;
    Gre[(int64_t)x * M + k] = __float2bfloat16((float)(w * c / L));
    Gim[(int64_t)x * M + k] = __float2bfloat16((float)(-w * s / L));
}

// deterministic uniform(-scale, scale) from a counter-based hash (splitmix64)
__global__ void init_uniform_kernel(float *p, int64_t n, float scale, uint64_t seed)
{
    const int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (i >= n) return;
    uint64_t z = seed + 0x9E3779B97F4A7C15ull * (uint64_t)(i + 1);
    z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ull;
    z = (z ^ (z >> 27)) * 0x94D049BB133111EBull;
    z ^= z >> 31;
    const double u = (double)(z >> 11) * (1.0 / 9007199254740992.0);  // [0,1)
    p[i] = (float)((2.0 * u - 1.0) * scale);
}

}  // namespace fno
}  // namespace hfs
