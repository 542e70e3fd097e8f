// hfs_internal.cuh -- device data layouts shared by the library's kernels
// and its host code (not part of the public ABI).
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include <cmath>

#include "hfs.h"

namespace hfs {

// ---------------------------------------------------------------------------
// complex values: interleaved (re, im), 8- or 16-byte aligned
// ---------------------------------------------------------------------------
template <typename R> struct alignas(2 * sizeof(R)) cpx {
    R x, y;
};

template <typename R> __device__ __forceinline__ cpx<R> cadd(cpx<R> a, cpx<R> b) { return {a.x + b.x, a.y + b.y}; }
template <typename R> __device__ __forceinline__ cpx<R> csub(cpx<R> a, cpx<R> b) { return {a.x - b.x, a.y - b.y}; }

// Packed FP32 complex add / subtract (one two-lane instruction, sm_100
// family).  Each lane is the same IEEE round-to-nearest operation as the
// scalar form, so results are bit-identical to cadd / csub.
#ifndef HFS_PACK_SUBNEG
#define HFS_PACK_SUBNEG 1
#endif
__device__ __forceinline__ float2 f2(cpx<float> a) { return make_float2(a.x, a.y); }
__device__ __forceinline__ cpx<float> cadd_p(cpx<float> a, cpx<float> b)
{
    const float2 r = __fadd2_rn(f2(a), f2(b));
    return {r.x, r.y};
}
__device__ __forceinline__ cpx<float> csub_p(cpx<float> a, cpx<float> b)
{
#if HFS_PACK_SUBNEG
    const float2 r = __fadd2_rn(f2(a), make_float2(-b.x, -b.y));
#else
    const float2 r = __ffma2_rn(f2(b), make_float2(-1.0f, -1.0f), f2(a));  // exact product
#endif
    return {r.x, r.y};
}
// t + SG (-i) d = (t.x + SG d.y, t.y - SG d.x), SG = +-1, as one packed fma
template <int SG> __device__ __forceinline__ cpx<float> cadd_rot_p(cpx<float> t, cpx<float> d)
{
    const float2 r = __ffma2_rn(make_float2(d.y, d.x), make_float2((float)SG, (float)-SG), f2(t));
    return {r.x, r.y};
}

template <typename R> __device__ __forceinline__ cpx<R> cmul(cpx<R> a, cpx<R> b)
{
    return {a.x * b.x - a.y * b.y, a.x * b.y + a.y * b.x};
}
// a * conj(b)
template <typename R> __device__ __forceinline__ cpx<R> cmulc(cpx<R> a, cpx<R> b)
{
    return {a.x * b.x + a.y * b.y, a.y * b.x - a.x * b.y};
}

// ---------------------------------------------------------------------------
// per-instance parameters as the kernels see them
// ---------------------------------------------------------------------------
struct DevInst {
    int64_t off;          // element offset of the instance in psi
    int32_t n[3];         // points per axis
    int32_t plan;         // 1D: index into the plan table (grid size class)
    double xc[3];         // box centre per axis, x_j = xc + (j - n/2) dx
    double dx[3];         // mesh width per axis
    double len[3];        // box length per axis
    double mu;
    int32_t omega_law;
    int32_t vi_kind;
    double w0;
    double law[3];
    double axis_scale[3];
    double eps, vi_k, sigma;
    // 1D, V_I = cos(k x): k x / (2 pi) in turns as (a_hi + a_lo) + (b_hi + b_lo) m
    // for x = xc + m dx (a = k xc / (2 pi) mod 1, b = k dx / (2 pi)), FP32 pairs
    float vi_turns[4];
    // 1D FP32 kernels: xc, dx, eps, vi_k, sigma rounded to FP32, the
    // perturbation kind in effect (none where eps = 0) and whether xc != 0
    float f32[5];
    int32_t vi_kind_eff, asym;
};

// vi_turns and the FP32 copies of a 1D instance from its FP64 parameters
// (host; the same roundings as converting on the device)
inline void set_1d_fp32_params(DevInst &d)
{
    d.f32[0] = (float)d.xc[0];
    d.f32[1] = (float)d.dx[0];
    d.f32[2] = (float)d.eps;
    d.f32[3] = (float)d.vi_k;
    d.f32[4] = (float)d.sigma;
    d.vi_kind_eff = d.eps != 0.0 ? d.vi_kind : HFS_VI_NONE;
    d.asym = d.xc[0] != 0.0 ? 1 : 0;
    const double inv_2pi = 0.159154943091895335768883763372514362;
    const double b = d.vi_k * d.dx[0] * inv_2pi;
    double a = d.vi_k * d.xc[0] * inv_2pi;
    a -= std::nearbyint(a);
    d.vi_turns[0] = (float)b;
    d.vi_turns[1] = (float)(b - (double)d.vi_turns[0]);
    d.vi_turns[2] = (float)a;
    d.vi_turns[3] = (float)(a - (double)d.vi_turns[2]);
}

// FSAL-merged record of sub-stage j (FP32 path, 32 bytes):
//   x-phase X_j :  turns(x) = K2 m^2 + K1 m + K0   with m = j - n/2
//                  plus sB2pi * (eps V_I(x) + sigma |u|^2)   [+ F-split trap]
//   drift D_{j+1}: turns(k) = G m_k^2             with m_k the signed wavenumber index
// Every "turns" coefficient is carried as an unevaluated float sum hi + lo.
struct alignas(16) RecF {
    float k2hi, k2lo, k1hi, k1lo;
    float k0, sb2pi, ghi, glo;
};
// FP64 path (48 bytes)
struct alignas(16) RecD {
    double k2, k1, k0, sb2pi, g, pad;
};

// per-stage harmonic-flow coefficients (FP64), one record per axis
struct alignas(16) StageFGE {
    double f, g, e, tau;
};

// device status word bits
enum : unsigned {
    ST_NONFINITE = 1u,
    ST_TIMEOUT = 2u,
    ST_BADPLAN = 4u,
};

// 1D work item: `count` consecutive instances (after sorting) of one plan
struct WorkItem {
    int32_t first;  // index into the sorted instance order
    int32_t count;  // instances in this item (<= instances per CTA)
    int32_t plan;   // plan id (grid size class + elements per thread)
    int32_t pad;
};

// supported 1D sizes
constexpr int kNumSizes = 6;  // 128 ... 4096
__host__ __device__ constexpr int size_class(int n)
{
    return n == 128 ? 0 : n == 256 ? 1 : n == 512 ? 2 : n == 1024 ? 3 : n == 2048 ? 4 : n == 4096 ? 5 : -1;
}
// 1D plans: E values per thread and the order of the Stockham radices.
// plan code 0: E = 16, radix-16 passes first; 1: E = 8 (radix 8); 2: E = 16,
// the alternative order (radix 8 throughout for n = 4096, the small radix
// first otherwise); 3: E = 4 (radix 4).  plan id = size_class * 4 + code.
constexpr int kPlanCodes = 4;
__host__ __device__ constexpr int plan_code(int ept, bool alt) { return ept == 16 ? (alt ? 2 : 0) : ept == 8 ? 1 : 3; }
__host__ __device__ constexpr int plan_id(int n, int ept, bool alt = false) { return size_class(n) * kPlanCodes + plan_code(ept, alt); }
// codes 2 and 3 live in the "wide" step kernels only (the default kernels
// keep the smaller instruction footprint)
__host__ __device__ constexpr bool plan_is_wide(int plan) { return (plan % kPlanCodes) >= 2; }

constexpr int kCtaThreads = 256;

// Twiddle table, one region per Stockham pass shape: a radix-R pass that
// forms sub-transforms of length L = NS R (NS >= 2 earlier length) needs
// exp(-2 pi i j r / L) for r = 1..R-1, j = 0..NS-1, stored at
// tw_pass_offset(L, R) + (r - 1) NS + j, so the lanes of a warp (consecutive
// j) read consecutive entries.  Regions for L = 4..4096, R = 2, 4, 8, 16.
__host__ __device__ constexpr int64_t tw_region_size(int L, int R) { return (R <= L / 2) ? (int64_t)(L / R) * (R - 1) : 0; }
__host__ __device__ constexpr int64_t tw_length_size(int L)
{
    return tw_region_size(L, 2) + tw_region_size(L, 4) + tw_region_size(L, 8) + tw_region_size(L, 16);
}
__host__ __device__ constexpr int64_t tw_pass_offset(int L, int R)
{
    int64_t off = 0;
    for (int l = 4; l < L; l <<= 1) off += tw_length_size(l);
    for (int r = 2; r < R; r <<= 1) off += tw_region_size(L, r);
    return off;
}
constexpr int kTwiddleMaxLength = 4096;
constexpr int64_t kTwiddleTotal = tw_pass_offset(2 * kTwiddleMaxLength, 2);

}  // namespace hfs
