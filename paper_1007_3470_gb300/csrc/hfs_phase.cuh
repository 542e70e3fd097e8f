// hfs_phase.cuh -- pointwise phase factors of the merged x-phase (kick +
// B flow, Lemma 1) and of the kinetic k-phase (Eq. GP1ODE_T).
//
// Phases are carried in turns (1 turn = 2 pi rad).  The quadratic parts use
// an exact integer m^2 (|m| <= n/2 <= 2048, so m^2 < 2^23 is exact in FP32)
// times a per-stage coefficient that the FP64 schedule hands over as an
// unevaluated sum hi + lo of two floats.  frac_turns() forms (hi + lo) m2
// modulo 1 with an error of a few 2^-24 turns independent of the size of
// the product, so the FP32 path keeps its phase error near one ulp of a
// turn even where the chirp reaches many turns.
#pragma once

#include "hfs_internal.cuh"

namespace hfs {

// (hi + lo) * m2 mod 1, result in about [-1, 1]; m2 an exact float integer.
__device__ __forceinline__ float frac_turns(float m2, float hi, float lo)
{
    const float p = hi * m2;
    const float err = fmaf(hi, m2, -p);  // exact rounding error of the product
    const float r = p - rintf(p);        // exact for |p| < 2^23
    return r + fmaf(lo, m2, err);
}

__device__ __forceinline__ double frac_turns(double m2, double c, double /*unused*/)
{
    const double p = c * m2;
    return p - rint(p);
}

// u * exp(-2 pi i turns) * scale (FP32).
// The quarter turn q = rint(4 turns) is split off exactly (only q mod 4
// matters), leaving theta = 2 pi (turns - q/4) with |theta| <= pi/4, where sin is the
// Taylor series to theta^9 and cos - 1 the series to theta^10 (truncation
// below 2e-9).  The small rotation is applied as u + u (cos - 1 - i sin):
// rounding cos theta itself to FP32 would return exactly 1 for
// |theta| < 2.4e-4 while sin theta stays accurate, so |exp(-i theta)|^2 would
// come out as 1 + theta^2, a norm gain of fixed sign at every step for the
// low wavenumbers and the trap centre, where most of the norm sits.  The
// quarter turn (-i)^q is then an exact swap / negation.
__device__ __forceinline__ cpx<float> apply_turns(cpx<float> u, float turns, float scale)
{
    // rint(4 turns) and turns - q/4 are exact: the same quarter turn mod 4 and
    // remainder as after a reduction of turns mod 1
    const float q = rintf(4.0f * turns);
    const float f = fmaf(q, -0.25f, turns);  // exact
    const float th = f * 6.28318530717958647692f;
    const float t2 = th * th;
    float ps = fmaf(t2, 1.0f / 362880.0f, -1.0f / 5040.0f);
    ps = fmaf(ps, t2, 1.0f / 120.0f);
    ps = fmaf(ps, t2, -1.0f / 6.0f);
    const float sn = fmaf(th * t2, ps, th);
    float pc = fmaf(t2, -1.0f / 3628800.0f, 1.0f / 40320.0f);
    pc = fmaf(pc, t2, -1.0f / 720.0f);
    pc = fmaf(pc, t2, 1.0f / 24.0f);
    pc = fmaf(pc, t2, -0.5f);
    const float cm1 = t2 * pc;  // cos(theta) - 1
    const float wx = u.x + fmaf(u.x, cm1, u.y * sn);
    const float wy = u.y + fmaf(u.y, cm1, -u.x * sn);
    const int qi = ((int)q) & 3;
    float ox = (qi & 1) ? wy : wx;
    float oy = (qi & 1) ? wx : wy;
    ox = (qi >= 2) ? -ox : ox;
    oy = (qi == 1 || qi == 2) ? -oy : oy;
    return {ox * scale, oy * scale};
}

// Two grid points at once: the same per-lane operations as frac_turns /
// apply_turns above; with PK the FP32 arithmetic runs in packed two-lane
// instructions (sm_100 family), so the results are bit-identical either way.
__device__ __forceinline__ float2 neg2(float2 a) { return make_float2(-a.x, -a.y); }
__device__ __forceinline__ float2 rint2(float2 a) { return make_float2(rintf(a.x), rintf(a.y)); }
__device__ __forceinline__ float2 bc2(float c) { return make_float2(c, c); }

template <bool PK> __device__ __forceinline__ float2 frac_turns2(float2 m2, float hi, float lo)
{
    if constexpr (PK) {
        const float2 p = __fmul2_rn(bc2(hi), m2);
        const float2 err = __ffma2_rn(bc2(hi), m2, neg2(p));
        const float2 r = __fadd2_rn(p, neg2(rint2(p)));
        return __fadd2_rn(r, __ffma2_rn(bc2(lo), m2, err));
    } else {
        return make_float2(frac_turns(m2.x, hi, lo), frac_turns(m2.y, hi, lo));
    }
}

// the small-rotation part of apply_turns for two points: quarter turns q,
// sin theta and cos theta - 1
// (no separate reduction mod 1: rint(4 turns) and turns - q/4 are exact and
// give the same quarter turn mod 4 and the same remainder as after one)
__device__ __forceinline__ void small_rotation2(float2 turns, float2 &q, float2 &sn, float2 &cm1)
{
    q = rint2(__fmul2_rn(bc2(4.0f), turns));
    const float2 f = __ffma2_rn(q, bc2(-0.25f), turns);
    const float2 th = __fmul2_rn(f, bc2(6.28318530717958647692f));
    const float2 t2 = __fmul2_rn(th, th);
    float2 ps = __ffma2_rn(t2, bc2(1.0f / 362880.0f), bc2(-1.0f / 5040.0f));
    ps = __ffma2_rn(ps, t2, bc2(1.0f / 120.0f));
    ps = __ffma2_rn(ps, t2, bc2(-1.0f / 6.0f));
    sn = __ffma2_rn(__fmul2_rn(th, t2), ps, th);
    float2 pc = __ffma2_rn(t2, bc2(-1.0f / 3628800.0f), bc2(1.0f / 40320.0f));
    pc = __ffma2_rn(pc, t2, bc2(-1.0f / 720.0f));
    pc = __ffma2_rn(pc, t2, bc2(1.0f / 24.0f));
    pc = __ffma2_rn(pc, t2, bc2(-0.5f));
    cm1 = __fmul2_rn(t2, pc);
}

// u (1 + cm1 - i sn) followed by the exact quarter turn (-i)^q and the scale
__device__ __forceinline__ cpx<float> finish_rotation(cpx<float> u, float q, float sn, float cm1, float scale)
{
    const float wx = u.x + fmaf(u.x, cm1, u.y * sn);
    const float wy = u.y + fmaf(u.y, cm1, -u.x * sn);
    const int qi = ((int)q) & 3;
    float ox = (qi & 1) ? wy : wx;
    float oy = (qi & 1) ? wx : wy;
    ox = (qi >= 2) ? -ox : ox;
    oy = (qi == 1 || qi == 2) ? -oy : oy;
    return {ox * scale, oy * scale};
}

template <bool PK>
__device__ __forceinline__ void apply_turns2(cpx<float> &u0, cpx<float> &u1, float2 turns, float scale)
{
    if constexpr (PK) {
        float2 q, sn, cm1;
        small_rotation2(turns, q, sn, cm1);
        u0 = finish_rotation(u0, q.x, sn.x, cm1.x, scale);
        u1 = finish_rotation(u1, q.y, sn.y, cm1.y, scale);
    } else {
        u0 = apply_turns(u0, turns.x, scale);
        u1 = apply_turns(u1, turns.y, scale);
    }
}

__device__ __forceinline__ cpx<double> apply_turns(cpx<double> u, double turns, double scale)
{
    turns -= rint(turns);
    double s, c;
    sincospi(2.0 * turns, &s, &c);
    c *= scale;
    s *= scale;
    return {u.x * c + u.y * s, u.y * c - u.x * s};
}

// the perturbation V_I(x) of one axis
__device__ __forceinline__ float vi_eval(int kind, float x, float k)
{
    if (kind == HFS_VI_X4) {
        const float x2 = x * x;
        return x2 * x2;
    }
    if (kind == HFS_VI_COS) return __cosf(k * x);
    return 0.0f;
}

__device__ __forceinline__ double vi_eval(int kind, double x, double k)
{
    if (kind == HFS_VI_X4) {
        const double x2 = x * x;
        return x2 * x2;
    }
    if (kind == HFS_VI_COS) return cos(k * x);
    return 0.0;
}

}  // namespace hfs
