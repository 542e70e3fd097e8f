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
// The quarter turn q = rint(4r) of r = turns mod 1 is split off exactly,
// leaving theta = 2 pi (r - q/4) with |theta| <= pi/4, where sin is the
// Taylor series to theta^9 and cos - 1 the series to theta^10 (truncation
// below 2e-9).  The small rotation is applied as u + u (cos - 1 - i sin):
// rounding cos theta itself to FP32 would return exactly 1 for
// |theta| < 2.4e-4 while sin theta stays accurate, so |exp(-i theta)|^2 would
// come out as 1 + theta^2, a norm gain of fixed sign at every step for the
// low wavenumbers and the trap centre, where most of the norm sits.  The
// quarter turn (-i)^q is then an exact swap / negation.
__device__ __forceinline__ cpx<float> apply_turns(cpx<float> u, float turns, float scale)
{
    const float r = turns - rintf(turns);
    const float q = rintf(4.0f * r);
    const float f = fmaf(q, -0.25f, r);  // exact
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
