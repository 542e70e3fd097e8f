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

// sin theta and cos theta - 1 for theta = 2 pi f, |f| <= 1/8 (plus
// rounding).  sin / theta and (cos - 1) / theta^2 as polynomials of degree
// 3 in t2 = theta^2 (sin of degree 7, cos - 1 of degree 8 in theta),
// near-minimax on |theta| <= pi/4: fitted by
// Lawson-reweighted least squares on Chebyshev nodes for the relative error,
// the coefficients rounded to FP32 one at a time with the later ones refitted.
// Relative error <= 4.0e-9 (sin) and <= 8.9e-10 (cos - 1), well below FP32
// rounding, and alternating in sign over the interval.  cos - 1 rather than
// cos: rounding cos theta itself to FP32 would return exactly 1 for
// |theta| < 2.4e-4 while sin theta stays accurate, so |exp(-i theta)|^2 would
// come out as 1 + theta^2, a norm gain of fixed sign at every step for the
// low wavenumbers and the trap centre, where most of the norm sits.
constexpr float kSin3 = -1.666665524e-01f, kSin5 = 8.332189173e-03f, kSin7 = -1.951829181e-04f;
constexpr float kCos2 = -0.5f, kCos4 = 4.166665301e-02f, kCos6 = -1.388761215e-03f, kCos8 = 2.446113103e-05f;

__device__ __forceinline__ void small_rotation(float f, float &sn, float &cm1)
{
    const float th = f * 6.28318530717958647692f;
    const float t2 = th * th;
    float ps = fmaf(t2, kSin7, kSin5);
    ps = fmaf(ps, t2, kSin3);
    sn = fmaf(th * t2, ps, th);
    float pc = fmaf(t2, kCos8, kCos6);
    pc = fmaf(pc, t2, kCos4);
    pc = fmaf(pc, t2, kCos2);
    cm1 = t2 * pc;
}

// 1.5 * 2^23: for |x| < 2^22, x + kRoundMagic is rounded to an integer (to
// nearest, ties to even, as rint) held in the low mantissa bits, so one
// addition gives rint(x) (the sum minus kRoundMagic, exact) and rint(x) mod 4
// (the low two bits of the sum's encoding: 2^22 + rint(x) = rint(x) mod 4).
// x = 4 turns here; an FP32 phase of 2^20 turns or more has lost its angle
// to rounding (ulp >= 1/8 turn) in any form.
constexpr float kRoundMagic = 12582912.0f;

// u (1 + cm1 - i sn) scale, then the exact quarter turn (-i)^qi (a swap and
// sign flips).  The power-of-two scale is folded in: the caller passes
// sn scale and cm1 scale (exact), and u scale + u (cm1 - i sn) scale rounds
// exactly as (u + u (cm1 - i sn)) scale would.
__device__ __forceinline__ cpx<float> finish_rotation(cpx<float> u, int qi, float sn, float cm1, float scale)
{
    const float wx = fmaf(u.x, scale, fmaf(u.x, cm1, u.y * sn));
    const float wy = fmaf(u.y, scale, fmaf(u.y, cm1, -u.x * sn));
    const bool swap = qi & 1;
    const float ox = swap ? wy : wx;
    const float oy = swap ? wx : wy;
    const unsigned nx = (unsigned)(qi & 2) << 30;                // -x for qi = 2, 3
    const unsigned ny = (unsigned)((qi ^ (qi << 1)) & 2) << 30;  // -y for qi = 1, 2
    return {__int_as_float(__float_as_int(ox) ^ nx), __int_as_float(__float_as_int(oy) ^ ny)};
}

// u * exp(-2 pi i turns) * scale (FP32, scale a power of two).  The quarter
// turn q = rint(4 turns) is split off exactly: rint(4 turns) and
// turns - q/4 are exact and give the same quarter turn mod 4 and the same
// remainder as after a reduction of turns mod 1, leaving
// theta = 2 pi (turns - q/4), |theta| <= pi/4.
__device__ __forceinline__ cpx<float> apply_turns(cpx<float> u, float turns, float scale)
{
    const float tq = fmaf(4.0f, turns, kRoundMagic);
    const float q = tq - kRoundMagic;
    float sn, cm1;
    small_rotation(fmaf(q, -0.25f, turns), sn, cm1);
    return finish_rotation(u, __float_as_int(tq) & 3, sn * scale, cm1 * scale, scale);
}

// cos and sin of 2 pi (r + c) for an exact reduced part |r| <= 1/2 and a
// small correction c: the quarter turn split off as in apply_turns, the
// remainder through small_rotation, then the quarter turn applied exactly
// (cos(a + q pi/2), sin(a + q pi/2) are +-cos a, +-sin a).
__device__ __forceinline__ void sincos_turns(float r, float c, float &cs, float &sn)
{
    const float tq = fmaf(4.0f, r + c, kRoundMagic);
    const float q = tq - kRoundMagic;
    float s, cm1;
    small_rotation(fmaf(q, -0.25f, r) + c, s, cm1);
    const float co = 1.0f + cm1;
    const int qi = __float_as_int(tq) & 3;
    const float a = (qi & 1) ? s : co;  // cos or sin of the remainder
    const float b = (qi & 1) ? co : s;
    cs = (qi == 1 || qi == 2) ? -a : a;
    sn = (qi >= 2) ? -b : b;
}

// The merged phases of a pair of grid points, in turns, as an exact part r
// (the reduced product hi m2 - rint(hi m2), |r| <= 1/2) plus a correction c
// (the product's rounding error, lo m2 and any further terms).  The angle is
// rounded once, after the quarter turn is split off: (r - q/4) is exact and
// |r - q/4 + c| <= 1/8, so the rounding is 4x finer than that of the sum
// r + c at magnitude up to 1/2 (the error of the FP32 path is set by phase
// and state rounding accumulated over the steps).
struct Turns2 {
    float2 r, c;
};

__device__ __forceinline__ float2 neg2(float2 a) { return make_float2(-a.x, -a.y); }
__device__ __forceinline__ float2 rint2(float2 a) { return make_float2(rintf(a.x), rintf(a.y)); }
__device__ __forceinline__ float2 bc2(float c) { return make_float2(c, c); }

// With PK the FP32 arithmetic runs in packed two-lane instructions (sm_100
// family) on both points at once, otherwise lane by lane; the per-lane
// operations are the same, so the results are bit-identical either way.
template <bool PK> __device__ __forceinline__ float2 add2(float2 a, float2 b)
{
    if constexpr (PK) return __fadd2_rn(a, b);
    else return make_float2(a.x + b.x, a.y + b.y);
}

template <bool PK> __device__ __forceinline__ float2 mul2(float2 a, float2 b)
{
    if constexpr (PK) return __fmul2_rn(a, b);
    else return make_float2(a.x * b.x, a.y * b.y);
}

template <bool PK> __device__ __forceinline__ float2 fma2(float2 a, float2 b, float2 c)
{
    if constexpr (PK) return __ffma2_rn(a, b, c);
    else return make_float2(fmaf(a.x, b.x, c.x), fmaf(a.y, b.y, c.y));
}

// small_rotation for two angles in packed FP32; cm1 comes out multiplied by
// cs, a power of two folded into the polynomial's coefficients (every Horner
// step scales exactly, so cm1 cs rounds exactly as cm1 times cs would)
__device__ __forceinline__ void small_rotation2(float2 f, float2 &sn, float2 &cm1, float cs = 1.0f)
{
    const float2 th = __fmul2_rn(f, bc2(6.28318530717958647692f));
    const float2 t2 = __fmul2_rn(th, th);
    float2 ps = __ffma2_rn(t2, bc2(kSin7), bc2(kSin5));
    ps = __ffma2_rn(ps, t2, bc2(kSin3));
    sn = __ffma2_rn(__fmul2_rn(th, t2), ps, th);
    float2 pc = __ffma2_rn(t2, bc2(kCos8 * cs), bc2(kCos6 * cs));
    pc = __ffma2_rn(pc, t2, bc2(kCos4 * cs));
    pc = __ffma2_rn(pc, t2, bc2(kCos2 * cs));
    cm1 = __fmul2_rn(t2, pc);
}

// (hi + lo) m2 mod 1 for two exact float integers m2 (< 2^23)
template <bool PK> __device__ __forceinline__ Turns2 frac_turns2(float2 m2, float hi, float lo)
{
    if constexpr (PK) {
        const float2 p = __fmul2_rn(bc2(hi), m2);
        const float2 err = __ffma2_rn(bc2(hi), m2, neg2(p));  // exact rounding error of the product
        return {__fadd2_rn(p, neg2(rint2(p))), __ffma2_rn(bc2(lo), m2, err)};
    } else {
        Turns2 t;
        const float px = hi * m2.x, py = hi * m2.y;
        t.r = make_float2(px - rintf(px), py - rintf(py));
        t.c = make_float2(fmaf(lo, m2.x, fmaf(hi, m2.x, -px)), fmaf(lo, m2.y, fmaf(hi, m2.y, -py)));
        return t;
    }
}

//
// scale: a compile-time power of two (folded into the polynomial); C: a
// run-time factor near 1 (the norm projection of the k-phase), applied as
// u C scale + u (cm1 - i sn) C scale; C = 1 gives bit-identical results to
// the unprojected form.
template <bool PK, bool CORR = false>
__device__ __forceinline__ void apply_turns2(cpx<float> &u0, cpx<float> &u1, Turns2 t, float scale, float C = 1.0f)
{
    const float2 tq = fma2<PK>(bc2(4.0f), add2<PK>(t.r, t.c), bc2(kRoundMagic));
    const float2 q = add2<PK>(tq, bc2(-kRoundMagic));
    const float2 f = add2<PK>(fma2<PK>(q, bc2(-0.25f), t.r), t.c);
    float2 sn, cm1;
    const float sc = CORR ? scale * C : scale;  // exact: scale is a power of two
    if constexpr (PK) {
        small_rotation2(f, sn, cm1, scale);
        if (CORR || scale != 1.0f) sn = __fmul2_rn(sn, bc2(sc));  // folded away for the unscaled x-phase
        if constexpr (CORR) cm1 = __fmul2_rn(cm1, bc2(C));
    } else {
        small_rotation(f.x, sn.x, cm1.x);
        small_rotation(f.y, sn.y, cm1.y);
        if (CORR || scale != 1.0f) {
            sn = mul2<PK>(sn, bc2(sc));
            cm1 = mul2<PK>(cm1, bc2(sc));
        }
    }
    u0 = finish_rotation(u0, __float_as_int(tq.x) & 3, sn.x, cm1.x, sc);
    u1 = finish_rotation(u1, __float_as_int(tq.y) & 3, sn.y, cm1.y, sc);
}

// One-part form in packed FP32: the phase summed first, then the quarter turn
// split off as in apply_turns (the 3D plane kernels, where keeping the two
// parts live costs register spills).  These kernels keep the Taylor series of
// sin to theta^9 and cos - 1 to theta^10 (truncation below 2e-9): with the
// shorter fitted polynomials their instruction schedule ran 2 % slower.
__device__ __forceinline__ void apply_turns2(cpx<float> &u0, cpx<float> &u1, float2 turns, float scale)
{
    const float2 tq = __ffma2_rn(bc2(4.0f), turns, bc2(kRoundMagic));
    const float2 q = __fadd2_rn(tq, bc2(-kRoundMagic));
    const float2 th = __fmul2_rn(__ffma2_rn(q, bc2(-0.25f), turns), bc2(6.28318530717958647692f));
    const float2 t2 = __fmul2_rn(th, th);
    float2 ps = __ffma2_rn(t2, bc2(1.0f / 362880.0f), bc2(-1.0f / 5040.0f));
    ps = __ffma2_rn(ps, t2, bc2(1.0f / 120.0f));
    ps = __ffma2_rn(ps, t2, bc2(-1.0f / 6.0f));
    float2 sn = __ffma2_rn(__fmul2_rn(th, t2), ps, th);
    float2 pc = __ffma2_rn(t2, bc2(-1.0f / 3628800.0f), bc2(1.0f / 40320.0f));
    pc = __ffma2_rn(pc, t2, bc2(-1.0f / 720.0f));
    pc = __ffma2_rn(pc, t2, bc2(1.0f / 24.0f));
    pc = __ffma2_rn(pc, t2, bc2(-0.5f));
    float2 cm1 = __fmul2_rn(t2, pc);
    sn = __fmul2_rn(sn, bc2(scale));
    cm1 = __fmul2_rn(cm1, bc2(scale));
    u0 = finish_rotation(u0, __float_as_int(tq.x) & 3, sn.x, cm1.x, scale);
    u1 = finish_rotation(u1, __float_as_int(tq.y) & 3, sn.y, cm1.y, scale);
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

// the perturbation V_I(x) of one axis; the accurate cosf (the fast intrinsic's
// error grows with the argument, and |k x| reaches a few hundred radians on
// the wide batched boxes).  Kernels evaluate it once per grid point and keep
// it in shared memory, not per step.
__device__ __forceinline__ float vi_eval(int kind, float x, float k)
{
    if (kind == HFS_VI_X4) {
        const float x2 = x * x;
        return x2 * x2;
    }
    if (kind == HFS_VI_COS) return cosf(k * x);
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
