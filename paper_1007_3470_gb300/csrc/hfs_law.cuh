// hfs_law.cuh -- the trap law omega^2(t) of Eq. GP1b (device, FP64).
//
// Every law is omega^2(t) = omega0^2 S(t) with a shape factor S that depends
// only on the law and its parameters: a batch whose instances share those
// evaluates S once per time node (law_factor*), each instance multiplies by
// its own omega0^2 (and the axis scale^2 in 3D).
#pragma once

#include "hfs_internal.cuh"

namespace hfs {

// LAW >= 0: the law is known at compile time (every instance of a batch uses
// it); LAW = -1 reads it from the instance
template <int LAW = -1> __device__ __forceinline__ double law_factor(const DevInst &p, double t)
{
    double u;
    switch (LAW >= 0 ? LAW : p.omega_law) {
    case HFS_OMEGA_CONST:
        return 1.0;
    case HFS_OMEGA_SIN:  // omega = omega0 (1 + A sin(W t + phi))
        u = 1.0 + p.law[0] * sin(fma(p.law[1], t, p.law[2]));
        return u * u;
    case HFS_OMEGA_COS_SQ:  // omega^2 = omega0^2 (1 + A cos(W t))
        return 1.0 + p.law[0] * cos(p.law[1] * t);
    case HFS_OMEGA_PULSE: {  // omega = omega0 (1 + A t / cosh^2(B (t - t_c)))
        const double ch = cosh(p.law[1] * (t - p.law[2]));
        u = 1.0 + p.law[0] * t / (ch * ch);
        return u * u;
    }
    default:
        return nan("");
    }
}

template <int LAW = -1> __device__ __forceinline__ double law_omega2(const DevInst &p, double t)
{
    return p.w0 * p.w0 * law_factor<LAW>(p, t);
}

template <int LAW = -1> __device__ __forceinline__ double axis_omega2(const DevInst &p, int dim, int axis, double t)
{
    const double c = (dim == 1) ? 1.0 : p.axis_scale[axis];
    return c * c * law_omega2<LAW>(p, t);
}

// sin and cos of a small angle (|d| <= 1/32) by their Taylor series (the
// first omitted terms are below 1e-21), otherwise by sincos
__device__ __forceinline__ void sincos_small(double d, double &s, double &c)
{
    if (fabs(d) <= 0.03125) {
        const double d2 = d * d;
        s = d * (1.0 - d2 * (1.0 / 6.0) * (1.0 - d2 * (1.0 / 20.0) * (1.0 - d2 * (1.0 / 42.0) * (1.0 - d2 * (1.0 / 72.0)))));
        c = 1.0 - d2 * 0.5 * (1.0 - d2 * (1.0 / 12.0) * (1.0 - d2 * (1.0 / 30.0) * (1.0 - d2 * (1.0 / 56.0))));
    } else {
        sincos(d, &s, &c);
    }
}

// S at the two symmetric nodes tm - d and tm + d (the Gauss nodes of a
// stage): the periodic laws take both from one sincos of the midpoint
// argument, sin(th -+ de) = sin th cos de -+ cos th sin de
template <int LAW = -1>
__device__ __forceinline__ void law_factor_pair(const DevInst &p, double tm, double d, double &s1, double &s2)
{
    const int law = LAW >= 0 ? LAW : p.omega_law;
    if (law == HFS_OMEGA_SIN) {
        double st, ct, sd, cd;
        sincos(fma(p.law[1], tm, p.law[2]), &st, &ct);
        sincos_small(p.law[1] * d, sd, cd);
        const double a = st * cd, b = ct * sd;
        const double u1 = 1.0 + p.law[0] * (a - b), u2 = 1.0 + p.law[0] * (a + b);
        s1 = u1 * u1;
        s2 = u2 * u2;
    } else if (law == HFS_OMEGA_COS_SQ) {
        double st, ct, sd, cd;
        sincos(p.law[1] * tm, &st, &ct);
        sincos_small(p.law[1] * d, sd, cd);
        const double a = ct * cd, b = st * sd;
        s1 = 1.0 + p.law[0] * (a + b);
        s2 = 1.0 + p.law[0] * (a - b);
    } else {
        s1 = law_factor<LAW>(p, tm - d);
        s2 = law_factor<LAW>(p, tm + d);
    }
}

}  // namespace hfs
