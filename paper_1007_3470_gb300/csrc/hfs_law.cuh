// hfs_law.cuh -- the trap law omega^2(t) of Eq. GP1b (device, FP64).
#pragma once

#include "hfs_internal.cuh"

namespace hfs {

__device__ __forceinline__ double law_omega2(const DevInst &p, double t)
{
    double w;
    switch (p.omega_law) {
    case HFS_OMEGA_CONST:
        return p.w0 * p.w0;
    case HFS_OMEGA_SIN:
        w = p.w0 * (1.0 + p.law[0] * sin(fma(p.law[1], t, p.law[2])));
        return w * w;
    case HFS_OMEGA_COS_SQ:
        return p.w0 * p.w0 * (1.0 + p.law[0] * cos(p.law[1] * t));
    case HFS_OMEGA_PULSE: {
        const double ch = cosh(p.law[1] * (t - p.law[2]));
        w = p.w0 * (1.0 + p.law[0] * t / (ch * ch));
        return w * w;
    }
    default:
        return nan("");
    }
}

__device__ __forceinline__ double axis_omega2(const DevInst &p, int dim, int axis, double t)
{
    const double c = (dim == 1) ? 1.0 : p.axis_scale[axis];
    return c * c * law_omega2(p, t);
}

}  // namespace hfs
