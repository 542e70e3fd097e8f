// hfs_step3d.h -- the 3D split step (diagonal trap x^T M(t) x, separable
// per axis) and its diagnostics (library-internal).
#pragma once

#include "hfs_internal.cuh"

namespace hfs {

struct Step3DArgs {
    void *psi;  // cpx<R>[n^3], x fastest
    const DevInst *inst;
    const void *rec;  // Rec3F / Rec3D [nstage + 1]
    int64_t nstage;
    const void *tw;
    unsigned *status;
    int n;   // points per axis
    int vi;  // perturbation kind in effect (HFS_VI_NONE where eps = 0)
    int dft_tc;  // complex64, n = 64 / 128: first z-pass radix-16 stages on the tensor cores
    // norm projection (complex64, n = 128): plain FP32 twiddles (float2), the
    // per-sub-stage sums of |u|^2 (three FP64 slots, zeroed by the host at
    // each chunk start), the call's target sum, PROJ_OFF / PROJ_SET / PROJ_USE
    const void *tw2;
    double *nsum;
    double *ntarget;
    int proj;
};

struct Diag3DArgs {
    const void *psi;
    const DevInst *inst;
    const void *tw;
    const double *t_dev;
    double *out;  // [2]: norm, energy
    int n;
};

bool step3d_supported(int nx, int ny, int nz);
cudaError_t launch_step3d(bool fp64, const Step3DArgs &a, cudaStream_t st);
cudaError_t launch_diag3d(bool fp64, const Diag3DArgs &a, cudaStream_t st);

}  // namespace hfs
