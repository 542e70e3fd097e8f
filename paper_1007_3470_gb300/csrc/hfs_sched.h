// hfs_sched.h -- schedule constants, 3D record layouts and the launchers of
// hfs_schedule.cu (library-internal).
#pragma once

#include "hfs_internal.cuh"

namespace hfs {

constexpr int kMaxStages = 16;

// composition passed by value to the schedule kernels
struct SchedConst {
    int split, flow, m, pad;
    double h;
    double a[kMaxStages];
    double b[kMaxStages + 1];
    double cuma[kMaxStages];  // a_1 + ... + a_{i-1}
};

// 3D sub-stage record (symmetric boxes): per-axis kick K2 and drift G
struct alignas(16) Rec3F {
    float k2[3], k2lo[3], g[3], glo[3];
    float sb2pi, pad[3];
};
struct alignas(16) Rec3D {
    double k2[3], k2lo[3], g[3], glo[3];
    double sb2pi, pad;
};

// uniform_law: the HFS_OMEGA_* law shared by all instances, or -1 for a mixed
// batch; shared: the law parameters are shared too (law_shared), so the trap's
// shape factors are evaluated once per stage into `nodes` (law_nodes_bytes)
cudaError_t launch_stage_flow(const DevInst *inst, int64_t count, int dim, const SchedConst &sc, const double *t_dev,
                              double t_off, int64_t nstage, int uniform_law, bool shared, void *nodes,
                              StageFGE *out, unsigned *status, cudaStream_t st);
// the law shared by every instance of inst[0..count), or -1
int uniform_law(const hfs_instance *inst, int64_t count);
// every instance has the same law and law parameters
bool law_shared(const hfs_instance *inst, int64_t count);
size_t law_nodes_bytes(int64_t nstage);
cudaError_t launch_records1d(bool fp64, const DevInst *inst, int64_t count, const SchedConst &sc, const double *t_dev,
                             double t_off, int64_t nstage, const StageFGE *fge, void *rec, unsigned *status,
                             cudaStream_t st);
cudaError_t launch_records3d(bool fp64, const DevInst *inst, const SchedConst &sc, const double *t_dev, double t_off,
                             int64_t nstage, const StageFGE *fge, void *rec, unsigned *status, cudaStream_t st);
cudaError_t launch_set_time(double *t_dev, double t, cudaStream_t st);
cudaError_t launch_advance_time(double *t_dev, double dt, cudaStream_t st);

// 1D step and diagnostics (hfs_step1d.cu)
struct Step1DArgs {
    void *psi;                      // cpx<R>*
    const DevInst *inst;
    const int32_t *order;           // sorted position -> instance index
    const WorkItem *work;
    int32_t nwork;
    const void *rec;                // RecF* / RecD*, instance-major, nrec per instance
    int64_t nrec;                   // records per instance (nstage + 1)
    int64_t j0, j1;                 // sub-stages [j0, j1) of this launch: X_j then D_{j+1}
    int32_t final_x;                // apply X_{j1} at the end (last launch of a chunk)
    const void *tw;                 // twiddle table (cpx<R>)
    unsigned *ticket;
    unsigned *status;
    const void *tw2;                // plain FP32 twiddle table (float2), read with the norm projection
    float *norm_target;             // per instance: target sum |u|^2 of the norm projection
    int32_t proj;                   // PROJ_OFF, PROJ_SET (first launch of a call), PROJ_USE
    int32_t streaming;              // fewer sub-stages per launch than the chunk holds (streaming mode)
};
enum : int32_t { PROJ_OFF = 0, PROJ_SET = 1, PROJ_USE = 2 };
// variant: HFS_VI_* when every instance has that perturbation kind and a box
// symmetric about 0 (FP32 only; from step1d_variant), -1 for the generic kernel
// wide: the work list holds plans of the wide set (plan_is_wide; FP32 only)
// priority: scheduling priority of the launch (0: the stream's)
cudaError_t launch_step1d(bool fp64, int variant, const Step1DArgs &a, int grid, cudaStream_t st, bool wide = false,
                          int priority = 0);
int step1d_ctas_per_sm(bool fp64, int variant, bool wide = false);
int step1d_variant(const hfs_instance *inst, int64_t count);
size_t step1d_smem_bytes(bool fp64);

struct Diag1DArgs {
    const void *psi;
    const DevInst *inst;
    const int32_t *order;
    const WorkItem *work;
    int32_t nwork;
    const void *tw;
    const double *t_dev;
    double *out;  // [count][2]: norm, energy
    unsigned *ticket;
};
cudaError_t launch_diag1d(bool fp64, const Diag1DArgs &a, int grid, cudaStream_t st);

cudaError_t launch_twiddles(void *tw_f, void *tw_d, cudaStream_t st);
// the plain FP32 table (same layout, the FP64 value rounded to float2)
cudaError_t launch_twiddles_plain(void *tw_p, cudaStream_t st);

// host helpers shared by the entry points (hfs_api.cu)
int composition_fixed(int comp, double *a, double *b, int *m);
double omega_bound(const hfs_instance &p, double t0, double t1);

}  // namespace hfs
