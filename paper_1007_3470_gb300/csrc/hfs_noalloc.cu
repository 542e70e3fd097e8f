// hfs_noalloc.cu -- hfs_step1d_noalloc(): the batched 1D split step for
// callers that cannot allocate device memory.
//
// The context-based API needs a caller-provided workspace.  Some callers
// cannot provide one: code running where cudaMalloc is not allowed or not
// wanted (inside a memory-pool or allocator callback, under a strict
// device-memory budget fixed at start-up, or in a host library that only
// receives a device pointer to the state).  This entry point takes only the
// state and the problem description and keeps all of its scratch (instance
// table, work list, twiddle tables, per-stage coefficients and phase
// records, work ticket, status word) in one file-scope __device__ array of
// fixed size that every GPU loading the library holds until process exit.
#include <math.h>
#include <string.h>

#include <algorithm>
#include <mutex>

#include "hfs.h"
#include "hfs_internal.cuh"
#include "hfs_sched.h"

namespace hfs {
namespace {

constexpr int kNoAllocMaxInstances = HFS_NOALLOC_MAX_INSTANCES;
constexpr int kNoAllocChunk = 16;   // time steps per schedule chunk
constexpr int kNoAllocMaxStages = 6;  // largest built-in composition (SRKN_6 4)
constexpr size_t kNoAllocBytes = HFS_NOALLOC_SCRATCH_BYTES;

constexpr size_t al256(size_t v) { return (v + 255) / 256 * 256; }
// layout of the scratch array
constexpr size_t kOffStatus = 0;
constexpr size_t kOffTicket = kOffStatus + 256;
constexpr size_t kOffTime = kOffTicket + 256;
constexpr size_t kOffInst = kOffTime + 256;
constexpr size_t kOffOrder = kOffInst + al256(sizeof(DevInst) * kNoAllocMaxInstances);
constexpr size_t kOffWork = kOffOrder + al256(sizeof(int32_t) * kNoAllocMaxInstances);
constexpr size_t kOffTwf = kOffWork + al256(sizeof(WorkItem) * kNoAllocMaxInstances);
constexpr size_t kOffTwd = kOffTwf + al256(sizeof(float4) * kTwiddleTotal);
constexpr size_t kOffFge = kOffTwd + al256(sizeof(double2) * kTwiddleTotal);
constexpr size_t kOffNodes = kOffFge + al256(sizeof(StageFGE) * kNoAllocMaxInstances * kNoAllocChunk * kNoAllocMaxStages);
constexpr size_t kOffRec = kOffNodes + al256(3 * sizeof(double) * kNoAllocChunk * kNoAllocMaxStages);
constexpr size_t kRecMax = sizeof(RecD) > sizeof(RecF) ? sizeof(RecD) : sizeof(RecF);
constexpr size_t kEnd = kOffRec + al256(kRecMax * kNoAllocMaxInstances * (kNoAllocChunk * kNoAllocMaxStages + 1));
static_assert(kEnd <= kNoAllocBytes, "scratch layout exceeds HFS_NOALLOC_SCRATCH_BYTES");

// The scratch.  In host code `g_noalloc_scratch` names a host-side stand-in,
// not the device array: its device address comes from cudaGetSymbolAddress.
static __device__ __align__(256) unsigned char g_noalloc_scratch[kNoAllocBytes];

constexpr int kMaxDevices = 64;
std::mutex g_setup_mutex;
unsigned char *g_scratch_ptr[kMaxDevices] = {};  // device address per device, set once

// Once per device, with that device current: resolve the array's device
// address and fill the twiddle tables (they are never overwritten later).
int device_scratch(cudaStream_t st, unsigned char **out)
{
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= kMaxDevices) return HFS_ERR_CUDA;
    std::lock_guard<std::mutex> lock(g_setup_mutex);
    if (!g_scratch_ptr[dev]) {
        void *p = nullptr;
        if (cudaGetSymbolAddress(&p, g_noalloc_scratch) != cudaSuccess || !p) return HFS_ERR_CUDA;
        unsigned char *base = static_cast<unsigned char *>(p);
        if (launch_twiddles(base + kOffTwf, base + kOffTwd, st) != cudaSuccess) return HFS_ERR_CUDA;
        if (cudaStreamSynchronize(st) != cudaSuccess) return HFS_ERR_CUDA;
        g_scratch_ptr[dev] = base;
    }
    *out = g_scratch_ptr[dev];
    return HFS_OK;
}

// host staging of the tables (per host thread, fixed size)
thread_local DevInst t_inst[kNoAllocMaxInstances];
thread_local int32_t t_order[kNoAllocMaxInstances];
thread_local WorkItem t_work[kNoAllocMaxInstances];

bool pow2(int n) { return n > 0 && (n & (n - 1)) == 0; }

}  // namespace
}  // namespace hfs

using namespace hfs;

extern "C" int hfs_step1d_noalloc(void *psi, int precision, const hfs_instance *inst, int64_t count, int split,
                                  int ho_flow, int composition, double dt, double t0, int64_t nsteps,
                                  void *stream, int wait)
{
    // ---- host-side validation -----------------------------------------
    if (!psi || !inst || count < 1 || nsteps < 0) return HFS_ERR_INVALID_ARG;
    if (count > kNoAllocMaxInstances) return HFS_ERR_WORKSPACE;
    if (precision != HFS_C64 && precision != HFS_C128) return HFS_ERR_INVALID_ARG;
    if ((uintptr_t)psi % (precision == HFS_C128 ? 16 : 8)) return HFS_ERR_ALIGNMENT;
    if (split != HFS_SPLIT_HO && split != HFS_SPLIT_FOURIER) return HFS_ERR_INVALID_ARG;
    if (ho_flow < HFS_FLOW_LEMMA2 || ho_flow > HFS_FLOW_M6) return HFS_ERR_INVALID_ARG;
    if (!(dt != 0.0) || !isfinite(dt) || !isfinite(t0)) return HFS_ERR_INVALID_ARG;
    SchedConst sc{};
    if (composition_fixed(composition, sc.a, sc.b, &sc.m) || sc.m > kNoAllocMaxStages) return HFS_ERR_INVALID_ARG;
    sc.split = split;
    sc.flow = ho_flow;
    sc.h = dt;
    double cum = 0.0, amax = 0.0;
    for (int i = 0; i < sc.m; ++i) {
        sc.cuma[i] = cum;
        cum += sc.a[i];
        amax = std::max(amax, fabs(sc.a[i] * dt));
    }
    int64_t off = 0;
    for (int64_t i = 0; i < count; ++i) {
        const hfs_instance &p = inst[i];
        const int n = p.n[0];
        if (!pow2(n) || n < 128 || n > 4096) return HFS_ERR_UNSUPPORTED;
        if (!(p.hi[0] > p.lo[0]) || !(p.mu > 0.0) || p.omega_law < 0 || p.omega_law > 3 || p.vi_kind < 0 ||
            p.vi_kind > 2)
            return HFS_ERR_INVALID_ARG;
        if (split == HFS_SPLIT_HO && !(amax * omega_bound(p, t0, t0 + (double)nsteps * dt) < M_PI))
            return HFS_ERR_STEP_TOO_LARGE;
        DevInst &d = t_inst[i];
        memset(&d, 0, sizeof(d));
        d.off = off;
        d.n[0] = n;
        d.n[1] = d.n[2] = 1;
        d.plan = size_class(n);
        d.len[0] = p.hi[0] - p.lo[0];
        d.dx[0] = d.len[0] / n;
        d.xc[0] = 0.5 * (p.lo[0] + p.hi[0]);
        d.mu = p.mu;
        d.omega_law = p.omega_law;
        d.vi_kind = p.vi_kind;
        d.w0 = p.w0;
        for (int a = 0; a < 3; ++a) {
            d.law[a] = p.law[a];
            d.axis_scale[a] = 1.0;
        }
        d.eps = p.eps;
        d.vi_k = p.vi_k;
        d.sigma = p.sigma;
        set_1d_fp32_params(d);
        off += n;
    }
    if (nsteps == 0) return HFS_OK;

    // ---- work list: sorted by decreasing N, 256/T instances per item -----
    for (int64_t i = 0; i < count; ++i) t_order[i] = (int32_t)i;
    std::stable_sort(t_order, t_order + count, [](int32_t x, int32_t y) { return t_inst[x].n[0] > t_inst[y].n[0]; });
    int32_t nwork = 0;
    for (int64_t i = 0; i < count;) {
        const int n = t_inst[t_order[i]].n[0];
        const int per = kCtaThreads / (n / 16);
        int64_t j = i;
        while (j < count && j - i < per && t_inst[t_order[j]].n[0] == n) ++j;
        t_work[nwork].first = (int32_t)i;
        t_work[nwork].count = (int32_t)(j - i);
        t_work[nwork].plan = plan_id(n, 16);
        t_work[nwork].pad = 0;
        ++nwork;
        i = j;
    }

    // ---- device side ------------------------------------------------------
    cudaStream_t st = (cudaStream_t)stream;
    (void)cudaGetLastError();
    unsigned char *base = nullptr;
    int s = device_scratch(st, &base);
    if (s) return s;
    const bool fp64 = precision == HFS_C128;
    unsigned *status = reinterpret_cast<unsigned *>(base + kOffStatus);
    unsigned *ticket = reinterpret_cast<unsigned *>(base + kOffTicket);
    double *tdev = reinterpret_cast<double *>(base + kOffTime);
    DevInst *dinst = reinterpret_cast<DevInst *>(base + kOffInst);
    StageFGE *fge = reinterpret_cast<StageFGE *>(base + kOffFge);
    void *rec = base + kOffRec;
#define HFS_NA_CK(expr)                                                                                           \
    do {                                                                                                          \
        if ((expr) != cudaSuccess) return HFS_ERR_CUDA;                                                           \
    } while (0)
    // the array keeps the previous call's contents: reset what must start at zero
    HFS_NA_CK(cudaMemsetAsync(status, 0, sizeof(unsigned), st));
    HFS_NA_CK(cudaMemcpyAsync(dinst, t_inst, sizeof(DevInst) * count, cudaMemcpyHostToDevice, st));
    HFS_NA_CK(cudaMemcpyAsync(base + kOffOrder, t_order, sizeof(int32_t) * count, cudaMemcpyHostToDevice, st));
    HFS_NA_CK(cudaMemcpyAsync(base + kOffWork, t_work, sizeof(WorkItem) * nwork, cudaMemcpyHostToDevice, st));
    HFS_NA_CK(launch_set_time(tdev, t0, st));
    int dev = 0, sms = 0;
    HFS_NA_CK(cudaGetDevice(&dev));
    HFS_NA_CK(cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev));
    const int variant = step1d_variant(inst, count);
    const int grid = std::max(1, std::min(nwork, sms * step1d_ctas_per_sm(fp64, variant)));
    for (int64_t done = 0; done < nsteps; done += kNoAllocChunk) {
        const int64_t S = std::min<int64_t>(kNoAllocChunk, nsteps - done);
        const int64_t nstage = S * sc.m;
        const double toff = (double)done * dt;
        if (split == HFS_SPLIT_HO)
            HFS_NA_CK(launch_stage_flow(dinst, count, 1, sc, tdev, toff, nstage, uniform_law(inst, count),
                                        law_shared(inst, count), base + kOffNodes, fge, status, st));
        HFS_NA_CK(launch_records1d(fp64, dinst, count, sc, tdev, toff, nstage, fge, rec, status, st));
        Step1DArgs a{};
        a.psi = psi;
        a.inst = dinst;
        a.order = reinterpret_cast<const int32_t *>(base + kOffOrder);
        a.work = reinterpret_cast<const WorkItem *>(base + kOffWork);
        a.nwork = nwork;
        a.rec = rec;
        a.nrec = nstage + 1;
        a.j0 = 0;
        a.j1 = nstage;
        a.final_x = 1;
        a.tw = fp64 ? (const void *)(base + kOffTwd) : (const void *)(base + kOffTwf);
        a.ticket = ticket;
        a.status = status;
        HFS_NA_CK(cudaMemsetAsync(ticket, 0, sizeof(unsigned), st));
        HFS_NA_CK(launch_step1d(fp64, variant, a, grid, st));
    }
    if (wait) {
        unsigned h_status = 0;
        HFS_NA_CK(cudaMemcpyAsync(&h_status, status, sizeof(unsigned), cudaMemcpyDeviceToHost, st));
        HFS_NA_CK(cudaStreamSynchronize(st));
        if (h_status & ST_NONFINITE) return HFS_ERR_NONFINITE;
        if (h_status & ST_BADPLAN) return HFS_ERR_UNSUPPORTED;
    }
#undef HFS_NA_CK
    return HFS_OK;
}
