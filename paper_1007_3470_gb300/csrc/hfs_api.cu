// hfs_api.cu -- the C ABI of include/hfs.h: contexts, caller-owned buffer
// binding, host-side validation, chunked schedule + step launches, CUDA
// graph capture, diagnostics and the 1D plan autotuner.
#include <math.h>
#include <string.h>

#include <stdio.h>

#include <algorithm>
#include <map>
#include <new>
#include <numeric>
#include <string>
#include <vector>

#include <nvtx3/nvToolsExt.h>

#include "hfs.h"
#include "hfs_internal.cuh"
#include "hfs_sched.h"
#include "hfs_step3d.h"

using namespace hfs;

namespace {
// NVTX range around an entry point (a no-op unless a profiler is attached)
struct NvtxRange {
    explicit NvtxRange(const char *name) { nvtxRangePushA(name); }
    ~NvtxRange() { nvtxRangePop(); }
    NvtxRange(const NvtxRange &) = delete;
    NvtxRange &operator=(const NvtxRange &) = delete;
};
}  // namespace

namespace hfs {

// BAB compositions into fixed arrays (m A-stages, m + 1 B-stages)
int composition_fixed(int comp, double *a, double *b, int *m)
{
    // BAB compositions, b_1 applied first (Eq. LeapFrogB; Table 1)
    switch (comp) {
    case HFS_COMP_STRANG:
        a[0] = 1.0; *m = 1;
        b[0] = 0.5; b[1] = 0.5;
        return 0;
    case HFS_COMP_SRKN6_4: {
        const double b1 = 0.0829844064174052, b2 = 0.396309801498368, b3 = -0.0390563049223486;
        const double b4 = 1.0 - 2.0 * (b1 + b2 + b3);
        const double a1 = 0.245298957184271, a2 = 0.604872665711080, a3 = 0.5 - (a1 + a2);
        a[0] = a1; a[1] = a2; a[2] = a3; a[3] = a3; a[4] = a2; a[5] = a1; *m = 6;
        b[0] = b1; b[1] = b2; b[2] = b3; b[3] = b4; b[4] = b3; b[5] = b2; b[6] = b1;
        return 0;
    }
    case HFS_COMP_NI4_82: {
        // Table 1 prints b_2 = 49/18; the (8,2) method's weights are the
        // Lobatto weights 1/20, 49/180, 16/45, so b_2 = 49/180.
        const double b1 = 1.0 / 20.0, b2 = 49.0 / 180.0, b3 = 1.0 - 2.0 * (b1 + b2);
        const double a1 = 0.5 - sqrt(3.0 / 28.0), a2 = 0.5 - a1;
        a[0] = a1; a[1] = a2; a[2] = a2; a[3] = a1; *m = 4;
        b[0] = b1; b[1] = b2; b[2] = b3; b[3] = b2; b[4] = b1;
        return 0;
    }
    case HFS_COMP_NI5_84: {
        const double b1 = 0.811862738544516, b2 = -0.677480399532169, b3 = 0.5 - (b1 + b2);
        const double a1 = -0.00758691311877447, a2 = 0.317218277973169, a3 = 1.0 - 2.0 * (a1 + a2);
        a[0] = a1; a[1] = a2; a[2] = a3; a[3] = a2; a[4] = a1; *m = 5;
        b[0] = b1; b[1] = b2; b[2] = b3; b[3] = b3; b[4] = b2; b[5] = b1;
        return 0;
    }
    default:
        return -1;
    }
}

// upper bound of omega over [t0, t1] for the validity check
double omega_bound(const hfs_instance &p, double t0, double t1)
{
    const double aw = fabs(p.w0);
    switch (p.omega_law) {
    case HFS_OMEGA_CONST:
        return aw;
    case HFS_OMEGA_SIN:
        return aw * (1.0 + fabs(p.law[0]));
    case HFS_OMEGA_COS_SQ:
        return aw * sqrt(1.0 + fabs(p.law[0]));
    case HFS_OMEGA_PULSE:
        return aw * (1.0 + fabs(p.law[0]) * std::max(fabs(t0), fabs(t1)));
    default:
        return INFINITY;
    }
}

}  // namespace hfs

namespace {

struct Layout {
    size_t status, ticket, tdev, inst, order, work, twf, twd, twp, fge, nodes, rec, diag, norm, nsum3, rec2, total;
};

inline size_t align_up(size_t v, size_t a) { return (v + a - 1) / a * a; }

}  // namespace

struct hfs_ctx_s {
    int dim = 1, precision = HFS_C64;
    int64_t count = 0;
    std::vector<hfs_instance> inst;
    std::vector<DevInst> dinst;
    std::vector<int64_t> offsets;
    int64_t elems = 0;
    // 1D plans per size class: elements per thread (4, 8, 16) and the
    // alternative radix order (16 only); CTAs per SM of the step grid (0: as
    // many as fit)
    int ept[kNumSizes] = {16, 16, 16, 16, 16, 16};
    bool alt[kNumSizes] = {false, false, false, false, false, false};
    int ctas_per_sm = 0;
    // trap law shared by every instance (HFS_OMEGA_*), -1 for a mixed batch,
    // and whether its parameters are shared too
    int law = -1;
    bool law_shared = false;
    // specialised 1D step kernel (step1d_variant), -1 for the generic one
    int variant = -1;
    std::vector<int32_t> order;  // sorted position -> instance
    std::vector<WorkItem> work;
    // schedule
    bool have_sched = false;
    SchedConst sc{};
    int composition = HFS_COMP_STRANG;
    // execution
    int mode = HFS_MODE_RESIDENT, spl = 1;
    bool graphs = false;
    bool norm_projection = false;  // 1D complex64: hfs_set_norm_projection
    int dft_engine = HFS_DFT_SIMT;  // 3D complex64: hfs_set_dft_engine
    cudaStream_t stream = nullptr;
    // bound buffers
    void *psi = nullptr;
    unsigned char *work_base = nullptr;
    size_t work_bytes = 0;
    int64_t chunk = 0;
    Layout lay{};
    double t = 0.0;
    int sm_count = 0;
    // graph cache keyed by graph_key (steps per call and schedule-reuse plan)
    std::map<int64_t, cudaGraphExec_t> graphs_by_n;
    uint64_t version = 0;  // bumps invalidate cached graphs
    std::vector<double> diag_host;
    // profiling events around the fused step kernels
    bool profiling = false, prof_valid = false;
    cudaEvent_t kev[2] = {nullptr, nullptr};
    // 1D schedule reuse (hfs_set_schedule_reuse): two record buffers, each
    // tagged with the call it holds (start time, steps, context version); the
    // next call's records are computed on an auxiliary stream, in a branch
    // parallel to the step kernel, which is launched at the highest priority
    struct RecSlot {
        bool valid = false;
        double t0 = 0.0;
        int64_t nsteps = 0;
        uint64_t version = 0;
    };
    bool sched_reuse = false;
    RecSlot slot[2];
    cudaStream_t aux = nullptr;
    cudaEvent_t fork_ev = nullptr, join_ev = nullptr;
    int prio_high = 0;
};

namespace {

#define CK(expr)                                                                                                  \
    do {                                                                                                          \
        cudaError_t _e = (expr);                                                                                  \
        if (_e != cudaSuccess) return HFS_ERR_CUDA;                                                               \
    } while (0)

bool is_pow2(int n) { return n > 0 && (n & (n - 1)) == 0; }

int composition_coeffs(int comp, std::vector<double> &a, std::vector<double> &b)
{
    double av[kMaxStages], bv[kMaxStages + 1];
    int m = 0;
    if (hfs::composition_fixed(comp, av, bv, &m)) return -1;
    a.assign(av, av + m);
    b.assign(bv, bv + m + 1);
    return 0;
}

Layout make_layout(const hfs_ctx_s *c, int64_t chunk)
{
    Layout L{};
    size_t o = 0;
    auto take = [&](size_t bytes) {
        size_t at = o;
        o = align_up(o + bytes, 256);
        return at;
    };
    const int m = std::max(c->have_sched ? c->sc.m : 0, 6);
    const int64_t nstage = chunk * m;
    const size_t recsz = (c->dim == 1) ? (c->precision == HFS_C128 ? sizeof(RecD) : sizeof(RecF))
                                       : (c->precision == HFS_C128 ? sizeof(Rec3D) : sizeof(Rec3F));
    L.status = take(sizeof(unsigned));
    L.ticket = take(sizeof(unsigned));
    L.tdev = take(sizeof(double));
    L.inst = take(sizeof(DevInst) * c->count);
    L.order = take(sizeof(int32_t) * c->count);
    L.work = take(sizeof(WorkItem) * std::max<int64_t>(c->count, 1));
    L.twf = take(sizeof(float4) * kTwiddleTotal);
    L.twd = take(sizeof(cpx<double>) * kTwiddleTotal);
    L.twp = take(sizeof(float2) * kTwiddleTotal);
    L.fge = take(sizeof(StageFGE) * c->count * nstage * c->dim);
    L.nodes = take(law_nodes_bytes(nstage));
    L.rec = take(recsz * c->count * (nstage + 1));
    L.diag = take(sizeof(double) * 2 * std::max<int64_t>(c->count, 1));
    L.norm = take(sizeof(float) * std::max<int64_t>(c->count, 1));
    L.nsum3 = take(4 * sizeof(double));  // 3D projection: three sum slots and the target
    // the second record buffer of the schedule reuse, last so that the other
    // offsets do not depend on it
    L.rec2 = (c->sched_reuse && c->dim == 1) ? take(recsz * c->count * (nstage + 1)) : 0;
    L.total = o;
    return L;
}

template <typename T> T *wptr(hfs_ctx_s *c, size_t off) { return reinterpret_cast<T *>(c->work_base + off); }

void build_worklist(hfs_ctx_s *c)
{
    c->order.resize(c->count);
    std::iota(c->order.begin(), c->order.end(), 0);
    std::stable_sort(c->order.begin(), c->order.end(),
                     [&](int32_t x, int32_t y) { return c->inst[x].n[0] > c->inst[y].n[0]; });
    c->work.clear();
    int64_t i = 0;
    while (i < c->count) {
        const int n = c->inst[c->order[i]].n[0];
        const int e = c->ept[size_class(n)];
        const bool alt = c->alt[size_class(n)];
        const int per = kCtaThreads / (n / e);
        int64_t j = i;
        while (j < c->count && j - i < per && c->inst[c->order[j]].n[0] == n) ++j;
        WorkItem w;
        w.first = (int32_t)i;
        w.count = (int32_t)(j - i);
        w.plan = plan_id(n, e, alt);
        w.pad = 0;
        c->work.push_back(w);
        i = j;
    }
}

int upload_tables(hfs_ctx_s *c)
{
    CK(cudaMemcpyAsync(wptr<void>(c, c->lay.order), c->order.data(), sizeof(int32_t) * c->count,
                       cudaMemcpyHostToDevice, c->stream));
    CK(cudaMemcpyAsync(wptr<void>(c, c->lay.work), c->work.data(), sizeof(WorkItem) * c->work.size(),
                       cudaMemcpyHostToDevice, c->stream));
    return HFS_OK;
}

// events recorded while the stream is being captured must become event-record
// nodes of the graph (not fork/join markers), hence cudaEventRecordExternal
cudaError_t record_prof(hfs_ctx_s *c, int which)
{
    return c->graphs ? cudaEventRecordWithFlags(c->kev[which], c->stream, cudaEventRecordExternal)
                     : cudaEventRecord(c->kev[which], c->stream);
}

void drop_events(hfs_ctx_s *c)
{
    for (auto &e : c->kev)
        if (e) {
            cudaEventDestroy(e);
            e = nullptr;
        }
    c->prof_valid = false;
}

void drop_graphs(hfs_ctx_s *c)
{
    for (auto &kv : c->graphs_by_n) cudaGraphExecDestroy(kv.second);
    c->graphs_by_n.clear();
    c->version++;
}

// what one hfs_step() call does with the record buffers under schedule reuse:
// cur holds (or, with compute, receives) the records of this call; with
// prefetch the next call's records (start time t + nsteps h) go to nxt
struct ReusePlan {
    bool on = false, compute = true, prefetch = false;
    int cur = 0, nxt = 1;
};

ReusePlan plan_reuse(const hfs_ctx_s *c, int64_t nsteps)
{
    ReusePlan p;
    if (!(c->dim == 1 && c->sched_reuse && c->lay.rec2 != 0 && nsteps <= c->chunk)) return p;
    p.on = true;
    auto holds = [&](int k, double t0) {
        const hfs_ctx_s::RecSlot &r = c->slot[k];
        return r.valid && r.version == c->version && r.nsteps == nsteps && r.t0 == t0;
    };
    const double t1 = c->t + (double)nsteps * c->sc.h;
    p.cur = holds(0, c->t) ? 0 : holds(1, c->t) ? 1 : -1;
    p.compute = p.cur < 0;
    if (p.compute) p.cur = holds(0, t1) ? 1 : 0;  // keep a buffer that holds the next call's records
    p.nxt = 1 - p.cur;
    p.prefetch = !holds(p.nxt, t1);
    return p;
}

void commit_reuse(hfs_ctx_s *c, const ReusePlan &p, int64_t nsteps)
{
    if (!p.on) return;
    c->slot[p.cur] = {true, c->t, nsteps, c->version};
    if (p.prefetch) c->slot[p.nxt] = {true, c->t + (double)nsteps * c->sc.h, nsteps, c->version};
}

// graph cache key: the step count and the reuse plan
int64_t graph_key(int64_t nsteps, const ReusePlan &p)
{
    return nsteps * 16 + (p.on ? (p.cur * 4 + (p.compute ? 2 : 0) + (p.prefetch ? 1 : 0)) : 8);
}

int check_validity(const hfs_ctx_s *c, int64_t nsteps)
{
    if (c->sc.split != HFS_SPLIT_HO) return HFS_OK;
    double amax = 0.0;
    for (int i = 0; i < c->sc.m; ++i) amax = std::max(amax, fabs(c->sc.a[i] * c->sc.h));
    const double t0 = c->t, t1 = c->t + (double)nsteps * c->sc.h;
    for (int64_t i = 0; i < c->count; ++i) {
        const hfs_instance &p = c->inst[i];
        double scale = 1.0;
        if (c->dim == 3) scale = std::max({fabs(p.axis_scale[0]), fabs(p.axis_scale[1]), fabs(p.axis_scale[2])});
        const double om = omega_bound(p, t0, t1) * scale;
        if (!(amax * om < M_PI)) return HFS_ERR_STEP_TOO_LARGE;
    }
    return HFS_OK;
}

// the work list holds a plan of the wide set
bool worklist_wide(const hfs_ctx_s *c)
{
    for (const WorkItem &w : c->work)
        if (plan_is_wide(w.plan)) return true;
    return false;
}

// persistent grid of the 1D step: CTAs per SM (the tuned value, else as many
// as fit) times the SMs, at most one CTA per work item
int step_grid(const hfs_ctx_s *c, bool wide)
{
    const bool fp64 = c->precision == HFS_C128;
    const int fit = step1d_ctas_per_sm(fp64, c->variant, wide);
    const int per_sm = c->ctas_per_sm > 0 ? std::min(c->ctas_per_sm, fit) : fit;
    return std::max(1, std::min<int>((int)c->work.size(), c->sm_count * per_sm));
}

// enqueue nsteps steps (no graph logic); work list already uploaded; rp:
// the schedule-reuse plan of the call (plan_reuse; off by default)
int enqueue_steps(hfs_ctx_s *c, int64_t nsteps, const ReusePlan &rp = ReusePlan())
{
    (void)cudaGetLastError();  // a failed earlier runtime call must not be reported by the launches below
    const bool fp64 = c->precision == HFS_C128;
    const int m = c->sc.m;
    unsigned *status = wptr<unsigned>(c, c->lay.status);
    unsigned *ticket = wptr<unsigned>(c, c->lay.ticket);
    double *tdev = wptr<double>(c, c->lay.tdev);
    const DevInst *dinst = wptr<DevInst>(c, c->lay.inst);
    StageFGE *fge = wptr<StageFGE>(c, c->lay.fge);
    void *rec = wptr<void>(c, c->lay.rec);
    int64_t done = 0;
    while (done < nsteps) {
        const int64_t S = std::min(c->chunk, nsteps - done);
        const int64_t nstage = S * m;
        const double toff = (double)done * c->sc.h;
        // the FP64 schedule of sub-stages from time t + t_off into record buffer r
        auto schedule = [&](cudaStream_t st, double t_off, void *r) -> int {
            if (c->sc.split == HFS_SPLIT_HO)
                CK(launch_stage_flow(dinst, c->count, c->dim, c->sc, tdev, t_off, nstage, c->law, c->law_shared,
                                     wptr<void>(c, c->lay.nodes), fge, status, st));
            if (c->dim == 1) CK(launch_records1d(fp64, dinst, c->count, c->sc, tdev, t_off, nstage, fge, r, status, st));
            else CK(launch_records3d(fp64, dinst, c->sc, tdev, t_off, nstage, fge, r, status, st));
            return HFS_OK;
        };
        // under schedule reuse a call is one chunk (done = 0, S = nsteps)
        void *rec_now = (rp.on && rp.cur == 1) ? wptr<void>(c, c->lay.rec2) : rec;
        if (!rp.on || rp.compute) {
            const int s = schedule(c->stream, toff, rec_now);
            if (s) return s;
        }
        if (rp.on && rp.prefetch) {
            // the next call's records, parallel to the step kernel
            void *rec_next = rp.nxt == 1 ? wptr<void>(c, c->lay.rec2) : rec;
            CK(cudaEventRecord(c->fork_ev, c->stream));
            CK(cudaStreamWaitEvent(c->aux, c->fork_ev, 0));
            const int s = schedule(c->aux, (double)nsteps * c->sc.h, rec_next);
            if (s) return s;
            CK(cudaEventRecord(c->join_ev, c->aux));
        }
        if (c->dim == 1) {
            Step1DArgs a{};
            a.psi = c->psi;
            a.inst = dinst;
            a.order = wptr<int32_t>(c, c->lay.order);
            a.work = wptr<WorkItem>(c, c->lay.work);
            a.nwork = (int32_t)c->work.size();
            a.rec = rec_now;
            a.nrec = nstage + 1;
            a.tw = fp64 ? wptr<void>(c, c->lay.twd) : wptr<void>(c, c->lay.twf);
            a.ticket = ticket;
            a.status = status;
            a.norm_target = wptr<float>(c, c->lay.norm);
            a.tw2 = wptr<void>(c, c->lay.twp);
            a.streaming = c->mode != HFS_MODE_RESIDENT ? 1 : 0;
            const bool wide = worklist_wide(c);
            const int grid = step_grid(c, wide);
            const int64_t per = (c->mode == HFS_MODE_RESIDENT) ? S : std::max(1, c->spl);
            if (c->profiling && done == 0) CK(record_prof(c, 0));
            for (int64_t s0 = 0; s0 < S; s0 += per) {
                const int64_t s1 = std::min(S, s0 + per);
                a.j0 = s0 * m;
                a.j1 = s1 * m;
                a.final_x = (s1 == S) ? 1 : 0;
                // the first launch of the call records the norm it projects onto
                a.proj = !c->norm_projection ? PROJ_OFF : (done == 0 && s0 == 0) ? PROJ_SET : PROJ_USE;
                CK(cudaMemsetAsync(ticket, 0, sizeof(unsigned), c->stream));
                CK(launch_step1d(fp64, c->variant, a, grid, c->stream, wide, rp.prefetch ? c->prio_high : 0));
            }
            if (rp.on && rp.prefetch) CK(cudaStreamWaitEvent(c->stream, c->join_ev, 0));
            if (c->profiling && done + S >= nsteps) CK(record_prof(c, 1));
        } else {
            Step3DArgs a{};
            a.psi = c->psi;
            a.inst = dinst;
            a.rec = rec;
            a.nstage = nstage;
            a.tw = fp64 ? wptr<void>(c, c->lay.twd) : wptr<void>(c, c->lay.twf);
            a.status = status;
            a.n = c->inst[0].n[0];
            a.vi = c->inst[0].eps != 0.0 ? c->inst[0].vi_kind : HFS_VI_NONE;
            a.dft_tc = c->dft_engine == HFS_DFT_TENSOR_3XTF32 ? 1 : 0;
            a.tw2 = wptr<void>(c, c->lay.twp);
            a.nsum = wptr<double>(c, c->lay.nsum3);
            a.ntarget = a.nsum + 3;
            a.proj = !c->norm_projection ? PROJ_OFF : (done == 0 ? PROJ_SET : PROJ_USE);
            if (a.proj != PROJ_OFF) CK(cudaMemsetAsync(a.nsum, 0, 3 * sizeof(double), c->stream));
            if (c->profiling && done == 0) CK(record_prof(c, 0));
            CK(launch_step3d(fp64, a, c->stream));
            if (c->profiling && done + S >= nsteps) CK(record_prof(c, 1));
        }
        done += S;
    }
    CK(launch_advance_time(tdev, (double)nsteps * c->sc.h, c->stream));
    return HFS_OK;
}

int ready(const hfs_ctx_s *c)
{
    if (!c) return HFS_ERR_INVALID_ARG;
    if (!c->psi || !c->work_base) return HFS_ERR_NOT_READY;
    return HFS_OK;
}

}  // namespace

extern "C" {

const char *hfs_error_string(int s)
{
    switch (s) {
    case HFS_OK: return "ok";
    case HFS_ERR_INVALID_ARG: return "invalid argument";
    case HFS_ERR_UNSUPPORTED: return "unsupported grid size, dimension or precision";
    case HFS_ERR_STEP_TOO_LARGE: return "time step outside the validity of the chirp-kinetic-chirp decomposition";
    case HFS_ERR_CUDA: return "CUDA runtime error";
    case HFS_ERR_NONFINITE: return "non-finite value detected";
    case HFS_ERR_NOT_READY: return "buffers not bound or schedule not set";
    case HFS_ERR_ALIGNMENT: return "buffer not 256-byte aligned";
    case HFS_ERR_WORKSPACE: return "workspace too small";
    case HFS_ERR_DEVICE_TIMEOUT: return "bounded device wait ran out";
    default: return "unknown status";
    }
}

int hfs_create(hfs_ctx_t *out, int dim, int precision, const hfs_instance *inst, int64_t count)
{
    if (!out || !inst || count <= 0) return HFS_ERR_INVALID_ARG;
    *out = nullptr;
    if (precision != HFS_C64 && precision != HFS_C128) return HFS_ERR_INVALID_ARG;
    if (dim != 1 && dim != 3) return HFS_ERR_UNSUPPORTED;
    if (dim == 3 && count != 1) return HFS_ERR_UNSUPPORTED;
    if (count > (int64_t)1 << 30) return HFS_ERR_INVALID_ARG;
    hfs_ctx_s *c = new (std::nothrow) hfs_ctx_s();
    if (!c) return HFS_ERR_INVALID_ARG;
    c->dim = dim;
    c->precision = precision;
    c->count = count;
    c->inst.assign(inst, inst + count);
    c->law = uniform_law(inst, count);
    c->law_shared = law_shared(inst, count);
    c->variant = (dim == 1) ? step1d_variant(inst, count) : -1;
    c->dinst.resize(count);
    c->offsets.resize(count);
    int64_t off = 0;
    for (int64_t i = 0; i < count; ++i) {
        const hfs_instance &p = inst[i];
        DevInst &d = c->dinst[i];
        memset(&d, 0, sizeof(d));
        if (!(p.mu > 0.0) || p.omega_law < 0 || p.omega_law > 3 || p.vi_kind < 0 || p.vi_kind > 2) {
            delete c;
            return HFS_ERR_INVALID_ARG;
        }
        int64_t pts = 1;
        for (int a = 0; a < dim; ++a) {
            const int n = p.n[a];
            if (!is_pow2(n)) {
                delete c;
                return HFS_ERR_UNSUPPORTED;
            }
            if (dim == 1 && (n < 128 || n > 4096)) {
                delete c;
                return HFS_ERR_UNSUPPORTED;
            }
            if (!(p.hi[a] > p.lo[a])) {
                delete c;
                return HFS_ERR_INVALID_ARG;
            }
            d.n[a] = n;
            d.len[a] = p.hi[a] - p.lo[a];
            d.dx[a] = d.len[a] / n;
            d.xc[a] = 0.5 * (p.lo[a] + p.hi[a]);
            pts *= n;
        }
        if (dim == 3) {
            if (!step3d_supported(p.n[0], p.n[1], p.n[2]) || d.xc[0] != 0.0 || d.xc[1] != 0.0 || d.xc[2] != 0.0) {
                delete c;
                return HFS_ERR_UNSUPPORTED;
            }
        }
        d.off = off;
        c->offsets[i] = off;
        off += pts;
        d.mu = p.mu;
        d.omega_law = p.omega_law;
        d.vi_kind = p.vi_kind;
        d.w0 = p.w0;
        for (int a = 0; a < 3; ++a) {
            d.law[a] = p.law[a];
            d.axis_scale[a] = (dim == 3) ? p.axis_scale[a] : 1.0;
        }
        d.eps = p.eps;
        d.vi_k = p.vi_k;
        d.sigma = p.sigma;
        d.plan = (dim == 1) ? size_class(p.n[0]) : 0;
        if (dim == 1) set_1d_fp32_params(d);
    }
    c->elems = off;
    if (dim == 1) build_worklist(c);
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess ||
        cudaDeviceGetAttribute(&c->sm_count, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess) {
        delete c;
        return HFS_ERR_CUDA;
    }
    c->diag_host.resize(2 * count);
    *out = c;
    return HFS_OK;
}

void hfs_destroy(hfs_ctx_t c)
{
    if (!c) return;
    drop_graphs(c);
    drop_events(c);
    if (c->fork_ev) cudaEventDestroy(c->fork_ev);
    if (c->join_ev) cudaEventDestroy(c->join_ev);
    if (c->aux) cudaStreamDestroy(c->aux);
    delete c;
}

int hfs_set_profiling(hfs_ctx_t c, int enable)
{
    if (!c) return HFS_ERR_INVALID_ARG;
    drop_graphs(c);
    drop_events(c);
    c->profiling = enable != 0;
    if (c->profiling) {
        CK(cudaEventCreate(&c->kev[0]));
        CK(cudaEventCreate(&c->kev[1]));
    }
    return HFS_OK;
}

int hfs_last_step_kernel_ms(hfs_ctx_t c, float *ms)
{
    if (!c || !ms) return HFS_ERR_INVALID_ARG;
    if (!c->profiling || !c->prof_valid) return HFS_ERR_NOT_READY;
    CK(cudaEventSynchronize(c->kev[1]));
    CK(cudaEventElapsedTime(ms, c->kev[0], c->kev[1]));
    return HFS_OK;
}

int hfs_set_stream(hfs_ctx_t c, void *stream)
{
    if (!c) return HFS_ERR_INVALID_ARG;
    if (c->stream != (cudaStream_t)stream) drop_graphs(c);
    c->stream = (cudaStream_t)stream;
    return HFS_OK;
}

int hfs_state_size(hfs_ctx_t c, int64_t *elems, size_t *bytes)
{
    if (!c) return HFS_ERR_INVALID_ARG;
    const size_t es = (c->precision == HFS_C128) ? 16 : 8;
    if (elems) *elems = c->elems;
    if (bytes) *bytes = (size_t)c->elems * es;
    return HFS_OK;
}

int hfs_instance_offset(hfs_ctx_t c, int64_t i, int64_t *off)
{
    if (!c || !off || i < 0 || i >= c->count) return HFS_ERR_INVALID_ARG;
    *off = c->offsets[i];
    return HFS_OK;
}

int hfs_workspace_size(hfs_ctx_t c, int64_t chunk_steps, size_t *bytes)
{
    if (!c || !bytes || chunk_steps <= 0) return HFS_ERR_INVALID_ARG;
    *bytes = make_layout(c, chunk_steps).total;
    return HFS_OK;
}

int hfs_bind(hfs_ctx_t c, void *psi, void *work, size_t work_bytes, int64_t chunk_steps)
{
    if (!c || !psi || !work || chunk_steps <= 0) return HFS_ERR_INVALID_ARG;
    if (((uintptr_t)psi & 255) || ((uintptr_t)work & 255)) return HFS_ERR_ALIGNMENT;
    const Layout L = make_layout(c, chunk_steps);
    if (work_bytes < L.total) return HFS_ERR_WORKSPACE;
    drop_graphs(c);
    c->psi = psi;
    c->work_base = (unsigned char *)work;
    c->work_bytes = work_bytes;
    c->chunk = chunk_steps;
    c->lay = L;
    (void)cudaGetLastError();
    CK(cudaMemsetAsync(wptr<void>(c, L.status), 0, sizeof(unsigned), c->stream));
    CK(cudaMemcpyAsync(wptr<void>(c, L.inst), c->dinst.data(), sizeof(DevInst) * c->count, cudaMemcpyHostToDevice,
                       c->stream));
    if (c->dim == 1) {
        int s = upload_tables(c);
        if (s) return s;
    }
    CK(launch_twiddles(wptr<void>(c, L.twf), wptr<void>(c, L.twd), c->stream));
    CK(launch_twiddles_plain(wptr<void>(c, L.twp), c->stream));
    CK(launch_set_time(wptr<double>(c, L.tdev), c->t, c->stream));
    return HFS_OK;
}

int hfs_set_schedule(hfs_ctx_t c, int split, int ho_flow, int composition, const double *a, int na,
                     const double *b, int nb, double dt)
{
    if (!c) return HFS_ERR_INVALID_ARG;
    if (split != HFS_SPLIT_HO && split != HFS_SPLIT_FOURIER) return HFS_ERR_INVALID_ARG;
    if (ho_flow < HFS_FLOW_LEMMA2 || ho_flow > HFS_FLOW_M6) return HFS_ERR_INVALID_ARG;
    if (!(dt != 0.0) || !isfinite(dt)) return HFS_ERR_INVALID_ARG;
    std::vector<double> av, bv;
    if (composition == HFS_COMP_CUSTOM) {
        if (!a || !b || na < 1 || na > kMaxStages || nb != na + 1) return HFS_ERR_INVALID_ARG;
        av.assign(a, a + na);
        bv.assign(b, b + nb);
    } else if (composition_coeffs(composition, av, bv)) {
        return HFS_ERR_INVALID_ARG;
    }
    SchedConst sc{};
    sc.split = split;
    sc.flow = ho_flow;
    sc.m = (int)av.size();
    sc.h = dt;
    double cum = 0.0;
    for (int i = 0; i < sc.m; ++i) {
        sc.a[i] = av[i];
        sc.cuma[i] = cum;
        cum += av[i];
    }
    for (int i = 0; i <= sc.m; ++i) sc.b[i] = bv[i];
    if (c->work_base) {
        // the bound workspace must hold this schedule's chunk
        hfs_ctx_s probe = {};
        probe.dim = c->dim;
        probe.precision = c->precision;
        probe.count = c->count;
        probe.have_sched = true;
        probe.sc = sc;
        if (make_layout(&probe, c->chunk).total > c->work_bytes) return HFS_ERR_WORKSPACE;
        c->lay = make_layout(&probe, c->chunk);
    }
    c->sc = sc;
    c->have_sched = true;
    c->composition = composition;
    drop_graphs(c);
    return HFS_OK;
}

int hfs_set_mode(hfs_ctx_t c, int mode, int spl)
{
    if (!c || (mode != HFS_MODE_RESIDENT && mode != HFS_MODE_STREAMING) || spl < 1) return HFS_ERR_INVALID_ARG;
    c->mode = mode;
    c->spl = spl;
    drop_graphs(c);
    return HFS_OK;
}

int hfs_set_norm_projection(hfs_ctx_t c, int enable)
{
    if (!c) return HFS_ERR_INVALID_ARG;
    if (c->precision != HFS_C64) return HFS_ERR_UNSUPPORTED;
    // 3D: the plane-pass path (n = 128 per axis)
    if (c->dim == 3 && c->inst[0].n[0] != 128) return HFS_ERR_UNSUPPORTED;
    c->norm_projection = enable != 0;
    drop_graphs(c);
    return HFS_OK;
}

int hfs_set_dft_engine(hfs_ctx_t c, int engine)
{
    if (!c || (engine != HFS_DFT_SIMT && engine != HFS_DFT_TENSOR_3XTF32)) return HFS_ERR_INVALID_ARG;
    if (engine == HFS_DFT_TENSOR_3XTF32 &&
        (c->dim != 3 || c->precision != HFS_C64 || (c->inst[0].n[0] != 64 && c->inst[0].n[0] != 128)))
        return HFS_ERR_UNSUPPORTED;
    c->dft_engine = engine;
    drop_graphs(c);
    return HFS_OK;
}

int hfs_set_schedule_reuse(hfs_ctx_t c, int enable)
{
    if (!c) return HFS_ERR_INVALID_ARG;
    if (c->dim != 1) return enable ? HFS_ERR_UNSUPPORTED : HFS_OK;
    if (enable && !c->aux) {
        int least = 0, greatest = 0;
        CK(cudaDeviceGetStreamPriorityRange(&least, &greatest));
        c->prio_high = greatest;
        CK(cudaStreamCreateWithFlags(&c->aux, cudaStreamNonBlocking));
        CK(cudaEventCreateWithFlags(&c->fork_ev, cudaEventDisableTiming));
        CK(cudaEventCreateWithFlags(&c->join_ev, cudaEventDisableTiming));
    }
    drop_graphs(c);
    c->slot[0] = c->slot[1] = hfs_ctx_s::RecSlot{};
    c->sched_reuse = enable != 0;
    if (c->work_base) {
        const Layout L = make_layout(c, c->chunk);
        if (L.total > c->work_bytes) {
            // the bound workspace has no room for the second record buffer
            c->psi = nullptr;
            c->work_base = nullptr;
            c->work_bytes = 0;
            return HFS_ERR_WORKSPACE;
        }
        c->lay = L;
    }
    return HFS_OK;
}

int hfs_set_graphs(hfs_ctx_t c, int enable)
{
    if (!c) return HFS_ERR_INVALID_ARG;
    c->graphs = enable != 0;
    drop_graphs(c);
    return HFS_OK;
}

int hfs_set_time(hfs_ctx_t c, double t)
{
    if (!c || !isfinite(t)) return HFS_ERR_INVALID_ARG;
    c->t = t;
    if (c->work_base) CK(launch_set_time(wptr<double>(c, c->lay.tdev), t, c->stream));
    return HFS_OK;
}

int hfs_get_time(hfs_ctx_t c, double *t)
{
    if (!c || !t) return HFS_ERR_INVALID_ARG;
    *t = c->t;
    return HFS_OK;
}

int hfs_set_psi(hfs_ctx_t c, const void *src, int on_device)
{
    int s = ready(c);
    if (s) return s;
    if (!src) return HFS_ERR_INVALID_ARG;
    size_t bytes = 0;
    hfs_state_size(c, nullptr, &bytes);
    CK(cudaMemcpyAsync(c->psi, src, bytes, on_device ? cudaMemcpyDeviceToDevice : cudaMemcpyHostToDevice, c->stream));
    if (!on_device) CK(cudaStreamSynchronize(c->stream));
    return HFS_OK;
}

int hfs_get_psi(hfs_ctx_t c, void *dst, int on_device)
{
    int s = ready(c);
    if (s) return s;
    if (!dst) return HFS_ERR_INVALID_ARG;
    size_t bytes = 0;
    hfs_state_size(c, nullptr, &bytes);
    CK(cudaMemcpyAsync(dst, c->psi, bytes, on_device ? cudaMemcpyDeviceToDevice : cudaMemcpyDeviceToHost, c->stream));
    if (!on_device) CK(cudaStreamSynchronize(c->stream));
    return HFS_OK;
}

int hfs_step(hfs_ctx_t c, int64_t nsteps)
{
    NvtxRange nvtx_range("hfs_step");
    int s = ready(c);
    if (s) return s;
    if (!c->have_sched) return HFS_ERR_NOT_READY;
    if (nsteps < 0) return HFS_ERR_INVALID_ARG;
    if (nsteps == 0) return HFS_OK;
    if (make_layout(c, c->chunk).total > c->work_bytes) return HFS_ERR_WORKSPACE;
    s = check_validity(c, nsteps);
    if (s) return s;
    const ReusePlan rp = plan_reuse(c, nsteps);
    if (c->graphs) {
        if (c->stream == nullptr) return HFS_ERR_INVALID_ARG;  // the legacy stream cannot be captured
        const int64_t key = graph_key(nsteps, rp);
        auto it = c->graphs_by_n.find(key);
        if (it == c->graphs_by_n.end()) {
            cudaGraph_t g = nullptr;
            CK(cudaStreamBeginCapture(c->stream, cudaStreamCaptureModeThreadLocal));
            s = enqueue_steps(c, nsteps, rp);
            cudaError_t e = cudaStreamEndCapture(c->stream, &g);
            if (s) {
                if (g) cudaGraphDestroy(g);
                return s;
            }
            CK(e);
            cudaGraphExec_t ge = nullptr;
            // per-node priorities: the step kernel's launch priority survives capture
            e = cudaGraphInstantiate(&ge, g, cudaGraphInstantiateFlagUseNodePriority);
            cudaGraphDestroy(g);
            CK(e);
            it = c->graphs_by_n.emplace(key, ge).first;
        }
        CK(cudaGraphLaunch(it->second, c->stream));
    } else {
        s = enqueue_steps(c, nsteps, rp);
        if (s) return s;
    }
    // record buffer 0 is the one a call without reuse writes
    if (rp.on) commit_reuse(c, rp, nsteps);
    else c->slot[0].valid = false;
    c->t += (double)nsteps * c->sc.h;
    if (c->profiling) c->prof_valid = true;
    return HFS_OK;
}

static int run_diag(hfs_ctx_s *c)
{
    (void)cudaGetLastError();
    const bool fp64 = c->precision == HFS_C128;
    double *dout = wptr<double>(c, c->lay.diag);
    if (c->dim == 1) {
        Diag1DArgs a{};
        a.psi = c->psi;
        a.inst = wptr<DevInst>(c, c->lay.inst);
        a.order = wptr<int32_t>(c, c->lay.order);
        a.work = wptr<WorkItem>(c, c->lay.work);
        a.nwork = (int32_t)c->work.size();
        a.tw = fp64 ? wptr<void>(c, c->lay.twd) : wptr<void>(c, c->lay.twf);
        a.t_dev = wptr<double>(c, c->lay.tdev);
        a.out = dout;
        a.ticket = wptr<unsigned>(c, c->lay.ticket);
        CK(cudaMemsetAsync(a.ticket, 0, sizeof(unsigned), c->stream));
        const int grid = std::max(1, std::min<int>(a.nwork, c->sm_count * step1d_ctas_per_sm(fp64, c->variant)));
        CK(launch_diag1d(fp64, a, grid, c->stream));
    } else {
        Diag3DArgs a{};
        a.psi = c->psi;
        a.inst = wptr<DevInst>(c, c->lay.inst);
        a.tw = fp64 ? wptr<void>(c, c->lay.twd) : wptr<void>(c, c->lay.twf);
        a.t_dev = wptr<double>(c, c->lay.tdev);
        a.out = dout;
        a.n = c->inst[0].n[0];
        CK(launch_diag3d(fp64, a, c->stream));
    }
    CK(cudaMemcpyAsync(c->diag_host.data(), dout, sizeof(double) * 2 * c->count, cudaMemcpyDeviceToHost, c->stream));
    CK(cudaStreamSynchronize(c->stream));
    return HFS_OK;
}

int hfs_norm(hfs_ctx_t c, double *out)
{
    NvtxRange nvtx_range("hfs_norm");
    int s = ready(c);
    if (s) return s;
    if (!out) return HFS_ERR_INVALID_ARG;
    s = run_diag(c);
    if (s) return s;
    for (int64_t i = 0; i < c->count; ++i) out[i] = c->diag_host[2 * i];
    return HFS_OK;
}

int hfs_energy(hfs_ctx_t c, double *out)
{
    NvtxRange nvtx_range("hfs_energy");
    int s = ready(c);
    if (s) return s;
    if (!out) return HFS_ERR_INVALID_ARG;
    s = run_diag(c);
    if (s) return s;
    for (int64_t i = 0; i < c->count; ++i) out[i] = c->diag_host[2 * i + 1];
    return HFS_OK;
}

int hfs_sync_status(hfs_ctx_t c)
{
    int s = ready(c);
    if (s) return s;
    unsigned st = 0;
    CK(cudaMemcpyAsync(&st, wptr<unsigned>(c, c->lay.status), sizeof(unsigned), cudaMemcpyDeviceToHost, c->stream));
    CK(cudaMemsetAsync(wptr<unsigned>(c, c->lay.status), 0, sizeof(unsigned), c->stream));
    CK(cudaStreamSynchronize(c->stream));
    if (st & ST_TIMEOUT) return HFS_ERR_DEVICE_TIMEOUT;
    if (st & ST_NONFINITE) return HFS_ERR_NONFINITE;
    if (st & ST_BADPLAN) return HFS_ERR_UNSUPPORTED;
    return HFS_OK;
}

int hfs_set_plan(hfs_ctx_t c, int n, int plan)
{
    if (!c || c->dim != 1) return HFS_ERR_INVALID_ARG;
    const int sc = size_class(n);
    const int ept = plan & 0xff;
    const bool alt = (plan & HFS_PLAN_ALT_ORDER) != 0;
    if (sc < 0 || (plan & ~(0xff | HFS_PLAN_ALT_ORDER))) return HFS_ERR_UNSUPPORTED;
    if (ept != 16 && ept != 8 && ept != 4) return HFS_ERR_UNSUPPORTED;
    if ((ept == 8 && n > 2048) || (ept == 4 && n > 1024) || (alt && ept != 16)) return HFS_ERR_UNSUPPORTED;
    // the wide plans (four values per thread, alternative orders) are FP32 only
    if ((ept == 4 || alt) && c->precision != HFS_C64) return HFS_ERR_UNSUPPORTED;
    c->ept[sc] = ept;
    c->alt[sc] = alt;
    build_worklist(c);
    drop_graphs(c);
    if (c->work_base) return upload_tables(c);
    return HFS_OK;
}

int hfs_set_occupancy(hfs_ctx_t c, int ctas_per_sm)
{
    if (!c || c->dim != 1 || ctas_per_sm < 0) return HFS_ERR_INVALID_ARG;
    c->ctas_per_sm = ctas_per_sm;
    drop_graphs(c);
    return HFS_OK;
}

}  // extern "C"

namespace {

int encode_plan(const hfs_ctx_s *c, int k) { return c->ept[k] | (c->alt[k] ? HFS_PLAN_ALT_ORDER : 0); }

// time `steps` steps of the current work list (resident or streaming as
// set): one warm-up run, then the best of three
int time_worklist(hfs_ctx_s *c, int64_t steps, cudaEvent_t e0, cudaEvent_t e1, float *ms)
{
    int s = upload_tables(c);
    if (s) return s;
    *ms = INFINITY;
    for (int rep = 0; rep < 4; ++rep) {
        CK(cudaEventRecord(e0, c->stream));
        s = enqueue_steps(c, steps);
        if (s) return s;
        CK(cudaEventRecord(e1, c->stream));
        CK(cudaEventSynchronize(e1));
        float t = 0.0f;
        CK(cudaEventElapsedTime(&t, e0, e1));
        if (rep > 0) *ms = std::min(*ms, t);
    }
    return HFS_OK;
}

// The search of hfs_autotune (see include/hfs.h): coordinate descent over
// the grid sizes present, every candidate timed on the WHOLE batch (a size
// class alone under-fills the GPU and favours plans with more, smaller
// teams; a wide plan anywhere also moves the launch to the wide kernel),
// two rounds; then one CTA per SM against as many as fit.
int autotune(hfs_ctx_s *c, int trial_steps, float *best_total)
{
    const int64_t steps = std::min<int64_t>(trial_steps, c->chunk);
    bool present[kNumSizes] = {};
    for (auto &p : c->inst) present[size_class(p.n[0])] = true;
    // a smooth (zero) state keeps every trial well defined
    size_t bytes = 0;
    hfs_state_size(c, nullptr, &bytes);
    CK(cudaMemsetAsync(c->psi, 0, bytes, c->stream));
    cudaEvent_t e0 = nullptr, e1 = nullptr;
    CK(cudaEventCreate(&e0));
    CK(cudaEventCreate(&e1));
    const bool fp32 = c->precision == HFS_C64;
    int s = HFS_OK;
    float total = INFINITY;
    // start point: 8 values per thread up to n = 1024 (several instances per
    // CTA), 16 above; each size's plan moves the batch time by about 1 %,
    // so the descent is sensitive to where it starts
    for (int k = 0; k < kNumSizes; ++k) {
        c->ept[k] = (128 << k) <= 1024 ? 8 : 16;
        c->alt[k] = false;
    }
    build_worklist(c);
    s = time_worklist(c, steps, e0, e1, &total);
    const int cand[4] = {16, 8, 16 | HFS_PLAN_ALT_ORDER, 4};
    for (int round = 0; round < 2 && !s; ++round) {
        for (int k = 0; k < kNumSizes && !s; ++k) {
            if (!present[k]) continue;
            const int n = 128 << k;
            const int keep = encode_plan(c, k);
            int best_plan = keep;
            for (int ci = 0; ci < 4 && !s; ++ci) {
                const int plan = cand[ci], ept = plan & 0xff;
                const bool alt = (plan & HFS_PLAN_ALT_ORDER) != 0;
                if (plan == keep || (ept == 8 && n > 2048) || (ept == 4 && n > 1024)) continue;
                if ((ept == 4 || alt) && !fp32) continue;
                c->ept[k] = ept;
                c->alt[k] = alt;
                build_worklist(c);
                float ms = 0.0f;
                s = time_worklist(c, steps, e0, e1, &ms);
                if (!s && ms < total) {
                    total = ms;
                    best_plan = plan;
                }
            }
            c->ept[k] = best_plan & 0xff;
            c->alt[k] = (best_plan & HFS_PLAN_ALT_ORDER) != 0;
        }
    }
    if (!s) {
        // one CTA per SM against the current setting (as many as fit)
        build_worklist(c);
        const int keep = c->ctas_per_sm;
        c->ctas_per_sm = keep == 1 ? 0 : 1;
        float ms = 0.0f;
        s = time_worklist(c, steps, e0, e1, &ms);
        if (!s && ms < total) total = ms;
        else c->ctas_per_sm = keep;
    }
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    if (best_total) *best_total = total;
    return s;
}

}  // namespace

extern "C" {

int hfs_autotune(hfs_ctx_t c, int trial_steps, int32_t *best_plans)
{
    NvtxRange nvtx_range("hfs_autotune");
    int s = ready(c);
    if (s) return s;
    if (!c->have_sched || c->dim != 1 || trial_steps < 1) return HFS_ERR_INVALID_ARG;
    const bool graphs = c->graphs;
    c->graphs = false;
    const double t_save = c->t;
    s = autotune(c, trial_steps, nullptr);
    c->graphs = graphs;
    build_worklist(c);
    int s2 = upload_tables(c);
    c->t = t_save;
    if (c->work_base) CK(launch_set_time(wptr<double>(c, c->lay.tdev), t_save, c->stream));
    drop_graphs(c);
    if (best_plans) {
        bool present[kNumSizes] = {};
        for (auto &p : c->inst) present[size_class(p.n[0])] = true;
        for (int k = 0; k < kNumSizes; ++k) best_plans[k] = present[k] ? encode_plan(c, k) : 0;
    }
    return s ? s : s2;
}

}  // extern "C"

// ---------------------------------------------------------------------------
// tuned-plan cache (a small JSON file; see hfs_autotune_cache in hfs.h)
// ---------------------------------------------------------------------------
namespace {

#ifndef HFS_SOURCE_HASH
#define HFS_SOURCE_HASH "unknown"
#endif

std::string cache_key(const hfs_ctx_s *c)
{
    int dev = 0;
    cudaDeviceProp prop{};
    if (cudaGetDevice(&dev) != cudaSuccess || cudaGetDeviceProperties(&prop, dev) != cudaSuccess) return "";
    int count[kNumSizes] = {};
    for (auto &p : c->inst) count[size_class(p.n[0])]++;
    char buf[512];
    snprintf(buf, sizeof(buf), "%s|sm%d|%s|src=%s|vi=%d|proj=%d|mode=%d/%d|flow=%d|split=%d|m=%d|n=%d,%d,%d,%d,%d,%d",
             prop.name, prop.multiProcessorCount, c->precision == HFS_C128 ? "c128" : "c64", HFS_SOURCE_HASH,
             c->variant, c->norm_projection ? 1 : 0, c->mode, c->mode == HFS_MODE_STREAMING ? c->spl : 0,
             c->sc.flow, c->sc.split, c->sc.m, count[0], count[1], count[2], count[3], count[4], count[5]);
    std::string k(buf);
    for (char &ch : k)
        if (ch == '"' || ch == '\\') ch = '_';
    return k;
}

struct CacheEntry {
    std::string key;
    int plans[kNumSizes];
    int ctas_per_sm;
    double ms;
};

bool read_file(const char *path, std::string &out)
{
    FILE *f = fopen(path, "rb");
    if (!f) return false;
    char buf[4096];
    size_t n;
    while ((n = fread(buf, 1, sizeof(buf), f)) > 0) out.append(buf, n);
    fclose(f);
    return true;
}

// entries of a cache file written by write_cache (one entry per line)
std::vector<CacheEntry> parse_cache(const std::string &text)
{
    std::vector<CacheEntry> v;
    size_t pos = 0;
    const std::string kk = "\"key\": \"";
    while ((pos = text.find(kk, pos)) != std::string::npos) {
        pos += kk.size();
        const size_t end = text.find('"', pos);
        if (end == std::string::npos) break;
        CacheEntry e{};
        e.key = text.substr(pos, end - pos);
        const size_t pl = text.find("\"plans\": [", end);
        const size_t nl = text.find('\n', end);
        if (pl == std::string::npos || (nl != std::string::npos && pl > nl)) continue;
        if (sscanf(text.c_str() + pl, "\"plans\": [%d, %d, %d, %d, %d, %d], \"ctas_per_sm\": %d, \"ms\": %lf",
                   &e.plans[0], &e.plans[1], &e.plans[2], &e.plans[3], &e.plans[4], &e.plans[5], &e.ctas_per_sm,
                   &e.ms) == 8)
            v.push_back(e);
        pos = end;
    }
    return v;
}

bool write_cache(const char *path, const std::vector<CacheEntry> &v)
{
    std::string tmp = std::string(path) + ".tmp";
    FILE *f = fopen(tmp.c_str(), "wb");
    if (!f) return false;
    fprintf(f, "{\"hfs_tuned_plans\": 1, \"entries\": [\n");
    for (size_t i = 0; i < v.size(); ++i) {
        const CacheEntry &e = v[i];
        fprintf(f, "  {\"key\": \"%s\", \"plans\": [%d, %d, %d, %d, %d, %d], \"ctas_per_sm\": %d, \"ms\": %.4f}%s\n",
                e.key.c_str(), e.plans[0], e.plans[1], e.plans[2], e.plans[3], e.plans[4], e.plans[5], e.ctas_per_sm,
                e.ms, i + 1 < v.size() ? "," : "");
    }
    fprintf(f, "]}\n");
    const bool ok = fclose(f) == 0;
    return ok && rename(tmp.c_str(), path) == 0;
}

}  // namespace

extern "C" {

int hfs_autotune_cache(hfs_ctx_t c, const char *path, int trial_steps, int32_t *best_plans, int *hit)
{
    int s = ready(c);
    if (s) return s;
    if (!path || !c->have_sched || c->dim != 1 || trial_steps < 1) return HFS_ERR_INVALID_ARG;
    const std::string key = cache_key(c);
    if (key.empty()) return HFS_ERR_CUDA;
    std::string text;
    std::vector<CacheEntry> entries;
    if (read_file(path, text)) entries = parse_cache(text);
    for (const CacheEntry &e : entries) {
        if (e.key != key) continue;
        for (int k = 0; k < kNumSizes; ++k) {
            if (!e.plans[k]) continue;
            s = hfs_set_plan(c, 128 << k, e.plans[k]);
            if (s) return s;
        }
        c->ctas_per_sm = e.ctas_per_sm;
        drop_graphs(c);
        if (best_plans) std::copy(e.plans, e.plans + kNumSizes, best_plans);
        if (hit) *hit = 1;
        return HFS_OK;
    }
    const bool graphs = c->graphs;
    c->graphs = false;
    const double t_save = c->t;
    float total = 0.0f;
    s = autotune(c, trial_steps, &total);
    c->graphs = graphs;
    build_worklist(c);
    int s2 = upload_tables(c);
    c->t = t_save;
    if (c->work_base) CK(launch_set_time(wptr<double>(c, c->lay.tdev), t_save, c->stream));
    drop_graphs(c);
    if (s || s2) return s ? s : s2;
    CacheEntry e{};
    e.key = key;
    bool present[kNumSizes] = {};
    for (auto &p : c->inst) present[size_class(p.n[0])] = true;
    for (int k = 0; k < kNumSizes; ++k) e.plans[k] = present[k] ? encode_plan(c, k) : 0;
    e.ctas_per_sm = c->ctas_per_sm;
    e.ms = total;
    bool replaced = false;
    for (CacheEntry &o : entries)
        if (o.key == key) {
            o = e;
            replaced = true;
        }
    if (!replaced) entries.push_back(e);
    // a cache that cannot be written leaves the tuned plans in effect
    (void)write_cache(path, entries);
    if (best_plans) std::copy(e.plans, e.plans + kNumSizes, best_plans);
    if (hit) *hit = 0;
    return HFS_OK;
}

}  // extern "C"
