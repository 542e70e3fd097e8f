// hfs_step1d.cuh -- the fused, persistent 1D Hermite-Fourier split-step
// kernel (Eq. prod-genHarmOsc) for batches of independent instances of
// mixed grid size, shared by the translation units that instantiate it.
//
// One launch processes sub-stages [j0, j1) of a schedule chunk for every
// instance: for each sub-stage the merged x-phase X_j (kick f_{j-1} + e_j,
// B flow of Lemma 1, F-split trap) in registers, the forward FFT, the
// kinetic phase of drift D_{j+1} (with the 1/N of the inverse transform),
// the inverse FFT; optionally the closing X_{j1}.  The state is read once
// and written once per launch: with j1 - j0 covering a whole call
// (resident mode) every step stays on chip; with one step per launch
// (streaming mode) each step is one global round trip of 2 x 8 bytes per
// complex64 point.
//
// Work distribution: persistent CTAs of 256 threads take work items from a
// global ticket counter; a work item is up to 256/T instances of one grid
// size N (T = N/E threads per instance, E values per thread), sorted by
// decreasing N so that the longest items start first.
#pragma once

#include "hfs_fft.cuh"
#include "hfs_law.cuh"
#include "hfs_phase.cuh"
#include "hfs_sched.h"

namespace hfs {

template <typename R> struct RecOf;
template <> struct RecOf<float> { using type = RecF; };
template <> struct RecOf<double> { using type = RecD; };

template <typename R> struct TeamParams {
    R xc, dx, eps, vik, sigma;
    int vikind;
    bool asym;
    float vt_b[2], vt_a[2];  // V_I = cos(k x) in turns (DevInst::vi_turns)
};

template <typename R> __device__ __forceinline__ TeamParams<R> team_params(const DevInst &p)
{
    TeamParams<R> tp;
    if constexpr (sizeof(R) == 4) {
        // rounded on the host: no FP64 conversions per work item
        tp.xc = p.f32[0];
        tp.dx = p.f32[1];
        tp.eps = p.f32[2];
        tp.vik = p.f32[3];
        tp.sigma = p.f32[4];
        tp.vikind = p.vi_kind_eff;
        tp.asym = p.asym != 0;
    } else {
        tp.xc = (R)p.xc[0];
        tp.dx = (R)p.dx[0];
        tp.eps = (R)p.eps;
        tp.vik = (R)p.vi_k;
        tp.sigma = (R)p.sigma;
        tp.vikind = (p.eps != 0.0) ? p.vi_kind : HFS_VI_NONE;
        tp.asym = (p.xc[0] != 0.0);
    }
    tp.vt_b[0] = p.vi_turns[0];
    tp.vt_b[1] = p.vi_turns[1];
    tp.vt_a[0] = p.vi_turns[2];
    tp.vt_a[1] = p.vi_turns[3];
    return tp;
}

// Opaque dependence on a group of register values: work on later groups
// cannot be scheduled before this point, so the phase loops below keep one
// group of PHASE_GROUP elements in flight instead of interleaving all E.
#ifndef HFS_PHASE_GROUP
#define HFS_PHASE_GROUP 4
#endif
constexpr int PHASE_GROUP = HFS_PHASE_GROUP;
// FFT exchanges synchronise each instance's team alone (named barrier 1 + g)
#ifndef HFS_TEAM_SYNC
#define HFS_TEAM_SYNC true
#endif
// Phase arithmetic of point pairs in packed FP32 instructions for plans with
// at least this many values per thread (all plans; measured 2-5 % faster
// than the scalar form for both 8 and 16 values per thread).
#ifndef HFS_PACK_PHASE_MIN_E
#define HFS_PACK_PHASE_MIN_E 8
#endif
template <int E> __device__ __forceinline__ void fence_group(cpx<float> (&v)[E], int e0)
{
#pragma unroll
    for (int e = e0; e < e0 + PHASE_GROUP && e < E; ++e) asm volatile("" : "+f"(v[e].x), "+f"(v[e].y));
}
template <int E> __device__ __forceinline__ void fence_group(cpx<double> (&v)[E], int e0)
{
#pragma unroll
    for (int e = e0; e < e0 + PHASE_GROUP && e < E; ++e) asm volatile("" : "+d"(v[e].x), "+d"(v[e].y));
}

// merged x-phase X_j on the register layout (position t + T e)
// The table vt of eps V_I at a thread's points m = t + T e - N/2 (VI = -1:
// the instance's kind, none when eps = 0; VI >= 0: the launch's kind on a
// box symmetric about 0).  For
// V_I = cos(k x) the phase exp(2 pi i k x_m) is formed in turns, (a + b m)
// mod 1 with the exact product reduction of frac_turns, at e = 0, then
// advanced E - 1 times by the constant factor exp(2 pi i b T) (b T is exact:
// T is a power of two).  Each product adds about one rounding, so the table
// is within a few E units of FP32 rounding of cos(k x) whatever the size of
// k x, at E - 1 complex products and two small rotations per thread instead
// of E calls of cosf (whose inlined reductions also crowd the instruction
// cache when the table is rebuilt every launch, as in the streaming mode).
template <int N, int E, int VI>
__device__ __forceinline__ void vi_table(float *vt, int t, const TeamParams<float> &tp)
{
    constexpr int T = N / E;
    const int kind = VI < 0 ? tp.vikind : VI;
    if (kind == HFS_VI_COS) {
        const float m0 = (float)(t - N / 2);
        // a + b m0 mod 1 as an exact part r plus a small correction c
        const float p = tp.vt_b[0] * m0;
        float r = p - rintf(p);
        float c = fmaf(tp.vt_b[1], m0, fmaf(tp.vt_b[0], m0, -p));
        if (VI < 0) {
            const float s = r + tp.vt_a[0];  // |r|, |a| <= 1/2: two-sum, then re-reduce
            const float bb = s - r;
            c += (r - (s - bb)) + (tp.vt_a[0] - bb) + tp.vt_a[1];
            r = s - rintf(s);
        }
        float zc, zs, wc, ws;
        sincos_turns(r, c, zc, zs);
        const float pw = tp.vt_b[0] * (float)T;
        sincos_turns(pw - rintf(pw), tp.vt_b[1] * (float)T, wc, ws);
#pragma unroll
        for (int e = 0; e < E; ++e) {
            vt[t + T * e] = tp.eps * zc;
            const float nc = fmaf(zc, wc, -zs * ws);
            zs = fmaf(zs, wc, zc * ws);
            zc = nc;
        }
    } else if (kind == HFS_VI_X4) {
#pragma unroll
        for (int e = 0; e < E; ++e) {
            const float mf = (float)(t + T * e - N / 2);
            const float x = VI < 0 ? fmaf(mf, tp.dx, tp.xc) : mf * tp.dx;
            const float x2 = x * x;
            vt[t + T * e] = tp.eps * (x2 * x2);
        }
    } else {
#pragma unroll
        for (int e = 0; e < E; ++e) vt[t + T * e] = 0.0f;
    }
}

// VI >= 0: every instance of the launch has the perturbation kind VI and a
// box symmetric about 0 (compile-time, no per-point tests); VI = -1: both
// read from the team's instance.  Run-time tests inside the unrolled loop
// were evaluated for every point, both branches (7 % of the kernel time).
// vt: eps V_I at positions t + T e, written once per work item by the same
// thread (V_I does not depend on time), so no step re-evaluates it.
// dsum: the sum of |u|^2 over the thread's points before the phase (the
// phase leaves |u| unchanged), for the norm projection.
template <int N, int E, int VI>
__device__ __forceinline__ void xphase(cpx<float> (&v)[E], int t, const RecF &rc, const TeamParams<float> &tp,
                                       const float *vt, float &dsum)
{
    constexpr int T = N / E;
    constexpr bool PK = E >= HFS_PACK_PHASE_MIN_E;
    static_assert(E % 2 == 0 && PHASE_GROUP % 2 == 0, "points are phased in pairs");
    // grid index m = t + T e - N/2 and m^2 in FP32 (exact: |m| <= 2048)
    float tb = (float)(t - N / 2);
#pragma unroll
    for (int e = 0; e < E; e += 2) {
        if (e % PHASE_GROUP == 0) {
            fence_group(v, e);
            asm volatile("" : "+f"(tb));
        }
        const float2 mf = make_float2(tb + (float)(T * e), tb + (float)(T * (e + 1)));
        Turns2 tt = frac_turns2<PK>(mul2<PK>(mf, mf), rc.k2hi, rc.k2lo);
        if (VI < 0 && tp.asym) {
            // the linear chirp term of an off-centre box, into the correction
            const Turns2 lin = frac_turns2<PK>(mf, rc.k1hi, rc.k1lo);
            tt.c = add2<PK>(tt.c, add2<PK>(add2<PK>(lin.r, lin.c), bc2(rc.k0)));
        }
        // F = sigma |u|^2 + eps V_I(x)
        const float d0 = v[e].x * v[e].x + v[e].y * v[e].y;
        const float d1 = v[e + 1].x * v[e + 1].x + v[e + 1].y * v[e + 1].y;
        dsum += d0 + d1;
        float2 F;
        if constexpr (VI == HFS_VI_NONE) F = mul2<PK>(bc2(tp.sigma), make_float2(d0, d1));
        else F = fma2<PK>(bc2(tp.sigma), make_float2(d0, d1), make_float2(vt[t + T * e], vt[t + T * (e + 1)]));
        tt.c = fma2<PK>(bc2(rc.sb2pi), F, tt.c);
        apply_turns2<PK>(v[e], v[e + 1], tt, 1.0f);
    }
}

template <int N, int E, int VI>
__device__ __forceinline__ void xphase(cpx<double> (&v)[E], int t, const RecD &rc, const TeamParams<double> &tp,
                                       const float *, float &)
{
    constexpr int T = N / E;
#pragma unroll
    for (int e = 0; e < E; ++e) {
        const int m = t + T * e - N / 2;
        const double mf = (double)m;
        double turns = frac_turns(mf * mf, rc.k2, 0.0);
        if (tp.asym) turns += frac_turns(mf, rc.k1, 0.0) + rc.k0;
        const double x = fma(mf, tp.dx, tp.xc);
        const double dens = v[e].x * v[e].x + v[e].y * v[e].y;
        const double F = fma(tp.sigma, dens, tp.eps * vi_eval(tp.vikind, x, tp.vik));
        turns = fma(rc.sb2pi, F, turns);
        v[e] = apply_turns(v[e], turns, 1.0);
    }
}

// kinetic phase of drift D_{j+1} with the inverse transform's 1/N and, with
// CORR, the norm projection's factor C
template <int N, int E, bool CORR>
__device__ __forceinline__ void kphase(cpx<float> (&v)[E], int t, const RecF &rc, float C)
{
    constexpr int T = N / E;
    constexpr bool PK = E >= HFS_PACK_PHASE_MIN_E;
    // wavenumber index of k = t + T e: k for k < N/2, k - N above; with
    // 0 <= t < T that is e < E/2, known at compile time.  In FP32, exact.
    float tf = (float)t;
#pragma unroll
    for (int e = 0; e < E; e += 2) {
        if (e % PHASE_GROUP == 0) {
            fence_group(v, e);
            asm volatile("" : "+f"(tf));
        }
        const float2 mf = make_float2(tf + (float)(T * e - (2 * e < E ? 0 : N)),
                                      tf + (float)(T * (e + 1) - (2 * (e + 1) < E ? 0 : N)));
        apply_turns2<PK, CORR>(v[e], v[e + 1], frac_turns2<PK>(mul2<PK>(mf, mf), rc.ghi, rc.glo), 1.0f / N, C);
    }
}

template <int N, int E, bool CORR>
__device__ __forceinline__ void kphase(cpx<double> (&v)[E], int t, const RecD &rc, float)
{
    constexpr int T = N / E;
#pragma unroll
    for (int e = 0; e < E; ++e) {
        const int k = t + T * e;
        const double m = (double)((k < N / 2) ? k : k - N);
        const double turns = frac_turns(m * m, rc.g, 0.0);
        v[e] = apply_turns(v[e], turns, 1.0 / N);
    }
}

// complex elements of the exchange buffers of a CTA (the largest over the
// plans: E = 16 values per thread), and floats of the eps V_I table and of
// the per-warp norm sums after them
constexpr int step1d_exchange_elems = (kCtaThreads / (4096 / 16)) * smem_elems(4096);
constexpr int step1d_vtable_floats = kCtaThreads * 16;
constexpr int step1d_slot_floats = kCtaThreads / 32;

// Norm projection (FP32 path).  The exact scheme is unitary: every sub-flow
// preserves the discrete norm dx sum |u|^2 (Lemma 1; the kicks and drifts
// are pure phases in x and k).  In FP32 each rounding of the FFT passes and
// phases changes it by an unbiased random amount, so the norm random-walks
// (rms ~ 8e-7 after 500 steps for a state spread over ~15 grid points).
// With projection on, every sub-stage measures the team's sum of |u|^2 in
// the x-phase and rescales the state in the k-phase by
// C = sqrt(target / sum), target being the sum at the start of the
// hfs_step() call: the radial (norm) component of the rounding error is
// removed each sub-stage instead of accumulating.
//
// Team sums: teams of T <= 32 threads occupy aligned lane segments and reduce
// by xor shuffles inside the segment; larger teams reduce per warp, lane 0
// stores the warp's sum in slots[warp], and the team adds its warps' slots
// after the next team barrier (the forward FFT has at least one exchange).
template <int T> __device__ __forceinline__ float team_sum_begin(float s, float *slots)
{
    constexpr int W = T < 32 ? T : 32;
#pragma unroll
    for (int o = W / 2; o > 0; o >>= 1) s += __shfl_xor_sync(0xffffffffu, s, o);
    if constexpr (T > 32) {
        if ((threadIdx.x & 31) == 0) slots[threadIdx.x >> 5] = s;
    }
    return s;
}
template <int T> __device__ __forceinline__ float team_sum_end(float s, const float *slots, int g)
{
    if constexpr (T <= 32) {
        return s;
    } else {
        float r = 0.0f;
#pragma unroll
        for (int w = 0; w < T / 32; ++w) r += slots[g * (T / 32) + w];
        return r;
    }
}

// The transforms of the step: with the norm projection (FP32) the plain
// twiddle table, otherwise the compensated one.
template <bool INV, bool PROJ, int N, bool ALT, int E, typename R>
__device__ __forceinline__ void fft(const Step1DArgs &a, cpx<R> (&v)[E], cpx<R> *sm, int t,
                                    const typename TwOf<R>::type *tw, int g)
{
    if constexpr (PROJ && sizeof(R) == 4)
        FftPlan<N, E, ALT>::template run<INV, R, 1, HFS_TEAM_SYNC, false>(v, sm, t,
                                                                          static_cast<const float2 *>(a.tw2), 1 + g);
    else FftPlan<N, E, ALT>::template run<INV, R, 1, HFS_TEAM_SYNC>(v, sm, t, tw, 1 + g);
}

// sub-stages [j0, j1): X_j, forward FFT, kinetic phase (+ projection), inverse FFT
template <typename R, int VI, int N, int E, bool ALT, bool PROJ, typename Rec>
__device__ __forceinline__ void step_loop(const Step1DArgs &a, cpx<R> (&v)[E], int t, int g, bool active, int idx,
                                          const Rec *rec, const TeamParams<R> &tp, cpx<R> *sm,
                                          const typename TwOf<R>::type *tw, const float *vt, float *slots)
{
    constexpr int T = N / E;
    // the team's target sum of |u|^2: read, or set from the first sub-stage
    float target = 0.0f;
    if constexpr (PROJ) {
        if (a.proj == PROJ_USE) target = active ? a.norm_target[idx] : 0.0f;
    }
    for (int64_t j = a.j0; j < a.j1; ++j) {
        const Rec rc = rec[j];
        // Position-dependent values (m^2, x, V_I(x)) are the same at every
        // step; an opaque copy of t makes the compiler recompute them (a few
        // integer and SFU operations) instead of holding 3E of them live
        // across the whole time loop.
        int tl = t;
        asm volatile("" : "+r"(tl));
        float dsum = 0.0f;
        xphase<N, E, VI>(v, tl, rc, tp, vt, dsum);
        if constexpr (PROJ) dsum = team_sum_begin<T>(dsum, slots);
        fft<false, PROJ, N, ALT>(a, v, sm, tl, tw, g);
        float C = 1.0f;
        if constexpr (PROJ) {
            const float s = team_sum_end<T>(dsum, slots, g);
            if (j == a.j0 && a.proj == PROJ_SET) {
                target = s;
                if (active && t == 0) a.norm_target[idx] = s;
            } else if (target > 0.0f && s > 0.0f && isfinite(s)) {
                C = sqrtf(target / s);
            }
        }
        kphase<N, E, PROJ>(v, tl, rc, C);
        fft<true, PROJ, N, ALT>(a, v, sm, tl, tw, g);
    }
}

// state loads and stores of streaming launches carry the evict-first hint,
// so that a state larger than L2 passing through it every step does not push
// out the kernel's code, tables and phase records
__device__ __forceinline__ cpx<float> ld_state(const cpx<float> *p, bool streaming)
{
    if (streaming) {
        const float2 f = __ldcs(reinterpret_cast<const float2 *>(p));
        return {f.x, f.y};
    }
    return *p;
}
__device__ __forceinline__ cpx<double> ld_state(const cpx<double> *p, bool streaming)
{
    if (streaming) {
        const double2 f = __ldcs(reinterpret_cast<const double2 *>(p));
        return {f.x, f.y};
    }
    return *p;
}
__device__ __forceinline__ void st_state(cpx<float> *p, cpx<float> v, bool streaming)
{
    if (streaming) __stcs(reinterpret_cast<float2 *>(p), make_float2(v.x, v.y));
    else *p = v;
}
__device__ __forceinline__ void st_state(cpx<double> *p, cpx<double> v, bool streaming)
{
    if (streaming) __stcs(reinterpret_cast<double2 *>(p), make_double2(v.x, v.y));
    else *p = v;
}

template <typename R, int VI, int N, int E, bool ALT, bool PROJ>
__device__ __forceinline__ void step_item(const Step1DArgs &a, const WorkItem &it, cpx<R> *smem)
{
    using Rec = typename RecOf<R>::type;
    constexpr int T = N / E;
    const int g = threadIdx.x / T;
    const int t = threadIdx.x - g * T;
    const bool active = g < it.count;
    const int idx = a.order[it.first + (active ? g : 0)];
    const DevInst &ip = a.inst[idx];
    const TeamParams<R> tp = team_params<R>(ip);
    cpx<R> *psi = reinterpret_cast<cpx<R> *>(a.psi) + ip.off;
    cpx<R> *sm = smem + g * smem_elems(N);
    const auto *tw = reinterpret_cast<const typename TwOf<R>::type *>(a.tw);
    const Rec *rec = reinterpret_cast<const Rec *>(a.rec) + (int64_t)idx * a.nrec;

    cpx<R> v[E];
#pragma unroll
    for (int e = 0; e < E; ++e) v[e] = active ? ld_state(psi + t + T * e, a.streaming) : cpx<R>{R(0), R(0)};
    // FP32: the table of eps V_I behind the exchange buffers (each thread
    // reads back only the entries it wrote), then the norm-sum slots
    float *vt = reinterpret_cast<float *>(smem + step1d_exchange_elems) + g * N;
    float *slots = reinterpret_cast<float *>(smem + step1d_exchange_elems) + step1d_vtable_floats;
    if constexpr (sizeof(R) == 4 && VI != HFS_VI_NONE) vi_table<N, E, VI>(vt, t, tp);
    step_loop<R, VI, N, E, ALT, PROJ && sizeof(R) == 4>(a, v, t, g, active, idx, rec, tp, sm, tw, vt, slots);
    if (a.final_x) {
        const Rec rc = rec[a.j1];
        float dsum = 0.0f;
        xphase<N, E, VI>(v, t, rc, tp, vt, dsum);
    }
    if (active) {
        bool bad = false;
#pragma unroll
        for (int e = 0; e < E; ++e) {
            st_state(psi + t + T * e, v[e], a.streaming);
            bad |= !(isfinite(v[e].x) && isfinite(v[e].y));
        }
        if (bad) atomicOr(a.status, (unsigned)ST_NONFINITE);
    }
}

// (N, E, ALT) of the plans in every step kernel, and of those only in the
// wide kernels (alternative radix orders, four values per thread)
#define HFS_FOR_EACH_PLAN(X)                                                                                      \
    X(4096, 16, false) X(2048, 16, false) X(1024, 16, false) X(512, 16, false) X(256, 16, false)                 \
        X(128, 16, false) X(2048, 8, false) X(1024, 8, false) X(512, 8, false) X(256, 8, false) X(128, 8, false)
#define HFS_FOR_EACH_WIDE_PLAN(X)                                                                                 \
    X(4096, 16, true) X(2048, 16, true) X(1024, 16, true) X(512, 16, true) X(256, 16, true) X(128, 16, true)     \
        X(1024, 4, false) X(512, 4, false) X(256, 4, false) X(128, 4, false)

// FP32: two CTAs per SM (128 registers); FP64 parity mode: one
#ifndef HFS_STEP1D_MIN_CTAS
#define HFS_STEP1D_MIN_CTAS 2
#endif
template <typename R> struct MinCtas { static constexpr int value = sizeof(R) == 4 ? HFS_STEP1D_MIN_CTAS : 1; };

// PROJ: the norm projection (its loop and the plain twiddle table); a kernel
// holds one of the two loops per plan, not both, to keep its instruction
// footprint down
template <typename R, int VI, bool WIDE, bool PROJ>
__global__ void __launch_bounds__(kCtaThreads, MinCtas<R>::value) step1d_kernel(const Step1DArgs a)
{
    extern __shared__ __align__(16) unsigned char smem_raw[];
    cpx<R> *smem = reinterpret_cast<cpx<R> *>(smem_raw);
    __shared__ int s_item;
    // streaming launches claim the next item when they start the current one
    // (the ticket's round trip overlaps the work); resident launches claim
    // when they need one, so that the long items at the end balance best
    if (a.streaming && threadIdx.x == 0) s_item = (int)atomicAdd(a.ticket, 1u);
    for (;;) {
        if (!a.streaming && threadIdx.x == 0) s_item = (int)atomicAdd(a.ticket, 1u);
        __syncthreads();
        const int w = s_item;
        if (w >= a.nwork) break;
        unsigned next = 0;
        if (a.streaming && threadIdx.x == 0) next = atomicAdd(a.ticket, 1u);
        const WorkItem it = a.work[w];
        switch (it.plan) {
#define HFS_CASE(NN, EE, AA)                                                                                      \
    case plan_id(NN, EE, AA):                                                                                     \
        step_item<R, VI, NN, EE, AA, PROJ>(a, it, smem);                                                          \
        break;
            HFS_FOR_EACH_PLAN(HFS_CASE)
#undef HFS_CASE
        default: {
            bool handled = false;
            if constexpr (WIDE) {
                switch (it.plan) {
#define HFS_CASE(NN, EE, AA)                                                                                      \
    case plan_id(NN, EE, AA):                                                                                     \
        step_item<R, VI, NN, EE, AA, PROJ>(a, it, smem);                                                          \
        handled = true;                                                                                           \
        break;
                    HFS_FOR_EACH_WIDE_PLAN(HFS_CASE)
#undef HFS_CASE
                default:
                    break;
                }
            }
            if (!handled && threadIdx.x == 0) atomicOr(a.status, (unsigned)ST_BADPLAN);
        }
        }
        __syncthreads();
        if (a.streaming && threadIdx.x == 0) s_item = (int)next;
    }
}


// ---------------------------------------------------------------------------
// per-variant host launch (instantiated in one translation unit per variant)
// ---------------------------------------------------------------------------
size_t step1d_smem_bytes(bool fp64);

template <typename R, int VI, bool WIDE> cudaError_t step1d_prepare_t()
{
    static bool done = false;
    if (done) return cudaSuccess;
    const int bytes = (int)step1d_smem_bytes(sizeof(R) == 8);
    cudaError_t e = cudaFuncSetAttribute(step1d_kernel<R, VI, WIDE, false>,
                                         cudaFuncAttributeMaxDynamicSharedMemorySize, bytes);
    if (e == cudaSuccess && sizeof(R) == 4)
        e = cudaFuncSetAttribute(step1d_kernel<R, VI, WIDE, true>, cudaFuncAttributeMaxDynamicSharedMemorySize, bytes);
    if (e == cudaSuccess) done = true;
    return e;
}

template <typename R, int VI, bool WIDE> int step1d_ctas_per_sm_t()
{
    if (step1d_prepare_t<R, VI, WIDE>() != cudaSuccess) return 1;
    int n = 0;
    const cudaError_t e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(
        &n, step1d_kernel<R, VI, WIDE, false>, kCtaThreads, step1d_smem_bytes(sizeof(R) == 8));
    return (e == cudaSuccess && n > 0) ? n : 1;
}

// priority != 0: launched with that scheduling priority (lower = dispatched
// first), so that its CTAs take the SMs before those of a concurrent branch
template <typename R, int VI, bool WIDE>
cudaError_t step1d_launch_t(const Step1DArgs &a, int grid, cudaStream_t st, int priority)
{
    const cudaError_t e = step1d_prepare_t<R, VI, WIDE>();
    if (e != cudaSuccess) return e;
    const size_t bytes = step1d_smem_bytes(sizeof(R) == 8);
    const bool proj = sizeof(R) == 4 && a.proj != PROJ_OFF;
    if (priority != 0) {
        cudaLaunchConfig_t cfg = {};
        cfg.gridDim = dim3((unsigned)grid);
        cfg.blockDim = dim3(kCtaThreads);
        cfg.dynamicSmemBytes = bytes;
        cfg.stream = st;
        cudaLaunchAttribute at[1];
        at[0].id = cudaLaunchAttributePriority;
        at[0].val.priority = priority;
        cfg.attrs = at;
        cfg.numAttrs = 1;
        return proj ? cudaLaunchKernelEx(&cfg, step1d_kernel<R, VI, WIDE, true>, a)
                    : cudaLaunchKernelEx(&cfg, step1d_kernel<R, VI, WIDE, false>, a);
    }
    if (proj) step1d_kernel<R, VI, WIDE, true><<<grid, kCtaThreads, bytes, st>>>(a);
    else step1d_kernel<R, VI, WIDE, false><<<grid, kCtaThreads, bytes, st>>>(a);
    return cudaGetLastError();
}

// explicit instantiations: the generic kernels in hfs_step1d.cu, one
// specialised FP32 kernel per perturbation kind in hfs_step1d_vi*.cu, the
// wide FP32 kernels in hfs_step1d_wide*.cu
#define HFS_STEP1D_VARIANT(EXTERN, R, VI, WIDE)                                                                   \
    EXTERN template cudaError_t step1d_launch_t<R, VI, WIDE>(const Step1DArgs &, int, cudaStream_t, int);           \
    EXTERN template int step1d_ctas_per_sm_t<R, VI, WIDE>();

}  // namespace hfs
