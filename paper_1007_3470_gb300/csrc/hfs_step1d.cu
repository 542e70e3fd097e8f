// hfs_step1d.cu -- the fused, persistent 1D Hermite-Fourier split-step
// kernel (Eq. prod-genHarmOsc) for batches of independent instances of
// mixed grid size, and the norm / energy diagnostics.
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
};

template <typename R> __device__ __forceinline__ TeamParams<R> team_params(const DevInst &p)
{
    TeamParams<R> tp;
    tp.xc = (R)p.xc[0];
    tp.dx = (R)p.dx[0];
    tp.eps = (R)p.eps;
    tp.vik = (R)p.vi_k;
    tp.sigma = (R)p.sigma;
    tp.vikind = (p.eps != 0.0) ? p.vi_kind : HFS_VI_NONE;
    tp.asym = (p.xc[0] != 0.0);
    return tp;
}

// Opaque dependence on a group of register values: work on later groups
// cannot be scheduled before this point, so the phase loops below keep one
// group of PHASE_GROUP elements in flight instead of interleaving all E.
#ifndef HFS_PHASE_GROUP
#define HFS_PHASE_GROUP 4
#endif
constexpr int PHASE_GROUP = HFS_PHASE_GROUP;
// Phase arithmetic of point pairs in packed FP32 instructions for plans with
// at least this many values per thread (all plans; measured 2-5 % faster
// than the scalar form for both 8 and 16 values per thread).
#ifndef HFS_PACK_PHASE_MIN_E
#define HFS_PACK_PHASE_MIN_E 8
#endif
template <int E> __device__ __forceinline__ void fence_group(cpx<float> (&v)[E], int e0)
{
#ifndef HFS_NO_PHASE_FENCE
#pragma unroll
    for (int e = e0; e < e0 + PHASE_GROUP && e < E; ++e) asm volatile("" : "+f"(v[e].x), "+f"(v[e].y));
#endif
}
template <int E> __device__ __forceinline__ void fence_group(cpx<double> (&v)[E], int e0)
{
#pragma unroll
    for (int e = e0; e < e0 + PHASE_GROUP && e < E; ++e) asm volatile("" : "+d"(v[e].x), "+d"(v[e].y));
}

// merged x-phase X_j on the register layout (position t + T e)
// the phase argument of one point (turns) before the B-flow term
__device__ __forceinline__ float xphase_F(cpx<float> u, float mf, const TeamParams<float> &tp)
{
    const float x = fmaf(mf, tp.dx, tp.xc);
    const float dens = u.x * u.x + u.y * u.y;
    return fmaf(tp.sigma, dens, tp.eps * vi_eval(tp.vikind, x, tp.vik));
}

template <int N, int E>
__device__ __forceinline__ void xphase(cpx<float> (&v)[E], int t, const RecF &rc, const TeamParams<float> &tp)
{
    constexpr int T = N / E;
    constexpr bool PK = E >= HFS_PACK_PHASE_MIN_E;
    static_assert(E % 2 == 0 && PHASE_GROUP % 2 == 0, "points are phased in pairs");
#pragma unroll
    for (int e = 0; e < E; e += 2) {
        if (e % PHASE_GROUP == 0) fence_group(v, e);
        const int m0 = t + T * e - N / 2, m1 = m0 + T;
        const float2 mf = make_float2((float)m0, (float)m1);
        float2 turns = frac_turns2<PK>(make_float2((float)(m0 * m0), (float)(m1 * m1)), rc.k2hi, rc.k2lo);
        if (tp.asym) {
            const float2 lin = frac_turns2<PK>(mf, rc.k1hi, rc.k1lo);
            turns = make_float2(turns.x + (lin.x + rc.k0), turns.y + (lin.y + rc.k0));
        }
        const float2 F = make_float2(xphase_F(v[e], mf.x, tp), xphase_F(v[e + 1], mf.y, tp));
        if constexpr (PK) turns = __ffma2_rn(bc2(rc.sb2pi), F, turns);
        else turns = make_float2(fmaf(rc.sb2pi, F.x, turns.x), fmaf(rc.sb2pi, F.y, turns.y));
        apply_turns2<PK>(v[e], v[e + 1], turns, 1.0f);
    }
}

template <int N, int E>
__device__ __forceinline__ void xphase(cpx<double> (&v)[E], int t, const RecD &rc, const TeamParams<double> &tp)
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

// kinetic phase of drift D_{j+1} with the inverse transform's 1/N
template <int N, int E> __device__ __forceinline__ void kphase(cpx<float> (&v)[E], int t, const RecF &rc)
{
    constexpr int T = N / E;
    constexpr bool PK = E >= HFS_PACK_PHASE_MIN_E;
#pragma unroll
    for (int e = 0; e < E; e += 2) {
        if (e % PHASE_GROUP == 0) fence_group(v, e);
        const int k0 = t + T * e, k1 = k0 + T;
        const int m0 = (k0 < N / 2) ? k0 : k0 - N;
        const int m1 = (k1 < N / 2) ? k1 : k1 - N;
        const float2 turns = frac_turns2<PK>(make_float2((float)(m0 * m0), (float)(m1 * m1)), rc.ghi, rc.glo);
        apply_turns2<PK>(v[e], v[e + 1], turns, 1.0f / N);
    }
}

template <int N, int E> __device__ __forceinline__ void kphase(cpx<double> (&v)[E], int t, const RecD &rc)
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

template <typename R, int N, int E>
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
    for (int e = 0; e < E; ++e) v[e] = active ? psi[t + T * e] : cpx<R>{R(0), R(0)};

    for (int64_t j = a.j0; j < a.j1; ++j) {
        const Rec rc = rec[j];
        // Position-dependent values (m^2, x, V_I(x)) are the same at every
        // step; an opaque copy of t makes the compiler recompute them (a few
        // integer and SFU operations) instead of holding 3E of them live
        // across the whole time loop.
        int tl = t;
#ifndef HFS_NO_STEP_LAUNDER
        asm volatile("" : "+r"(tl));
#endif
        xphase<N, E>(v, tl, rc, tp);
        FftPlan<N, E>::template run<false, R>(v, sm, tl, tw);
        kphase<N, E>(v, tl, rc);
        FftPlan<N, E>::template run<true, R>(v, sm, tl, tw);
    }
    if (a.final_x) {
        const Rec rc = rec[a.j1];
        xphase<N, E>(v, t, rc, tp);
    }
    if (active) {
        bool bad = false;
#pragma unroll
        for (int e = 0; e < E; ++e) {
            psi[t + T * e] = v[e];
            bad |= !(isfinite(v[e].x) && isfinite(v[e].y));
        }
        if (bad) atomicOr(a.status, (unsigned)ST_NONFINITE);
    }
}

#ifdef HFS_ONLY_EPT8
#define HFS_FOR_EACH_PLAN(X) X(2048, 8) X(1024, 8) X(512, 8) X(256, 8) X(128, 8)
#else
#define HFS_FOR_EACH_PLAN(X)                                                                                      \
    X(4096, 16) X(2048, 16) X(1024, 16) X(512, 16) X(256, 16) X(128, 16) X(2048, 8) X(1024, 8) X(512, 8)        \
        X(256, 8) X(128, 8)
#endif

// FP32: two CTAs per SM (128 registers); FP64 parity mode: one
#ifndef HFS_STEP1D_MIN_CTAS
#define HFS_STEP1D_MIN_CTAS 2
#endif
template <typename R> struct MinCtas { static constexpr int value = sizeof(R) == 4 ? HFS_STEP1D_MIN_CTAS : 1; };

template <typename R>
__global__ void __launch_bounds__(kCtaThreads, MinCtas<R>::value) step1d_kernel(const Step1DArgs a)
{
    extern __shared__ __align__(16) unsigned char smem_raw[];
    cpx<R> *smem = reinterpret_cast<cpx<R> *>(smem_raw);
    __shared__ int s_item;
    for (;;) {
        if (threadIdx.x == 0) s_item = (int)atomicAdd(a.ticket, 1u);
        __syncthreads();
        const int w = s_item;
        if (w >= a.nwork) break;
        const WorkItem it = a.work[w];
        switch (it.plan) {
#define HFS_CASE(NN, EE)                                                                                          \
    case plan_id(NN, EE):                                                                                         \
        step_item<R, NN, EE>(a, it, smem);                                                                        \
        break;
            HFS_FOR_EACH_PLAN(HFS_CASE)
#undef HFS_CASE
        default:
            if (threadIdx.x == 0) atomicOr(a.status, (unsigned)ST_BADPLAN);
        }
        __syncthreads();
    }
}

// ---------------------------------------------------------------------------
// diagnostics: norm and energy (FP64 accumulation)
// ---------------------------------------------------------------------------
template <typename R, int N, int E>
__device__ __forceinline__ void diag_item(const Diag1DArgs &a, const WorkItem &it, cpx<R> *smem)
{
    constexpr int T = N / E;
    const int g = threadIdx.x / T;
    const int t = threadIdx.x - g * T;
    const bool active = g < it.count;
    const int idx = a.order[it.first + (active ? g : 0)];
    const DevInst &ip = a.inst[idx];
    const cpx<R> *psi = reinterpret_cast<const cpx<R> *>(a.psi) + ip.off;
    cpx<R> *sm = smem + g * smem_elems(N);
    const auto *tw = reinterpret_cast<const typename TwOf<R>::type *>(a.tw);
    const double w2 = law_omega2(ip, *a.t_dev);
    cpx<R> v[E];
    double nrm = 0.0, pot = 0.0, inter = 0.0, kin = 0.0;
#pragma unroll
    for (int e = 0; e < E; ++e) {
        v[e] = active ? psi[t + T * e] : cpx<R>{R(0), R(0)};
        const double x = ip.xc[0] + (double)(t + T * e - N / 2) * ip.dx[0];
        const double d = (double)v[e].x * v[e].x + (double)v[e].y * v[e].y;
        nrm += d;
        pot += (0.5 * ip.mu * w2 * x * x + ip.eps * vi_eval(ip.vi_kind, x, ip.vi_k)) * d;
        inter += 0.5 * ip.sigma * d * d;
    }
    FftPlan<N, E>::template run<false, R>(v, sm, t, tw);
    const double kunit = 2.0 * 3.14159265358979323846 / ip.len[0];
#pragma unroll
    for (int e = 0; e < E; ++e) {
        const int k = t + T * e;
        const double kk = kunit * (double)((k < N / 2) ? k : k - N);
        kin += kk * kk * ((double)v[e].x * v[e].x + (double)v[e].y * v[e].y);
    }
    const double energy = kin / N / (2.0 * ip.mu) + pot + inter;
    __syncthreads();
    double *red = reinterpret_cast<double *>(smem);
    red[2 * threadIdx.x] = nrm;
    red[2 * threadIdx.x + 1] = energy;
    __syncthreads();
    if (active && t == 0) {
        double sn = 0.0, se = 0.0;
        for (int u = 0; u < T; ++u) {
            sn += red[2 * (threadIdx.x + u)];
            se += red[2 * (threadIdx.x + u) + 1];
        }
        a.out[2 * idx] = sn * ip.dx[0];
        a.out[2 * idx + 1] = se * ip.dx[0];
    }
    __syncthreads();
}

template <typename R> __global__ void __launch_bounds__(kCtaThreads) diag1d_kernel(const Diag1DArgs a)
{
    extern __shared__ __align__(16) unsigned char smem_raw[];
    cpx<R> *smem = reinterpret_cast<cpx<R> *>(smem_raw);
    __shared__ int s_item;
    for (;;) {
        if (threadIdx.x == 0) s_item = (int)atomicAdd(a.ticket, 1u);
        __syncthreads();
        const int w = s_item;
        if (w >= a.nwork) break;
        const WorkItem it = a.work[w];
        switch (it.plan) {
#define HFS_CASE(NN, EE)                                                                                          \
    case plan_id(NN, EE):                                                                                         \
        diag_item<R, NN, EE>(a, it, smem);                                                                        \
        break;
            HFS_FOR_EACH_PLAN(HFS_CASE)
#undef HFS_CASE
        default:
            break;
        }
        __syncthreads();
    }
}

// ---------------------------------------------------------------------------
// twiddle tables (layout: tw_pass_offset), computed in FP64: entry
// (r - 1) NS + j of region (L, R) is exp(-2 pi i j r / L)
__global__ void twiddle_kernel(float4 *tf, double2 *td)
{
    const int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (i >= kTwiddleTotal) return;
    int L = 4;
    while (i >= tw_pass_offset(2 * L, 2)) L <<= 1;
    int R = 2;
    while (R < 16 && i >= tw_pass_offset(L, 2 * R)) R <<= 1;
    const int64_t s = i - tw_pass_offset(L, R);
    const int NS = L / R;
    const int64_t r = s / NS + 1, j = s % NS;
    double sn, cs;
    sincospi(2.0 * (double)(j * r) / (double)L, &sn, &cs);
    td[i] = make_double2(cs, -sn);
    const float ch = (float)cs, sh = (float)-sn;
    tf[i] = make_float4(ch, sh, (float)(cs - (double)ch), (float)(-sn - (double)sh));
}

// ---------------------------------------------------------------------------
// host launchers
// ---------------------------------------------------------------------------
size_t step1d_smem_bytes(bool fp64)
{
    return (size_t)(kCtaThreads / (4096 / 16)) * smem_elems(4096) * (fp64 ? sizeof(cpx<double>) : sizeof(cpx<float>));
}

static cudaError_t prepare(bool fp64)
{
    static bool done[2] = {false, false};
    if (done[fp64]) return cudaSuccess;
    const int bytes = (int)step1d_smem_bytes(fp64);
    cudaError_t e;
    if (fp64) {
        e = cudaFuncSetAttribute(step1d_kernel<double>, cudaFuncAttributeMaxDynamicSharedMemorySize, bytes);
        if (e == cudaSuccess)
            e = cudaFuncSetAttribute(diag1d_kernel<double>, cudaFuncAttributeMaxDynamicSharedMemorySize, bytes);
    } else {
        e = cudaFuncSetAttribute(step1d_kernel<float>, cudaFuncAttributeMaxDynamicSharedMemorySize, bytes);
        if (e == cudaSuccess)
            e = cudaFuncSetAttribute(diag1d_kernel<float>, cudaFuncAttributeMaxDynamicSharedMemorySize, bytes);
    }
    if (e == cudaSuccess) done[fp64] = true;
    return e;
}

int step1d_ctas_per_sm(bool fp64)
{
    if (prepare(fp64) != cudaSuccess) return 1;
    int n = 0;
    const size_t bytes = step1d_smem_bytes(fp64);
    cudaError_t e = fp64 ? cudaOccupancyMaxActiveBlocksPerMultiprocessor(&n, step1d_kernel<double>, kCtaThreads, bytes)
                         : cudaOccupancyMaxActiveBlocksPerMultiprocessor(&n, step1d_kernel<float>, kCtaThreads, bytes);
    return (e == cudaSuccess && n > 0) ? n : 1;
}

cudaError_t launch_step1d(bool fp64, const Step1DArgs &a, int grid, cudaStream_t st)
{
    cudaError_t e = prepare(fp64);
    if (e != cudaSuccess) return e;
    const size_t bytes = step1d_smem_bytes(fp64);
    if (fp64) step1d_kernel<double><<<grid, kCtaThreads, bytes, st>>>(a);
    else step1d_kernel<float><<<grid, kCtaThreads, bytes, st>>>(a);
    return cudaGetLastError();
}

cudaError_t launch_diag1d(bool fp64, const Diag1DArgs &a, int grid, cudaStream_t st)
{
    cudaError_t e = prepare(fp64);
    if (e != cudaSuccess) return e;
    const size_t bytes = step1d_smem_bytes(fp64);
    if (fp64) diag1d_kernel<double><<<grid, kCtaThreads, bytes, st>>>(a);
    else diag1d_kernel<float><<<grid, kCtaThreads, bytes, st>>>(a);
    return cudaGetLastError();
}

cudaError_t launch_twiddles(void *tw_f, void *tw_d, cudaStream_t st)
{
    twiddle_kernel<<<(unsigned)((kTwiddleTotal + 255) / 256), 256, 0, st>>>((float4 *)tw_f, (double2 *)tw_d);
    return cudaGetLastError();
}

}  // namespace hfs
