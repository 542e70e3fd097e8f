// hfs_step3d.cu -- 3D Hermite-Fourier split step on an n^3 periodic grid
// (n = 32, 64, 128; symmetric box), complex64 or complex128.
//
// The harmonic part sum_d (p_d^2 + omega_d^2(t) x_d^2)/2 separates by axis,
// so each A stage is kick(f_d) . drift(g_d) . kick(e_d) per axis (Theorem 2
// with omega_d = c_d omega(t)); the kicks of the three axes and the B flow
// merge into one pointwise x-phase, the drifts into one k-space phase of the
// 3D transform.  One sub-stage is four passes over the state, each a batch
// of length-n line transforms held in registers (layout of hfs_fft.cuh):
//   z-pass  forward FFT_z, k-phase sum_d G_d m_d^2 (and 1/n^3), inverse FFT_z
//   y-pass  inverse FFT_y
//   x-pass  inverse FFT_x, x-phase X_{j+1}, forward FFT_x
//   y-pass  forward FFT_y
// The x-pass owns contiguous lines (private padded shared memory); the y-
// and z-passes own tiles of TX adjacent columns whose lanes interleave in
// shared memory, so global accesses stay coalesced along x.
#include <algorithm>

#include "hfs_fft.cuh"
#include "hfs_law.cuh"
#include "hfs_phase.cuh"
#include "hfs_sched.h"
#include "hfs_step3d.h"
#include "hfs_tc.cuh"

namespace hfs {

template <typename R> struct Rec3Of;
template <> struct Rec3Of<float> { using type = Rec3F; };
template <> struct Rec3Of<double> { using type = Rec3D; };

template <int N> struct Geo3 {
    static constexpr int E = 16;
    static constexpr int T = N / E;                 // threads per line
    static constexpr int G = kCtaThreads / T;       // x-lines per CTA
    static constexpr int TX = (kCtaThreads / T < N) ? kCtaThreads / T : N;  // columns per y/z tile
    static constexpr int TT = T * TX;               // threads of a y/z tile CTA
};

__device__ __forceinline__ float turns_q(int m, float hi, float lo) { return frac_turns((float)(m * m), hi, lo); }
__device__ __forceinline__ double turns_q(int m, double c, double) { return frac_turns((double)m * m, c, 0.0); }

enum : int { X_INV = 1, X_PHASE = 2, X_FWD = 4 };

// ---------------------------------------------------------------------------
// x-pass
// ---------------------------------------------------------------------------
template <typename R, int N, int MODE>
__global__ void __launch_bounds__(kCtaThreads) xpass3d(const Step3DArgs a, int64_t j)
{
    using Rec = typename Rec3Of<R>::type;
    using GEO = Geo3<N>;
    constexpr int E = GEO::E, T = GEO::T;
    extern __shared__ __align__(16) unsigned char smem_raw[];
    const int g = threadIdx.x / T, t = threadIdx.x - g * T;
    const int line = blockIdx.x * GEO::G + g;  // y + N z
    const int y = line % N, z = line / N;
    cpx<R> *sm = reinterpret_cast<cpx<R> *>(smem_raw) + g * smem_elems(N);
    cpx<R> *psi = reinterpret_cast<cpx<R> *>(a.psi) + (int64_t)line * N;
    const auto *tw = reinterpret_cast<const typename TwOf<R>::type *>(a.tw);
    cpx<R> v[E];
#pragma unroll
    for (int e = 0; e < E; ++e) v[e] = psi[t + T * e];
    if constexpr (MODE & X_INV) FftPlan<N, E>::template run<true, R>(v, sm, t, tw);
    if constexpr (MODE & X_PHASE) {
        const Rec rc = reinterpret_cast<const Rec *>(a.rec)[j];
        const DevInst &ip = *a.inst;
        const int my = y - N / 2, mz = z - N / 2;
        const R tyz = turns_q(my, rc.k2[1], rc.k2lo[1]) + turns_q(mz, rc.k2[2], rc.k2lo[2]);
        const R dx = (R)ip.dx[0], vk = (R)ip.vi_k, eps = (R)ip.eps, sig = (R)ip.sigma;
        const int vkind = (ip.eps != 0.0) ? ip.vi_kind : HFS_VI_NONE;
        const R vyz = vi_eval(vkind, (R)my * (R)ip.dx[1], vk) + vi_eval(vkind, (R)mz * (R)ip.dx[2], vk);
#pragma unroll
        for (int e = 0; e < E; ++e) {
            const int mx = t + T * e - N / 2;
            R turns = turns_q(mx, rc.k2[0], rc.k2lo[0]) + tyz;
            const R dens = v[e].x * v[e].x + v[e].y * v[e].y;
            const R F = sig * dens + eps * (vi_eval(vkind, (R)mx * dx, vk) + vyz);
            turns += (R)rc.sb2pi * F;
            v[e] = apply_turns(v[e], turns, R(1));
        }
    }
    if constexpr (MODE & X_FWD) FftPlan<N, E>::template run<false, R>(v, sm, t, tw);
    bool bad = false;
#pragma unroll
    for (int e = 0; e < E; ++e) {
        psi[t + T * e] = v[e];
        bad |= !(isfinite(v[e].x) && isfinite(v[e].y));
    }
    if ((MODE & X_PHASE) && !(MODE & X_FWD) && bad) atomicOr(a.status, (unsigned)ST_NONFINITE);
}

// ---------------------------------------------------------------------------
// y-pass: one CTA = fixed z, TX adjacent x columns; lines along y
// ---------------------------------------------------------------------------
template <typename R, int N, bool INV>
__global__ void __launch_bounds__(kCtaThreads) ypass3d(const Step3DArgs a)
{
    using GEO = Geo3<N>;
    constexpr int E = GEO::E, T = GEO::T, TX = GEO::TX;
    extern __shared__ __align__(16) unsigned char smem_raw[];
    const int l = threadIdx.x % TX, t = threadIdx.x / TX;
    const int z = blockIdx.y, x0 = blockIdx.x * TX;
    cpx<R> *sm = reinterpret_cast<cpx<R> *>(smem_raw) + l;
    cpx<R> *psi = reinterpret_cast<cpx<R> *>(a.psi) + (int64_t)z * N * N + x0 + l;
    const auto *tw = reinterpret_cast<const typename TwOf<R>::type *>(a.tw);
    cpx<R> v[E];
#pragma unroll
    for (int e = 0; e < E; ++e) v[e] = psi[(int64_t)(t + T * e) * N];
    FftPlan<N, E>::template run<INV, R, TX>(v, sm, t, tw);
#pragma unroll
    for (int e = 0; e < E; ++e) psi[(int64_t)(t + T * e) * N] = v[e];
}

// Programmatic dependent launch of the 128^3 chain (z-pass, plane pass, ...):
// a kernel launched with programmatic stream serialisation may start while
// its predecessor finishes; pdl_wait() returns once the predecessor has
// completed and its memory is visible (at once for a kernel launched
// normally), and pdl_trigger() lets the successor be scheduled as soon as
// every CTA of this grid has started.  Nothing before pdl_wait() reads or
// writes the state or the projection sums.
__device__ __forceinline__ void pdl_wait() { asm volatile("griddepcontrol.wait;" ::: "memory"); }
__device__ __forceinline__ void pdl_trigger() { asm volatile("griddepcontrol.launch_dependents;" ::: "memory"); }

// ---------------------------------------------------------------------------
// z-pass: one CTA = fixed y, TX adjacent x columns; forward FFT_z, k-phase,
// inverse FFT_z
// ---------------------------------------------------------------------------
// FP32: two CTAs per SM (128 registers; at 143 registers one CTA of 8 warps
// per SM left the column loads' latency exposed); FP64: one
template <typename R> struct ZpassMinCtas { static constexpr int value = sizeof(R) == 4 ? 2 : 1; };
// Norm projection in 3D: the plane pass of sub-stage j adds its plane's sum
// of |u|^2 (taken in the x-phase) to slot j mod 3; the z-pass j that follows
// reads the complete sum, scales its k-phase by C = sqrt(target / sum), and
// clears slot j + 1 for the next plane pass.  The first z-pass of a call
// records the target (PROJ_SET) and applies C = 1.
// Every thread loads the two sums at the kernel's start (the loads complete
// behind the forward transform) and forms the factor in FP32 where the
// k-phase needs it; no thread waits on another for it.
struct Proj3 {
    double s, tg;
};
__device__ __forceinline__ Proj3 proj3_load(const Step3DArgs &a, int64_t j)
{
    if (threadIdx.x == 0 && blockIdx.x == 0 && blockIdx.y == 0) {
        a.nsum[(j + 1) % 3] = 0.0;
        if (j == 0 && a.proj == PROJ_SET) *a.ntarget = a.nsum[0];
    }
    return {a.nsum[j % 3], (j == 0 && a.proj == PROJ_SET) ? 0.0 : *a.ntarget};
}
__device__ __forceinline__ float proj3_factor(Proj3 p)
{
    // the ratio is 1 + O(1e-7): FP32 suffices; C = 1 while recording the target
    return (p.tg > 0.0 && p.s > 0.0 && isfinite(p.s)) ? sqrtf((float)p.tg / (float)p.s) : 1.0f;
}

// the transforms of the 3D kernels: plain twiddles with the projection (FP32)
template <int N, bool INV, int ILV, bool PROJ, int E, typename R>
__device__ __forceinline__ void fft3(cpx<R> (&v)[E], cpx<R> *sm, int t, const Step3DArgs &a)
{
    if constexpr (PROJ && sizeof(R) == 4)
        FftPlan<N, E>::template run<INV, R, ILV, false, false>(v, sm, t, static_cast<const float2 *>(a.tw2));
    else
        FftPlan<N, E>::template run<INV, R, ILV>(v, sm, t,
                                                 reinterpret_cast<const typename TwOf<R>::type *>(a.tw));
}

template <typename R, int N, bool PROJ = false>
__global__ void __launch_bounds__(kCtaThreads, ZpassMinCtas<R>::value) zpass3d(const Step3DArgs a, int64_t j)
{
    using Rec = typename Rec3Of<R>::type;
    using GEO = Geo3<N>;
    constexpr int E = GEO::E, T = GEO::T, TX = GEO::TX;
    extern __shared__ __align__(16) unsigned char smem_raw[];
    const int l = threadIdx.x % TX, t = threadIdx.x / TX;
    const int y = blockIdx.y, x = blockIdx.x * TX + l;
    cpx<R> *sm = reinterpret_cast<cpx<R> *>(smem_raw) + l;
    cpx<R> *psi = reinterpret_cast<cpx<R> *>(a.psi) + (int64_t)y * N + x;
    pdl_wait();
    pdl_trigger();
    cpx<R> v[E];
#pragma unroll
    for (int e = 0; e < E; ++e) v[e] = psi[(int64_t)(t + T * e) * N * N];
    Proj3 pr{0.0, 0.0};
    if constexpr (PROJ) pr = proj3_load(a, j);
    fft3<N, false, TX, PROJ>(v, sm, t, a);
    R C = R(1);
    if constexpr (PROJ) C = (R)proj3_factor(pr);
    {
        const Rec rc = reinterpret_cast<const Rec *>(a.rec)[j];
        const int mx = (x < N / 2) ? x : x - N;
        const int my = (y < N / 2) ? y : y - N;
        const R txy = turns_q(mx, rc.g[0], rc.glo[0]) + turns_q(my, rc.g[1], rc.glo[1]);
        const R scale = C / (R(N) * R(N) * R(N));
        if constexpr (sizeof(R) == 4) {
            // points in pairs, the phase arithmetic in packed FP32 (bit-identical)
#pragma unroll
            for (int e = 0; e < E; e += 2) {
                const int kz0 = t + T * e, kz1 = kz0 + T;
                const int mz0 = (kz0 < N / 2) ? kz0 : kz0 - N, mz1 = (kz1 < N / 2) ? kz1 : kz1 - N;
                const Turns2 tz = frac_turns2<true>(make_float2((float)(mz0 * mz0), (float)(mz1 * mz1)), rc.g[2],
                                                    rc.glo[2]);
                apply_turns2(v[e], v[e + 1], __fadd2_rn(bc2(txy), __fadd2_rn(tz.r, tz.c)), scale);
            }
        } else {
#pragma unroll
            for (int e = 0; e < E; ++e) {
                const int kz = t + T * e;
                const int mz = (kz < N / 2) ? kz : kz - N;
                v[e] = apply_turns(v[e], txy + turns_q(mz, rc.g[2], rc.glo[2]), scale);
            }
        }
    }
    fft3<N, true, TX, PROJ>(v, sm, t, a);
#pragma unroll
    for (int e = 0; e < E; ++e) psi[(int64_t)(t + T * e) * N * N] = v[e];
}

// ---------------------------------------------------------------------------
// z-pass with tensor-core DFT stages (complex64, n = 64 or 128): the first
// pass of each transform (radix 16, one butterfly per thread) runs as a
// 3xTF32 matrix product on the tensor cores (hfs_tc.cuh); the exchange, the
// last pass (radix n/16, twiddles) and the k-phase are those of zpass3d.
// ---------------------------------------------------------------------------
template <int N> constexpr size_t zpass_tc_smem()
{
    return (size_t)Geo3<N>::TX * N * sizeof(cpx<float>) + 2 * tc::kWBytes + 16;
}

// the first Stockham pass's exchange (NS = 1, butterfly b = t) after its DFT
template <int N, int TX> __device__ __forceinline__ void first_pass_exchange(cpx<float> (&v)[16], cpx<float> *sm, int t)
{
    constexpr int T = N / 16;
    cpx<float> *w = sm + (t * 16) * TX;
#pragma unroll
    for (int r = 0; r < 16; ++r) w[r * TX] = v[r];
    __syncthreads();
#pragma unroll
    for (int e = 0; e < 16; ++e) v[e] = sm[(t + T * e) * TX];
    __syncthreads();
}

template <int N, bool PROJ = false>
__global__ void __launch_bounds__(kCtaThreads, 2) zpass3d_tc(const Step3DArgs a, int64_t j)
{
    using GEO = Geo3<N>;
    constexpr int E = GEO::E, T = GEO::T, TX = GEO::TX;
    static_assert(GEO::TT == kCtaThreads && E == 16, "one radix-16 butterfly per thread, 256 threads");
    extern __shared__ __align__(16) unsigned char smem_raw[];
    unsigned char *wbuf = smem_raw + (size_t)TX * N * sizeof(cpx<float>);
    uint64_t *mbar = reinterpret_cast<uint64_t *>(wbuf + 2 * tc::kWBytes);
    uint32_t *slot = reinterpret_cast<uint32_t *>(mbar + 1);
    if (threadIdx.x < 32) tc::alloc(slot);
    if (threadIdx.x == 0) tc::mbar_init(tc::smem_addr(mbar));
    tc::fill_w(wbuf, wbuf + tc::kWBytes);
    tc::fence_before_sync();
    __syncthreads();
    tc::fence_after_sync();
    tc::Dft16 st{*slot, tc::smem_addr(wbuf), tc::smem_addr(wbuf + tc::kWBytes), tc::smem_addr(mbar), 0u};
    pdl_wait();
    pdl_trigger();

    const int l = threadIdx.x % TX, t = threadIdx.x / TX;
    const int y = blockIdx.y, x = blockIdx.x * TX + l;
    cpx<float> *sm = reinterpret_cast<cpx<float> *>(smem_raw) + l;
    cpx<float> *psi = reinterpret_cast<cpx<float> *>(a.psi) + (int64_t)y * N + x;
    const float4 *tw = reinterpret_cast<const float4 *>(a.tw);
    cpx<float> v[E];
#pragma unroll
    for (int e = 0; e < E; ++e) v[e] = psi[(int64_t)(t + T * e) * N * N];
    Proj3 pr{0.0, 0.0};
    if constexpr (PROJ) pr = proj3_load(a, j);
    bool ok = tc::dft16<false>(v, st);
    first_pass_exchange<N, TX>(v, sm, t);
    stockham_pass<N, E, N / 16, 16, false, true, TX, false>(v, sm, t, tw, 0);
    {
        const Rec3F rc = reinterpret_cast<const Rec3F *>(a.rec)[j];
        const int mx = (x < N / 2) ? x : x - N;
        const int my = (y < N / 2) ? y : y - N;
        const float txy = turns_q(mx, rc.g[0], rc.glo[0]) + turns_q(my, rc.g[1], rc.glo[1]);
        const float scale = (PROJ ? proj3_factor(pr) : 1.0f) / ((float)N * (float)N * (float)N);
#pragma unroll
        for (int e = 0; e < E; e += 2) {
            const int kz0 = t + T * e, kz1 = kz0 + T;
            const int mz0 = (kz0 < N / 2) ? kz0 : kz0 - N, mz1 = (kz1 < N / 2) ? kz1 : kz1 - N;
            const Turns2 tz =
                frac_turns2<true>(make_float2((float)(mz0 * mz0), (float)(mz1 * mz1)), rc.g[2], rc.glo[2]);
            apply_turns2(v[e], v[e + 1], __fadd2_rn(bc2(txy), __fadd2_rn(tz.r, tz.c)), scale);
        }
    }
    ok = tc::dft16<true>(v, st) && ok;
    first_pass_exchange<N, TX>(v, sm, t);
    stockham_pass<N, E, N / 16, 16, true, true, TX, false>(v, sm, t, tw, 0);
#pragma unroll
    for (int e = 0; e < E; ++e) psi[(int64_t)(t + T * e) * N * N] = v[e];
    if (!ok && threadIdx.x == 0) atomicOr(a.status, (unsigned)ST_TIMEOUT);
    tc::fence_before_sync();
    __syncthreads();
    if (threadIdx.x < 32) {
        tc::fence_after_sync();
        tc::dealloc(st.tmem);
    }
}

// ---------------------------------------------------------------------------
// plane pass (complex64, n = 128): one CTA owns a whole z-plane in shared
// memory (rows y of 128 + 8 padded slots) and runs, as the mode asks,
//   inverse FFT_y -> [inverse FFT_x, x-phase, forward FFT_x] -> forward FFT_y
// so that a sub-stage costs this pass plus the z-pass: two global round
// trips instead of four.  512 threads: 64 lines of 8 threads per round.
// ---------------------------------------------------------------------------
enum : int { P_INV_Y = 1, P_INV_X = 2, P_PHASE = 4, P_FWD_X = 8, P_FWD_Y = 16 };
constexpr int kPlaneN = 128, kPlaneRow = kPlaneN + kPlaneN / 16, kPlaneThreads = 512;

// VI: the instance's perturbation kind, a template parameter so that the
// phase loop carries no per-point test of it
// PROJ: plain twiddles and the norm sum of the x-phase (proj3_factor)
template <int MODE, int VI, bool PROJ = false>
__global__ void __launch_bounds__(kPlaneThreads, 1) plane3d(const Step3DArgs a, int64_t j)
{
    constexpr int N = kPlaneN, E = 16, T = N / E, LINES = kPlaneThreads / T;  // 64 lines per round
    extern __shared__ __align__(16) unsigned char smem_raw[];
    cpx<float> *pl = reinterpret_cast<cpx<float> *>(smem_raw);
    // eps V_I(x_j) of the plane's x-columns, evaluated once per launch
    __shared__ float s_vx[N];
    if constexpr (MODE & P_PHASE) {
        const DevInst &ip = *a.inst;
        for (int i = threadIdx.x; i < N; i += kPlaneThreads)
            s_vx[i] = (float)ip.eps * vi_eval(VI, (float)(i - N / 2) * (float)ip.dx[0], (float)ip.vi_k);
    }
    pdl_wait();
    pdl_trigger();
    const int z = blockIdx.x;
    cpx<float> *psi = reinterpret_cast<cpx<float> *>(a.psi) + (int64_t)z * N * N;
    // With the inverse y-transform the columns come straight from global
    // memory (lanes are adjacent x: coalesced); otherwise the plane is loaded
    // into shared memory (row y, padded slot of x) by asynchronous 8-byte
    // copies, all in flight at once.
    if constexpr (!(MODE & P_INV_Y)) {
        for (int i = threadIdx.x; i < N * N; i += kPlaneThreads) {
            const unsigned dst = (unsigned)__cvta_generic_to_shared(pl + (i / N) * kPlaneRow + spad(i % N));
            asm volatile("cp.async.ca.shared.global [%0], [%1], 8;" ::"r"(dst), "l"(psi + i) : "memory");
        }
        asm volatile("cp.async.wait_all;" ::: "memory");
        __syncthreads();
    }
    cpx<float> v[E];
    if constexpr (MODE & P_INV_Y) {
        // columns: lanes are adjacent x, slots of a column are kPlaneRow apart
        const int l = threadIdx.x % LINES, t = threadIdx.x / LINES;
        for (int r = 0; r < N / LINES; ++r) {
            const int x = r * LINES + l;
            cpx<float> *col = pl + spad(x);
#pragma unroll
            for (int e = 0; e < E; ++e) v[e] = psi[(t + T * e) * N + x];
            fft3<N, true, kPlaneRow, PROJ>(v, col, t, a);
#pragma unroll
            for (int e = 0; e < E; ++e) col[(t + T * e) * kPlaneRow] = v[e];
            __syncthreads();
        }
    }
    float dsum = 0.0f;  // this thread's sum of |u|^2 in the x-phase (projection)
    __shared__ float s_red[kPlaneThreads / 32];
    if constexpr ((MODE & P_INV_X) || (MODE & P_PHASE) || (MODE & P_FWD_X)) {
        const int g = threadIdx.x / T, t = threadIdx.x - g * T;
        const DevInst &ip = *a.inst;
        const Rec3F rc = reinterpret_cast<const Rec3F *>(a.rec)[j];
        const int mz = z - N / 2;
        constexpr int vkind = VI;
        const float vk = (float)ip.vi_k, eps = (float)ip.eps, sig = (float)ip.sigma;
        const float tz = turns_q(mz, rc.k2[2], rc.k2lo[2]);
        const float vz = vi_eval(vkind, (float)mz * (float)ip.dx[2], vk);
        for (int r = 0; r < N / LINES; ++r) {
            const int y = r * LINES + g;
            cpx<float> *row = pl + y * kPlaneRow;
#pragma unroll
            for (int e = 0; e < E; ++e) v[e] = row[spad(t + T * e)];
            __syncthreads();
            if constexpr (MODE & P_INV_X) fft3<N, true, 1, PROJ>(v, row, t, a);
            if constexpr (MODE & P_PHASE) {
                const int my = y - N / 2;
                const float tyz = turns_q(my, rc.k2[1], rc.k2lo[1]) + tz;
                const float vyz = vi_eval(vkind, (float)my * (float)ip.dx[1], vk) + vz;
                // points in pairs, the phase arithmetic in packed FP32 (bit-identical)
                const float evyz = eps * vyz;
                auto Fof = [&](const cpx<float> &u, int mx) {
                    const float dens = u.x * u.x + u.y * u.y;
                    if constexpr (PROJ) dsum += dens;
                    return sig * dens + (s_vx[mx + N / 2] + evyz);
                };
#pragma unroll
                for (int e = 0; e < E; e += 2) {
                    const int mx0 = t + T * e - N / 2, mx1 = mx0 + T;
                    const Turns2 tx = frac_turns2<true>(make_float2((float)(mx0 * mx0), (float)(mx1 * mx1)), rc.k2[0],
                                                        rc.k2lo[0]);
                    float2 turns = __fadd2_rn(__fadd2_rn(tx.r, tx.c), bc2(tyz));
                    turns = __ffma2_rn(bc2(rc.sb2pi), make_float2(Fof(v[e], mx0), Fof(v[e + 1], mx1)), turns);
                    apply_turns2(v[e], v[e + 1], turns, 1.0f);
                }
            }
            if constexpr (MODE & P_FWD_X) fft3<N, false, 1, PROJ>(v, row, t, a);
#pragma unroll
            for (int e = 0; e < E; ++e) row[spad(t + T * e)] = v[e];
            if constexpr (PROJ && (MODE & P_PHASE)) {
                if (r == N / LINES - 1) {
                    // the plane's sum of |u|^2: warp sums here, published by
                    // the barrier below, added by one thread into slot j mod 3
#pragma unroll
                    for (int o = 16; o > 0; o >>= 1) dsum += __shfl_xor_sync(0xffffffffu, dsum, o);
                    if ((threadIdx.x & 31) == 0) s_red[threadIdx.x >> 5] = dsum;
                }
            }
            __syncthreads();
        }
        if constexpr (PROJ && (MODE & P_PHASE)) {
            if (threadIdx.x < 32) {
                // the sixteen warp sums in FP32, the planes' totals in FP64
                float w = threadIdx.x < kPlaneThreads / 32 ? s_red[threadIdx.x] : 0.0f;
#pragma unroll
                for (int o = 8; o > 0; o >>= 1) w += __shfl_xor_sync(0xffffffffu, w, o);
                if (threadIdx.x == 0) atomicAdd(a.nsum + (j % 3), (double)w);
            }
        }
    }
    bool bad = false;
    if constexpr (MODE & P_FWD_Y) {
        // the forward y-transform writes its columns straight to global memory
        const int l = threadIdx.x % LINES, t = threadIdx.x / LINES;
        for (int r = 0; r < N / LINES; ++r) {
            const int x = r * LINES + l;
            cpx<float> *col = pl + spad(x);
#pragma unroll
            for (int e = 0; e < E; ++e) v[e] = col[(t + T * e) * kPlaneRow];
            __syncthreads();
            fft3<N, false, kPlaneRow, PROJ>(v, col, t, a);
#pragma unroll
            for (int e = 0; e < E; ++e) psi[(t + T * e) * N + x] = v[e];
        }
    } else {
        for (int i = threadIdx.x; i < N * N; i += kPlaneThreads) {
            const cpx<float> w = pl[(i / N) * kPlaneRow + spad(i % N)];
            psi[i] = w;
            bad |= !(isfinite(w.x) && isfinite(w.y));
        }
    }
    if ((MODE & P_PHASE) && !(MODE & P_FWD_X) && bad) atomicOr(a.status, (unsigned)ST_NONFINITE);
}

// ---------------------------------------------------------------------------
// diagnostics: norm, potential + interaction, and the kinetic energy as a sum
// over axes of 1D Parseval sums  sum_x |d_d u|^2 = (1/n) sum_k k_d^2 |F_d u|^2
// ---------------------------------------------------------------------------
__device__ __forceinline__ void block_add2(double a0, double a1, double *out, double *red)
{
    __syncthreads();
    red[2 * threadIdx.x] = a0;
    red[2 * threadIdx.x + 1] = a1;
    __syncthreads();
    for (int s = blockDim.x / 2; s > 0; s >>= 1) {
        if ((int)threadIdx.x < s) {
            red[2 * threadIdx.x] += red[2 * (threadIdx.x + s)];
            red[2 * threadIdx.x + 1] += red[2 * (threadIdx.x + s) + 1];
        }
        __syncthreads();
    }
    if (threadIdx.x == 0) {
        atomicAdd(out, red[0]);
        atomicAdd(out + 1, red[1]);
    }
}

template <typename R, int N> __global__ void __launch_bounds__(kCtaThreads) diagx3d(const Diag3DArgs a)
{
    using GEO = Geo3<N>;
    constexpr int E = GEO::E, T = GEO::T;
    extern __shared__ __align__(16) unsigned char smem_raw[];
    const int g = threadIdx.x / T, t = threadIdx.x - g * T;
    const int line = blockIdx.x * GEO::G + g;
    const int y = line % N, z = line / N;
    cpx<R> *sm = reinterpret_cast<cpx<R> *>(smem_raw) + g * smem_elems(N);
    const cpx<R> *psi = reinterpret_cast<const cpx<R> *>(a.psi) + (int64_t)line * N;
    const auto *tw = reinterpret_cast<const typename TwOf<R>::type *>(a.tw);
    const DevInst &ip = *a.inst;
    const double w2 = law_omega2(ip, *a.t_dev);
    const double dx = ip.dx[0];
    const double xy = (y - N / 2) * ip.dx[1], xz = (z - N / 2) * ip.dx[2];
    const double vyz = 0.5 * ip.mu * w2 * (ip.axis_scale[1] * ip.axis_scale[1] * xy * xy +
                                           ip.axis_scale[2] * ip.axis_scale[2] * xz * xz) +
                       ip.eps * (vi_eval(ip.vi_kind, xy, ip.vi_k) + vi_eval(ip.vi_kind, xz, ip.vi_k));
    cpx<R> v[E];
    double nrm = 0.0, en = 0.0;
#pragma unroll
    for (int e = 0; e < E; ++e) {
        v[e] = psi[t + T * e];
        const double xx = (t + T * e - N / 2) * dx;
        const double d = (double)v[e].x * v[e].x + (double)v[e].y * v[e].y;
        const double V = 0.5 * ip.mu * w2 * ip.axis_scale[0] * ip.axis_scale[0] * xx * xx +
                         ip.eps * vi_eval(ip.vi_kind, xx, ip.vi_k) + vyz;
        nrm += d;
        en += V * d + 0.5 * ip.sigma * d * d;
    }
    FftPlan<N, E>::template run<false, R>(v, sm, t, tw);
    const double ku = 2.0 * 3.14159265358979323846 / ip.len[0];
    double kin = 0.0;
#pragma unroll
    for (int e = 0; e < E; ++e) {
        const int k = t + T * e;
        const double kk = ku * ((k < N / 2) ? k : k - N);
        kin += kk * kk * ((double)v[e].x * v[e].x + (double)v[e].y * v[e].y);
    }
    const double dv = ip.dx[0] * ip.dx[1] * ip.dx[2];
    block_add2(nrm * dv, (en + kin / N / (2.0 * ip.mu)) * dv, a.out, reinterpret_cast<double *>(smem_raw));
}

// kinetic energy along y (AXIS = 1) or z (AXIS = 2)
template <typename R, int N, int AXIS> __global__ void __launch_bounds__(kCtaThreads) diagyz3d(const Diag3DArgs a)
{
    using GEO = Geo3<N>;
    constexpr int E = GEO::E, T = GEO::T, TX = GEO::TX;
    extern __shared__ __align__(16) unsigned char smem_raw[];
    const int l = threadIdx.x % TX, t = threadIdx.x / TX;
    const int other = blockIdx.y, x = blockIdx.x * TX + l;
    const int64_t stride = (AXIS == 1) ? N : (int64_t)N * N;
    const int64_t base = (AXIS == 1) ? (int64_t)other * N * N + x : (int64_t)other * N + x;
    cpx<R> *sm = reinterpret_cast<cpx<R> *>(smem_raw) + l;
    const cpx<R> *psi = reinterpret_cast<const cpx<R> *>(a.psi) + base;
    const auto *tw = reinterpret_cast<const typename TwOf<R>::type *>(a.tw);
    const DevInst &ip = *a.inst;
    cpx<R> v[E];
#pragma unroll
    for (int e = 0; e < E; ++e) v[e] = psi[(int64_t)(t + T * e) * stride];
    FftPlan<N, E>::template run<false, R, TX>(v, sm, t, tw);
    const double ku = 2.0 * 3.14159265358979323846 / ip.len[AXIS];
    double kin = 0.0;
#pragma unroll
    for (int e = 0; e < E; ++e) {
        const int k = t + T * e;
        const double kk = ku * ((k < N / 2) ? k : k - N);
        kin += kk * kk * ((double)v[e].x * v[e].x + (double)v[e].y * v[e].y);
    }
    const double dv = ip.dx[0] * ip.dx[1] * ip.dx[2];
    block_add2(0.0, kin / N / (2.0 * ip.mu) * dv, a.out, reinterpret_cast<double *>(smem_raw));
}

// ---------------------------------------------------------------------------
// host side
// ---------------------------------------------------------------------------
bool step3d_supported(int nx, int ny, int nz) { return nx == ny && ny == nz && (nx == 32 || nx == 64 || nx == 128); }

template <typename R, int N> static size_t xsmem() { return (size_t)Geo3<N>::G * smem_elems(N) * sizeof(cpx<R>); }
template <typename R, int N> static size_t tsmem()
{
    const size_t a = (size_t)Geo3<N>::TX * N * sizeof(cpx<R>);
    const size_t b = 2 * sizeof(double) * Geo3<N>::TT;
    return a > b ? a : b;
}

template <typename K> static cudaError_t allow_smem(K kernel, size_t bytes)
{
    return cudaFuncSetAttribute(kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)bytes);
}

// launch with programmatic stream serialisation (see pdl_wait)
template <typename... P>
static cudaError_t launch_pdl(void (*kernel)(P...), dim3 grid, dim3 block, size_t smem, cudaStream_t st,
                              const Step3DArgs &a, int64_t j)
{
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = grid;
    cfg.blockDim = block;
    cfg.dynamicSmemBytes = smem;
    cfg.stream = st;
    cudaLaunchAttribute at[1];
    at[0].id = cudaLaunchAttributeProgrammaticStreamSerialization;
    at[0].val.programmaticStreamSerializationAllowed = 1;
    cfg.attrs = at;
    cfg.numAttrs = 1;
    return cudaLaunchKernelEx(&cfg, kernel, a, j);
}

template <typename R, int N> static cudaError_t run3d(const Step3DArgs &a, cudaStream_t st)
{
    using GEO = Geo3<N>;
    const size_t xs = xsmem<R, N>(), ts = tsmem<R, N>();
    static bool prepared = false;
    if (!prepared) {
        cudaError_t e;
        if ((e = allow_smem(xpass3d<R, N, X_PHASE | X_FWD>, xs)) != cudaSuccess) return e;
        if ((e = allow_smem(xpass3d<R, N, X_INV | X_PHASE | X_FWD>, xs)) != cudaSuccess) return e;
        if ((e = allow_smem(xpass3d<R, N, X_INV | X_PHASE>, xs)) != cudaSuccess) return e;
        if ((e = allow_smem(ypass3d<R, N, false>, ts)) != cudaSuccess) return e;
        if ((e = allow_smem(ypass3d<R, N, true>, ts)) != cudaSuccess) return e;
        if ((e = allow_smem(zpass3d<R, N>, ts)) != cudaSuccess) return e;
        if constexpr (sizeof(R) == 4 && (N == 64 || N == 128))
            if ((e = allow_smem(zpass3d_tc<N>, zpass_tc_smem<N>())) != cudaSuccess) return e;
        prepared = true;
    }
    const dim3 xg(N * N / GEO::G), tg(N / GEO::TX, N);
    xpass3d<R, N, X_PHASE | X_FWD><<<xg, kCtaThreads, xs, st>>>(a, 0);
    ypass3d<R, N, false><<<tg, GEO::TT, ts, st>>>(a);
    for (int64_t j = 0; j < a.nstage; ++j) {
        if constexpr (sizeof(R) == 4 && (N == 64 || N == 128)) {
            if (a.dft_tc) zpass3d_tc<N><<<tg, GEO::TT, zpass_tc_smem<N>(), st>>>(a, j);
            else zpass3d<R, N><<<tg, GEO::TT, ts, st>>>(a, j);
        } else {
            zpass3d<R, N><<<tg, GEO::TT, ts, st>>>(a, j);
        }
        ypass3d<R, N, true><<<tg, GEO::TT, ts, st>>>(a);
        if (j + 1 < a.nstage) {
            xpass3d<R, N, X_INV | X_PHASE | X_FWD><<<xg, kCtaThreads, xs, st>>>(a, j + 1);
            ypass3d<R, N, false><<<tg, GEO::TT, ts, st>>>(a);
        } else {
            xpass3d<R, N, X_INV | X_PHASE><<<xg, kCtaThreads, xs, st>>>(a, j + 1);
        }
    }
    return cudaGetLastError();
}

template <typename R, int N> static cudaError_t diag3d(const Diag3DArgs &a, cudaStream_t st)
{
    using GEO = Geo3<N>;
    const size_t xs = xsmem<R, N>(), ts = tsmem<R, N>();
    static bool prepared = false;
    if (!prepared) {
        cudaError_t e;
        if ((e = allow_smem(diagx3d<R, N>, std::max(xs, 2 * sizeof(double) * kCtaThreads))) != cudaSuccess) return e;
        if ((e = allow_smem(diagyz3d<R, N, 1>, ts)) != cudaSuccess) return e;
        if ((e = allow_smem(diagyz3d<R, N, 2>, ts)) != cudaSuccess) return e;
        prepared = true;
    }
    cudaError_t e = cudaMemsetAsync(a.out, 0, 2 * sizeof(double), st);
    if (e != cudaSuccess) return e;
    const dim3 xg(N * N / GEO::G), tg(N / GEO::TX, N);
    diagx3d<R, N><<<xg, kCtaThreads, std::max(xs, 2 * sizeof(double) * kCtaThreads), st>>>(a);
    diagyz3d<R, N, 1><<<tg, GEO::TT, ts, st>>>(a);
    diagyz3d<R, N, 2><<<tg, GEO::TT, ts, st>>>(a);
    return cudaGetLastError();
}

template <int VI, bool PROJ> static cudaError_t run3d_plane_vi(const Step3DArgs &a, cudaStream_t st)
{
    constexpr int N = kPlaneN;
    using GEO = Geo3<N>;
    constexpr int FIRST = P_PHASE | P_FWD_X | P_FWD_Y, MID = P_INV_Y | P_INV_X | P_PHASE | P_FWD_X | P_FWD_Y,
                  LAST = P_INV_Y | P_INV_X | P_PHASE;
    const size_t ps = (size_t)N * kPlaneRow * sizeof(cpx<float>), ts = tsmem<float, N>();
    static bool prepared = false;
    if (!prepared) {
        cudaError_t e;
        if ((e = allow_smem(plane3d<FIRST, VI, PROJ>, ps)) != cudaSuccess) return e;
        if ((e = allow_smem(plane3d<MID, VI, PROJ>, ps)) != cudaSuccess) return e;
        if ((e = allow_smem(plane3d<LAST, VI, PROJ>, ps)) != cudaSuccess) return e;
        if ((e = allow_smem(zpass3d<float, N, PROJ>, ts)) != cudaSuccess) return e;
        if ((e = allow_smem(zpass3d_tc<N, PROJ>, zpass_tc_smem<N>())) != cudaSuccess) return e;
        prepared = true;
    }
    const dim3 tg(N / GEO::TX, N);
    // the first plane pass follows the schedule kernels and the sums' reset
    // in plain stream order; every later launch overlaps its predecessor's end
    plane3d<FIRST, VI, PROJ><<<N, kPlaneThreads, ps, st>>>(a, 0);
    cudaError_t e = cudaGetLastError();
    for (int64_t j = 0; j < a.nstage && e == cudaSuccess; ++j) {
        if (a.dft_tc) e = launch_pdl(zpass3d_tc<N, PROJ>, tg, dim3(GEO::TT), zpass_tc_smem<N>(), st, a, j);
        else e = launch_pdl(zpass3d<float, N, PROJ>, tg, dim3(GEO::TT), ts, st, a, j);
        if (e != cudaSuccess) break;
        if (j + 1 < a.nstage) e = launch_pdl(plane3d<MID, VI, PROJ>, dim3(N), dim3(kPlaneThreads), ps, st, a, j + 1);
        else e = launch_pdl(plane3d<LAST, VI, PROJ>, dim3(N), dim3(kPlaneThreads), ps, st, a, j + 1);
    }
    return e;
}

static cudaError_t run3d_plane(const Step3DArgs &a, cudaStream_t st)
{
    const bool proj = a.proj != PROJ_OFF;
    switch (a.vi) {
    case HFS_VI_COS: return proj ? run3d_plane_vi<HFS_VI_COS, true>(a, st) : run3d_plane_vi<HFS_VI_COS, false>(a, st);
    case HFS_VI_X4: return proj ? run3d_plane_vi<HFS_VI_X4, true>(a, st) : run3d_plane_vi<HFS_VI_X4, false>(a, st);
    case HFS_VI_NONE:
        return proj ? run3d_plane_vi<HFS_VI_NONE, true>(a, st) : run3d_plane_vi<HFS_VI_NONE, false>(a, st);
    default: return cudaErrorInvalidValue;
    }
}

cudaError_t launch_step3d(bool fp64, const Step3DArgs &a, cudaStream_t st)
{
    if (!fp64 && a.n == kPlaneN) return run3d_plane(a, st);
    switch (a.n) {
    case 32: return fp64 ? run3d<double, 32>(a, st) : run3d<float, 32>(a, st);
    case 64: return fp64 ? run3d<double, 64>(a, st) : run3d<float, 64>(a, st);
    case 128: return fp64 ? run3d<double, 128>(a, st) : run3d<float, 128>(a, st);
    default: return cudaErrorInvalidValue;
    }
}

cudaError_t launch_diag3d(bool fp64, const Diag3DArgs &a, cudaStream_t st)
{
    switch (a.n) {
    case 32: return fp64 ? diag3d<double, 32>(a, st) : diag3d<float, 32>(a, st);
    case 64: return fp64 ? diag3d<double, 64>(a, st) : diag3d<float, 64>(a, st);
    case 128: return fp64 ? diag3d<double, 128>(a, st) : diag3d<float, 128>(a, st);
    default: return cudaErrorInvalidValue;
    }
}

}  // namespace hfs
