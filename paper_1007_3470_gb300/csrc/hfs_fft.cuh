// hfs_fft.cuh -- register/shared-memory Stockham FFT building blocks for the
// fused split-step kernels (the transform F_N of Eq. GP1ODE_T).
//
// Layout contract.  A team of T = N/E threads holds one length-N sequence,
// E values per thread in registers: thread t holds positions t + T*e,
// e = 0..E-1 (consecutive threads -> consecutive positions, so global loads
// and stores of a team are coalesced).  A radix-RAD Stockham pass with
// current sub-transform length NS lets butterfly b = t + q*T (q < E/RAD)
// read positions b + r*N/RAD (= register q + r*E/RAD of thread t), multiply
// by W_{NS*RAD}^{(b mod NS) r}, apply the radix-RAD DFT, and write position
// (b div NS)*NS*RAD + (b mod NS) + r*NS.  For the last pass (NS*RAD = N)
// that write position is the read position again, so the last pass needs
// no exchange and the transformed sequence ends in natural order in the
// same register layout.  Every other pass exchanges through padded shared
// memory (one pad slot per 16 values breaks the stride-RAD bank conflicts).
#pragma once

#include "hfs_internal.cuh"

namespace hfs {

// Multiplication by a fixed unit complex number.  In FP32 a rounded
// constant w has |w|^2 - 1 of order 1e-8 with a fixed sign, and since every
// grid point passes through the same constants at every step such a bias
// accumulates linearly over the time steps.  The FP32 path therefore
// carries each constant as an unevaluated sum hi + lo (|w|^2 - 1 ~ 1e-15)
// and multiplies with fused multiply-adds; FP64 uses plain products.
template <typename R> struct RotConst;
template <> struct RotConst<double> {
    static constexpr double c1 = 0.92387953251128675613;  // cos(pi/8)
    static constexpr double s1 = 0.38268343236508977173;  // sin(pi/8)
    static constexpr double r2 = 0.70710678118654752440;  // sqrt(1/2)
};

// a * (wc + i ws)
__device__ __forceinline__ cpx<double> mulw(cpx<double> a, double wc, double ws)
{
    return {a.x * wc - a.y * ws, a.x * ws + a.y * wc};
}
// a * ((ch + cl) + i (sh + sl)), compensated
__device__ __forceinline__ cpx<float> mulw2(cpx<float> a, float ch, float cl, float sh, float sl)
{
    const float tr = fmaf(a.x, cl, -a.y * sl);
    const float ti = fmaf(a.x, sl, a.y * cl);
    return {fmaf(a.x, ch, fmaf(-a.y, sh, tr)), fmaf(a.x, sh, fmaf(a.y, ch, ti))};
}
// v * sqrt(1/2), compensated
__device__ __forceinline__ float mul_r2(float v)
{
    constexpr float R2H = 0.7071067690849304f, R2L = 1.2101617485882343e-08f;
    return fmaf(v, R2H, v * R2L);
}
__device__ __forceinline__ double mul_r2(double v) { return v * RotConst<double>::r2; }

// a * exp(-2 pi i k / 16) for a compile-time k (forward); INV conjugates.
template <int K, bool INV, typename R> __device__ __forceinline__ cpx<R> rot16(cpx<R> a)
{
    constexpr int k = INV ? ((16 - (K % 16)) % 16) : (K % 16);
    if constexpr (k == 0) return a;
    else if constexpr (k == 4) return {a.y, -a.x};   // * (-i)
    else if constexpr (k == 8) return {-a.x, -a.y};  // * (-1)
    else if constexpr (k == 12) return {-a.y, a.x};  // * (+i)
    else if constexpr (k == 2) return {mul_r2(a.x + a.y), mul_r2(a.y - a.x)};    // (1 - i)/sqrt2
    else if constexpr (k == 6) return {mul_r2(a.y - a.x), -mul_r2(a.x + a.y)};   // (-1 - i)/sqrt2
    else if constexpr (k == 10) return {-mul_r2(a.x + a.y), mul_r2(a.x - a.y)};  // (-1 + i)/sqrt2
    else if constexpr (k == 14) return {mul_r2(a.x - a.y), mul_r2(a.x + a.y)};   // (1 + i)/sqrt2
    else {
        // odd k: w = (cos(pi k/8), -sin(pi k/8)) = (+-C, +-S) with C, S in {cos(pi/8), sin(pi/8)}
        constexpr bool c_is_c1 = (k == 1 || k == 7 || k == 9 || k == 15);
        constexpr int csign = (k == 1 || k == 3 || k == 13 || k == 15) ? 1 : -1;
        constexpr int ssign = (k == 9 || k == 11 || k == 13 || k == 15) ? 1 : -1;
        if constexpr (sizeof(R) == 4) {
            constexpr float C1H = 0.9238795042037964f, C1L = 2.830748968563057e-08f;
            constexpr float S1H = 0.3826834261417389f, S1L = 6.2233507236442165e-09f;
            constexpr float ch = c_is_c1 ? C1H : S1H, cl = c_is_c1 ? C1L : S1L;
            constexpr float sh = c_is_c1 ? S1H : C1H, sl = c_is_c1 ? S1L : C1L;
            return mulw2(a, csign * ch, csign * cl, ssign * sh, ssign * sl);
        } else {
            constexpr double c = c_is_c1 ? RotConst<double>::c1 : RotConst<double>::s1;
            constexpr double sn = c_is_c1 ? RotConst<double>::s1 : RotConst<double>::c1;
            return mulw(a, csign * c, ssign * sn);
        }
    }
}

// In-place DFT of RAD values: X_k = sum_j a_j exp(-+2 pi i jk/RAD).
template <bool INV, typename R> __device__ __forceinline__ void dft2(cpx<R> &a0, cpx<R> &a1)
{
    cpx<R> t = a0;
    a0 = cadd(t, a1);
    a1 = csub(t, a1);
}

template <bool INV, typename R>
__device__ __forceinline__ void dft4(cpx<R> &a0, cpx<R> &a1, cpx<R> &a2, cpx<R> &a3)
{
    cpx<R> t0 = cadd(a0, a2), t1 = csub(a0, a2);
    cpx<R> t2 = cadd(a1, a3), t3 = rot16<4, INV>(csub(a1, a3));
    a0 = cadd(t0, t2);
    a2 = csub(t0, t2);
    a1 = cadd(t1, t3);
    a3 = csub(t1, t3);
}

// FP32 radix-4 in packed two-lane instructions; the multiplication by -+i
// folds into the last two.  Bit-identical to dft4<INV, float>.
template <bool INV>
__device__ __forceinline__ void dft4p(cpx<float> &a0, cpx<float> &a1, cpx<float> &a2, cpx<float> &a3)
{
    const cpx<float> t0 = cadd_p(a0, a2), t1 = csub_p(a0, a2);
    const cpx<float> t2 = cadd_p(a1, a3), d = csub_p(a1, a3);
    a0 = cadd_p(t0, t2);
    a2 = csub_p(t0, t2);
    a1 = cadd_rot_p<INV ? -1 : 1>(t1, d);
    a3 = cadd_rot_p<INV ? 1 : -1>(t1, d);
}
// Radix-4 stages of the radix-16 and radix-8 butterflies in packed FP32
// (both measured faster than the scalar form).
#ifndef HFS_PACK_DFT16
#define HFS_PACK_DFT16 1
#endif
#ifndef HFS_PACK_DFT8
#define HFS_PACK_DFT8 1
#endif
template <bool INV, bool PACK, typename R>
__device__ __forceinline__ void dft4s(cpx<R> &a0, cpx<R> &a1, cpx<R> &a2, cpx<R> &a3)
{
    if constexpr (PACK && sizeof(R) == 4) dft4p<INV>(a0, a1, a2, a3);
    else dft4<INV>(a0, a1, a2, a3);
}

template <bool INV, typename R> __device__ __forceinline__ void dft4v(cpx<R> *a) { dft4<INV>(a[0], a[1], a[2], a[3]); }

// radix 8 = 2 x 4: even/odd radix-4 transforms combined with W_8^k
template <bool INV, typename R> __device__ __forceinline__ void dft8v(cpx<R> *a)
{
    cpx<R> e0 = a[0], e1 = a[2], e2 = a[4], e3 = a[6];
    cpx<R> o0 = a[1], o1 = a[3], o2 = a[5], o3 = a[7];
    dft4s<INV, HFS_PACK_DFT8 != 0>(e0, e1, e2, e3);
    dft4s<INV, HFS_PACK_DFT8 != 0>(o0, o1, o2, o3);
    o1 = rot16<2, INV>(o1);
    o2 = rot16<4, INV>(o2);
    o3 = rot16<6, INV>(o3);
    a[0] = cadd(e0, o0);
    a[4] = csub(e0, o0);
    a[1] = cadd(e1, o1);
    a[5] = csub(e1, o1);
    a[2] = cadd(e2, o2);
    a[6] = csub(e2, o2);
    a[3] = cadd(e3, o3);
    a[7] = csub(e3, o3);
}

// radix 16 = 4 x 4: X_{k1 + 4 k2} = sum_{j1} W_16^{j1 k1} W_4^{j1 k2} [sum_{j2} a_{j1+4 j2} W_4^{j2 k1}]
template <bool INV, typename R> __device__ __forceinline__ void dft16v(cpx<R> *a)
{
    // inner radix-4 over j2 for each j1 -> b[j1][k1] stored at a[j1 + 4 j2] with j2 := k1
    dft4s<INV, HFS_PACK_DFT16 != 0>(a[0], a[4], a[8], a[12]);
    dft4s<INV, HFS_PACK_DFT16 != 0>(a[1], a[5], a[9], a[13]);
    dft4s<INV, HFS_PACK_DFT16 != 0>(a[2], a[6], a[10], a[14]);
    dft4s<INV, HFS_PACK_DFT16 != 0>(a[3], a[7], a[11], a[15]);
    // twiddles W_16^{j1 k1}: element a[j1 + 4 k1]
    a[5] = rot16<1, INV>(a[5]);
    a[9] = rot16<2, INV>(a[9]);
    a[13] = rot16<3, INV>(a[13]);
    a[6] = rot16<2, INV>(a[6]);
    a[10] = rot16<4, INV>(a[10]);
    a[14] = rot16<6, INV>(a[14]);
    a[7] = rot16<3, INV>(a[7]);
    a[11] = rot16<6, INV>(a[11]);
    a[15] = rot16<9, INV>(a[15]);
    // outer radix-4 over j1 for each k1 -> X_{k1 + 4 k2}
    cpx<R> x[16];
#pragma unroll
    for (int k1 = 0; k1 < 4; ++k1) {
        cpx<R> b0 = a[4 * k1 + 0], b1 = a[4 * k1 + 1], b2 = a[4 * k1 + 2], b3 = a[4 * k1 + 3];
        dft4s<INV, HFS_PACK_DFT16 != 0>(b0, b1, b2, b3);
        x[k1 + 0] = b0;
        x[k1 + 4] = b1;
        x[k1 + 8] = b2;
        x[k1 + 12] = b3;
    }
#pragma unroll
    for (int i = 0; i < 16; ++i) a[i] = x[i];
}

template <int RAD, bool INV, typename R> __device__ __forceinline__ void dft_any(cpx<R> *a)
{
    if constexpr (RAD == 2) dft2<INV>(a[0], a[1]);
    else if constexpr (RAD == 4) dft4v<INV>(a);
    else if constexpr (RAD == 8) dft8v<INV>(a);
    else if constexpr (RAD == 16) dft16v<INV>(a);
    else static_assert(RAD == 2, "unsupported radix");
}

// Twiddle tables (layout: tw_pass_offset): FP32 entries are (hi.re, hi.im,
// lo.re, lo.im) with hi + lo the FP64 value; FP64 entries are plain.
template <typename R> struct TwOf;
template <> struct TwOf<float> { using type = float4; };
template <> struct TwOf<double> { using type = double2; };

// Table element type: TWC (compensated) FP32 twiddles are (hi, lo) pairs;
// without TWC a plain FP32 table (the rounded value only) serves kernels
// whose norm is restored every sub-stage (the projected 1D step), where the
// systematic norm bias of rounded twiddles does not accumulate.
template <typename R, bool TWC> struct TwTab { using type = typename TwOf<R>::type; };
template <> struct TwTab<float, false> { using type = float2; };

// a * w (forward) or a * conj(w) (inverse), w = tw[i]
template <bool INV> __device__ __forceinline__ cpx<float> tw_mul(cpx<float> a, const float2 *tw, int i)
{
    const float2 w = __ldg(tw + i);
    return INV ? cpx<float>{fmaf(a.x, w.x, a.y * w.y), fmaf(a.y, w.x, -(a.x * w.y))}
               : cpx<float>{fmaf(a.x, w.x, -(a.y * w.y)), fmaf(a.x, w.y, a.y * w.x)};
}
template <bool INV> __device__ __forceinline__ cpx<float> tw_mul(cpx<float> a, const float4 *tw, int i)
{
    const float4 w = __ldg(tw + i);
    return INV ? mulw2(a, w.x, w.z, -w.y, -w.w) : mulw2(a, w.x, w.z, w.y, w.w);
}
template <bool INV> __device__ __forceinline__ cpx<double> tw_mul(cpx<double> a, const double2 *tw, int i)
{
    const double2 w = __ldg(tw + i);
    return INV ? mulw(a, w.x, -w.y) : mulw(a, w.x, w.y);
}

// padded shared-memory index (one pad slot per 16 values)
__device__ __forceinline__ int spad(int p) { return p + (p >> 4); }
__host__ __device__ constexpr int smem_elems(int n) { return n + n / 16; }

// Shared-memory slots.  ILV == 1: the team owns a private region padded by
// one slot per 16 values.  ILV > 1: ILV teams interleave element by element
// (the caller offsets sm by its team index), so that a warp whose lanes are
// different teams at the same position touches consecutive addresses.
//
// Every access pattern of a pass is a runtime base A plus a compile-time
// offset c with (A mod 16) + (c mod 16) < 16 (true for all power-of-two
// plans: A = t for the reads, A = (b - j) RAD + j for the writes), so
// pad(A + c) = pad(A) + c + c/16 splits into one base register and an
// immediate offset.
template <int ILV> __device__ __forceinline__ int sbase(int a)
{
    if constexpr (ILV == 1) return a + (a >> 4);
    else return a * ILV;
}
template <int ILV> __host__ __device__ constexpr int soff(int c)
{
    if constexpr (ILV == 1) return c + (c >> 4);
    else return c * ILV;
}

// Barrier around a shared-memory exchange.  TEAM = false: the whole CTA.
// TEAM = true: only the T threads of the team that owns the buffer (named
// barrier `bar`, or the warp when a team fits in one), so the teams of a CTA
// holding several short transforms do not wait for one another.
template <int T, bool TEAM> __device__ __forceinline__ void exchange_sync(int bar)
{
    if constexpr (!TEAM || T >= kCtaThreads) {
        __syncthreads();
    } else if constexpr (T <= 32) {
        __syncwarp();
    } else {
        static_assert(T % 32 == 0, "a named barrier counts whole warps");
        asm volatile("bar.sync %0, %1;" ::"r"(bar), "n"(T) : "memory");
    }
}

// One Stockham pass; see the layout contract at the top of the file.
template <int N, int E, int RAD, int NS, bool INV, bool LAST, int ILV, bool TEAM, typename R, bool TWC = true>
__device__ __forceinline__ void stockham_pass(cpx<R> (&v)[E], cpx<R> *sm, int t,
                                              const typename TwTab<R, TWC>::type *__restrict__ tw, int bar)
{
    constexpr int T = N / E;
    constexpr int Q = E / RAD;
    static_assert(E % RAD == 0, "radix must divide the elements per thread");
    // The twiddles of a thread are the same at every time step; without this
    // opaque copy of the table pointer the compiler hoists all of them out of
    // the time loop and keeps every pass's twiddles live in registers.
    const typename TwTab<R, TWC>::type *twp = tw;
    asm volatile("" : "+l"(twp));
    // likewise the forward and inverse transforms compute identical integer
    // offsets; recomputing them per pass is cheaper than holding them live
    asm volatile("" : "+r"(t));
#pragma unroll
    for (int q = 0; q < Q; ++q) {
        cpx<R> a[RAD];
        const int b = t + q * T;
#pragma unroll
        for (int r = 0; r < RAD; ++r) a[r] = v[q + r * Q];
        const int j = b & (NS - 1);
        if constexpr (NS > 1) {
            // W_{NS RAD}^{j r} from this pass shape's region of the table
            constexpr int64_t OFF = tw_pass_offset(NS * RAD, RAD);
            static_assert(NS * RAD <= kTwiddleMaxLength, "twiddle table too short");
#pragma unroll
            for (int r = 1; r < RAD; ++r) a[r] = tw_mul<INV>(a[r], twp, (int)(OFF + (r - 1) * NS) + j);
        }
        dft_any<RAD, INV>(a);
        if constexpr (LAST) {
#pragma unroll
            for (int r = 0; r < RAD; ++r) v[q + r * Q] = a[r];
        } else {
            cpx<R> *w = sm + sbase<ILV>((b - j) * RAD + j);
#pragma unroll
            for (int r = 0; r < RAD; ++r) w[soff<ILV>(r * NS)] = a[r];
        }
    }
    if constexpr (!LAST) {
        exchange_sync<T, TEAM>(bar);
        const cpx<R> *rd = sm + sbase<ILV>(t);
#pragma unroll
        for (int e = 0; e < E; ++e) v[e] = rd[soff<ILV>(T * e)];
        exchange_sync<T, TEAM>(bar);
    }
}

template <int N, int E, bool INV, int ILV, bool TEAM, typename R, bool TWC, int NS, int RAD, int... REST>
__device__ __forceinline__ void fft_passes(cpx<R> (&v)[E], cpx<R> *sm, int t,
                                           const typename TwTab<R, TWC>::type *__restrict__ tw, int bar)
{
    stockham_pass<N, E, RAD, NS, INV, sizeof...(REST) == 0, ILV, TEAM, R, TWC>(v, sm, t, tw, bar);
    if constexpr (sizeof...(REST) > 0)
        fft_passes<N, E, INV, ILV, TEAM, R, TWC, NS * RAD, REST...>(v, sm, t, tw, bar);
}

// Radix sequences per (N, elements per thread, ALT: the alternative order).
template <int N, int E, bool ALT = false> struct FftPlan;
#define HFS_PLAN(NN, EE, ...) HFS_PLAN_ORDER(NN, EE, false, __VA_ARGS__)
#define HFS_PLAN_ORDER(NN, EE, AA, ...)                                                                \
    template <> struct FftPlan<NN, EE, AA> {                                                            \
        template <bool INV, typename R, int ILV = 1, bool TEAM = false, bool TWC = true>                \
        static __device__ __forceinline__ void run(cpx<R> (&v)[EE], cpx<R> *sm, int t,                   \
                                                   const typename TwTab<R, TWC>::type *tw, int bar = 0) \
        {                                                                                               \
            fft_passes<NN, EE, INV, ILV, TEAM, R, TWC, 1, __VA_ARGS__>(v, sm, t, tw, bar);              \
        }                                                                                               \
    };
HFS_PLAN(4096, 16, 16, 16, 16)
HFS_PLAN(2048, 16, 16, 16, 8)
HFS_PLAN(1024, 16, 16, 16, 4)
HFS_PLAN(512, 16, 16, 16, 2)
HFS_PLAN(256, 16, 16, 16)
HFS_PLAN(128, 16, 16, 8)
HFS_PLAN(64, 16, 16, 4)
HFS_PLAN(32, 16, 16, 2)
HFS_PLAN(32, 8, 8, 4)
HFS_PLAN(16, 8, 8, 2)
HFS_PLAN(2048, 8, 8, 8, 8, 4)
HFS_PLAN(1024, 8, 8, 8, 8, 2)
HFS_PLAN(512, 8, 8, 8, 8)
HFS_PLAN(256, 8, 8, 8, 4)
HFS_PLAN(128, 8, 8, 8, 2)
HFS_PLAN(64, 8, 8, 8)
// four values per thread (n <= 1024: at most 256 threads per instance)
HFS_PLAN(1024, 4, 4, 4, 4, 4, 4)
HFS_PLAN(512, 4, 4, 4, 4, 4, 2)
HFS_PLAN(256, 4, 4, 4, 4, 4)
HFS_PLAN(128, 4, 4, 4, 4, 2)
// sixteen values per thread, alternative radix orders
HFS_PLAN_ORDER(4096, 16, true, 8, 8, 8, 8)
HFS_PLAN_ORDER(2048, 16, true, 8, 16, 16)
HFS_PLAN_ORDER(1024, 16, true, 4, 16, 16)
HFS_PLAN_ORDER(512, 16, true, 2, 16, 16)
HFS_PLAN_ORDER(256, 16, true, 4, 4, 16)
HFS_PLAN_ORDER(128, 16, true, 8, 16)
#undef HFS_PLAN
#undef HFS_PLAN_ORDER

}  // namespace hfs
