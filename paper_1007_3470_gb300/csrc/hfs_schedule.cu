// hfs_schedule.cu -- device-side FP64 schedule of the Magnus and
// decomposition coefficients.
//
// Kernel 1 (stage_flow_kernel): for every instance, stage and axis, the
// harmonic flow of one A stage over [tau, tau + a_i h] as kick(f) .
// drift(g) . kick(e), e applied first:
//   * exact flow for constant omega (Lemma 2 with mu, omega):
//       g = sin(omega s)/(mu omega), f = e = mu omega tan(omega s/2);
//   * commutator-free Magnus-4 (Eq. CommutatorFree): two half steps with
//       omega_L^2 = al w1 + be w2, omega_R^2 = be w1 + al w2 (R first),
//       w_k = omega^2(tau + c_k s), c = 1/2 -+ sqrt(3)/6, al = 1/2 - 1/sqrt3,
//     decomposed by Theorem 2;
//   * sixth-order Magnus (Sec. 4.2), omega^2 read at the three Gauss nodes,
//     decomposed by Theorem 1.
// The trigonometric quantities are written in the forms C(w,t)=cos(sqrt(w)t)
// and S(w,t)=sin(sqrt(w)t)/sqrt(w), continued to w <= 0, with
// 1 - cos = 2 sin^2(half angle), so that no difference of nearly equal
// numbers is formed for small steps.
//
// Kernel 2 (records kernels): merges adjacent chirps and B flows as in
// Eq. prod-genHarmOsc -- the kick between drifts i and i+1 is f_i + e_{i+1}
// and the B flows at a step boundary add (b_{m+1} + b_1) h (FSAL) -- and
// converts every coefficient into phase "turns" per unit integer index:
//   kick   kappa x^2/2 / (2 pi),   x = xc + m dx
//          -> K2 = kappa dx^2/(4 pi), K1 = kappa xc dx/(2 pi), K0 = kappa xc^2/(4 pi) mod 1
//   drift  g k^2/2 / (2 pi),       k = 2 pi m_k / L  ->  G = g pi / L^2
//   B      s (eps V_I + sigma |u|^2) / (2 pi)       ->  sb2pi = s / (2 pi)
// For the F split (Eq. FourierSplit) the drift is g = a_i h / mu and the
// trap mu omega^2(tau) x^2/2 of every B flow joins the kick at its frozen
// time.
#include <math.h>

#include <algorithm>
#include <cstdint>

#include "hfs_internal.cuh"
#include "hfs_law.cuh"
#include "hfs_sched.h"

namespace hfs {

// C = cos(sqrt(w) t), S = sin(sqrt(w) t)/sqrt(w), OMC = 1 - C, continued to w <= 0
struct CS {
    double C, S, OMC;
};
__device__ CS cs_of(double w, double t)
{
    CS r;
    const double z = w * t * t;  // theta^2, negative for w < 0
    if (fabs(z) <= 1e-3) {
        // the same series to z^3: the first omitted terms, z^4/10! and z^4/9!,
        // are below 3e-18 of the sums
        const double c = fma(fma(fma(-z, 1.0 / 40320.0, 1.0 / 720.0), -z, 1.0 / 24.0), -z, 0.5);
        const double sv = fma(fma(fma(-z, 1.0 / 5040.0, 1.0 / 120.0), -z, 1.0 / 6.0), -z, 1.0);
        r.OMC = z * c;
        r.C = 1.0 - r.OMC;
        r.S = t * sv;
        return r;
    }
    if (fabs(z) <= 0.25) {
        // Power series of the entire functions in z = w t^2 (Taylor series of
        // cos and sin / theta), eight terms: truncation below 1e-18.  No square
        // root, no division, and w <= 0 needs no separate branch.
        double c = 1.0 / 20922789888000.0, s = 1.0 / 1307674368000.0;
        c = fma(c, -z, 1.0 / 87178291200.0);
        c = fma(c, -z, 1.0 / 479001600.0);
        c = fma(c, -z, 1.0 / 3628800.0);
        c = fma(c, -z, 1.0 / 40320.0);
        c = fma(c, -z, 1.0 / 720.0);
        c = fma(c, -z, 1.0 / 24.0);
        c = fma(c, -z, 1.0 / 2.0);  // (1 - C)/z
        s = fma(s, -z, 1.0 / 6227020800.0);
        s = fma(s, -z, 1.0 / 39916800.0);
        s = fma(s, -z, 1.0 / 362880.0);
        s = fma(s, -z, 1.0 / 5040.0);
        s = fma(s, -z, 1.0 / 120.0);
        s = fma(s, -z, 1.0 / 6.0);
        s = fma(s, -z, 1.0);  // S / t
        r.OMC = z * c;
        r.C = 1.0 - r.OMC;
        r.S = t * s;
        return r;
    }
    if (w > 0.0) {
        const double q = sqrt(w);
        double sh, ch;
        sincos(0.5 * q * t, &sh, &ch);
        r.C = 1.0 - 2.0 * sh * sh;
        r.OMC = 2.0 * sh * sh;
        r.S = 2.0 * sh * ch / q;
    } else {
        const double q = sqrt(-w);
        const double sh = sinh(0.5 * q * t), ch = cosh(0.5 * q * t);
        r.C = 1.0 + 2.0 * sh * sh;
        r.OMC = -2.0 * sh * sh;
        r.S = 2.0 * sh * ch / q;
    }
    return r;
}

// Theorem 2 for the product of two half steps (R applied first), mu = 1
__device__ void fge_thm2(double wl, double wr, double s, double &f, double &g, double &e)
{
    const CS L = cs_of(wl, 0.5 * s), Rr = cs_of(wr, 0.5 * s);
    g = L.S * Rr.C + L.C * Rr.S;
    const double omcc = L.OMC + L.C * Rr.OMC;  // 1 - C_L C_R
    const double ss = L.S * Rr.S;
    const double ig = 1.0 / g;
    f = (omcc + wl * ss) * ig;
    e = (omcc + wr * ss) * ig;
}

// Theorem 1 for exp(-i s/2 (al x^2 + be (xp+px) + ga p^2))
__device__ void fge_thm1(double al, double be, double ga, double s, double &f, double &g, double &e)
{
    const CS r = cs_of(al * ga - be * be, s);
    g = ga * r.S;
    const double ig = 1.0 / g;
    f = (r.OMC + be * r.S) * ig;
    e = (r.OMC - be * r.S) * ig;
}

constexpr double kR3 = 0.28867513459481288225;   // sqrt(3)/6
constexpr double kR15 = 0.38729833462074168852;  // sqrt(15)/10

// The trap's shape factors S (omega^2 = omega0^2 S) of one stage over
// [tau, tau + s] at the nodes its flow reads: the stage start (Lemma 2), the
// two Gauss nodes (Magnus-4), the three Gauss nodes (Magnus-6).
struct NodeS {
    double s[3];
};

template <int FLOW, int LAW> __device__ __forceinline__ NodeS stage_nodes(const DevInst &p, double tau, double s)
{
    NodeS r{};
    if constexpr (FLOW == HFS_FLOW_LEMMA2) {
        r.s[0] = law_factor<LAW>(p, tau);
    } else if constexpr (FLOW == HFS_FLOW_CF4) {
        law_factor_pair<LAW>(p, tau + 0.5 * s, kR3 * s, r.s[0], r.s[1]);
    } else {
        law_factor_pair<LAW>(p, tau + 0.5 * s, kR15 * s, r.s[0], r.s[2]);
        r.s[1] = law_factor<LAW>(p, tau + 0.5 * s);
    }
    return r;
}

// (f, g, e) of one stage on axis `axis` from the shape factors at its nodes.
// FLOW (and LAW, SHARED below) are template parameters: with a run-time flow
// the compiler evaluated all three branches and kept one result (3.6x the
// FP64 work).
template <int FLOW>
__device__ void stage_fge(const DevInst &p, int dim, int axis, const NodeS &ns, double s, double &f, double &g,
                          double &e)
{
    const double c = (dim == 1) ? 1.0 : p.axis_scale[axis];
    const double k = c * c * (p.w0 * p.w0);  // omega^2 = k S
    if constexpr (FLOW == HFS_FLOW_LEMMA2) {
        const double om = sqrt(k * ns.s[0]);
        double sh, ch;
        sincos(0.5 * om * s, &sh, &ch);
        g = 2.0 * sh * ch / om;
        f = om * sh / ch;
        e = f;
    } else if constexpr (FLOW == HFS_FLOW_CF4) {
        const double al = 0.5 - 2.0 * kR3;  // 1/2 - 1/sqrt(3)
        const double be = 1.0 - al;
        const double w1 = k * ns.s[0], w2 = k * ns.s[1];
        fge_thm2(al * w1 + be * w2, be * w1 + al * w2, s, f, g, e);
    } else {
        const double w1 = k * ns.s[0], w2 = k * ns.s[1], w3 = k * ns.s[2];
        const double s2 = s * s;
        const double avg = 5.0 * w1 + 8.0 * w2 + 5.0 * w3;
        const double al = avg / 18.0 + s2 / 486.0 * (4.25 * (w1 * w1 + w3 * w3) + 8.0 * w2 * w2 + w1 * w2 +
                                                     w2 * w3 - 18.5 * w1 * w3);
        const double be = s * 1.29099444873580562839 * (w3 - w1) * (1.0 / 12.0 + s2 / 3240.0 * avg);  // sqrt(5/3)
        const double ga = 1.0 + s2 / 54.0 * (w1 - 2.0 * w2 + w3);
        fge_thm1(al, be, ga, s, f, g, e);
    }
    // mass: the mu-problem is the mu = 1 problem conjugated by diag(1, mu)
    if (p.mu != 1.0) {
        f *= p.mu;
        e *= p.mu;
        g /= p.mu;
    }
}

// the shape factors of every stage of the chunk, once for a batch whose
// instances share the law and its parameters (read from instance 0)
template <int FLOW, int LAW>
__global__ void law_nodes_kernel(const DevInst *__restrict__ inst, SchedConst sc, const double *__restrict__ t_dev,
                                 double t_off, int nstage, NodeS *__restrict__ nodes)
{
    const int sg = blockIdx.x * blockDim.x + threadIdx.x;
    if (sg >= nstage) return;
    const int n = sg / sc.m, st = sg - n * sc.m;
    const double tau = *t_dev + t_off + (double)n * sc.h + sc.h * sc.cuma[st];
    nodes[sg] = stage_nodes<FLOW, LAW>(inst[0], tau, sc.a[st] * sc.h);
}

// one thread per (instance, time step of the chunk), all m stages of the
// step: instance = blockIdx.x, steps strided over blockIdx.y / threadIdx.x
// (no 64-bit integer division in the index arithmetic).  SHARED: the shape
// factors come from law_nodes_kernel instead of being evaluated per instance.
template <int FLOW, int LAW, bool SHARED>
__global__ void stage_flow_kernel(const DevInst *__restrict__ inst, int dim, SchedConst sc,
                                  const double *__restrict__ t_dev, double t_off, int nsteps,
                                  const NodeS *__restrict__ nodes, StageFGE *__restrict__ out, unsigned *status)
{
    const int64_t i = blockIdx.x;
    const DevInst p = inst[i];
    const double t0 = *t_dev + t_off;
    const int64_t nstage = (int64_t)nsteps * sc.m;
    for (int n = blockIdx.y * blockDim.x + threadIdx.x; n < nsteps; n += gridDim.y * blockDim.x) {
        for (int st = 0; st < sc.m; ++st) {
            const double tau = t0 + (double)n * sc.h + sc.h * sc.cuma[st];
            const double s = sc.a[st] * sc.h;
            const int64_t sg = (int64_t)n * sc.m + st;
            NodeS ns;
            if constexpr (SHARED) ns = nodes[sg];
            else ns = stage_nodes<FLOW, LAW>(p, tau, s);
            for (int d = 0; d < dim; ++d) {
                double f, g, e;
                stage_fge<FLOW>(p, dim, d, ns, s, f, g, e);
                if (!isfinite(f) || !isfinite(g) || !isfinite(e)) atomicOr(status, (unsigned)ST_NONFINITE);
                StageFGE r;
                r.f = f;
                r.g = g;
                r.e = e;
                r.tau = tau;
                out[(i * nstage + sg) * dim + d] = r;
            }
        }
    }
}

// kick coefficient kappa, B sum and drift g of sub-stage j on axis d
template <int SPLIT>
__device__ void merged_coeffs(const DevInst &p, int dim, int d, const SchedConst &sc, double t0, int j, int nstage,
                              const StageFGE *__restrict__ fge_i, double &kappa, double &bs, double &g)
{
    const int mm = sc.m;
    const int r = j % mm;
    if (r == 0) bs = (j > 0 ? sc.b[mm] : 0.0) + (j < nstage ? sc.b[0] : 0.0);
    else bs = sc.b[r];
    if constexpr (SPLIT == HFS_SPLIT_HO) {
        kappa = 0.0;
        if (j >= 1) kappa += fge_i[(j - 1) * dim + d].f;
        if (j < nstage) kappa += fge_i[j * dim + d].e;
        g = (j < nstage) ? fge_i[j * dim + d].g : 0.0;
    } else {
        // F split: B carries mu omega^2(tau_j) x^2/2 with the time frozen at the stage boundary
        const double tau = t0 + (double)(j / mm) * sc.h + sc.h * sc.cuma[r];
        kappa = bs * sc.h * p.mu * axis_omega2(p, dim, d, tau);
        g = (j < nstage) ? sc.a[r] * sc.h / p.mu : 0.0;
    }
}

__device__ __forceinline__ void split_hi_lo(double v, float &hi, float &lo)
{
    hi = (float)v;
    lo = (float)(v - (double)hi);
}

__device__ __forceinline__ double frac1(double v) { return v - rint(v); }

constexpr double kPi = 3.14159265358979323846;
constexpr double kInv4Pi = 0.079577471545947667884;  // 1/(4 pi)
constexpr double kInv2Pi = 0.15915494309189533577;   // 1/(2 pi)

// the phase record of 1D sub-stage j (turns per integer index, see above)
// per-instance factors of the turn coefficients: dx^2/(4 pi), xc dx/(2 pi),
// xc^2/(4 pi), pi/L^2, h/(2 pi)
struct RecScale {
    double k2, k1, k0, g, sb;
};
__device__ __forceinline__ RecScale rec_scale(const DevInst &p, const SchedConst &sc)
{
    RecScale c;
    c.k2 = p.dx[0] * p.dx[0] * kInv4Pi;
    c.k1 = p.xc[0] * p.dx[0] * kInv2Pi;
    c.k0 = p.xc[0] * p.xc[0] * kInv4Pi;
    c.g = kPi / (p.len[0] * p.len[0]);
    c.sb = sc.h * kInv2Pi;
    return c;
}

template <typename RecT, int SPLIT>
__device__ __forceinline__ void record1d(const DevInst &p, const SchedConst &sc, const RecScale &c, double t0, int j,
                                         int nstage, const StageFGE *__restrict__ fge_i, RecT *out, unsigned *status)
{
    double kappa, bs, g;
    merged_coeffs<SPLIT>(p, 1, 0, sc, t0, j, nstage, fge_i, kappa, bs, g);
    const double K2 = kappa * c.k2;
    const double K1 = kappa * c.k1;
    const double K0 = frac1(kappa * c.k0);
    const double G = g * c.g;
    const double SB = bs * c.sb;
    if (!isfinite(K2) || !isfinite(G) || !isfinite(K1)) atomicOr(status, (unsigned)ST_NONFINITE);
    RecT r;
    if constexpr (sizeof(RecT) == sizeof(RecF)) {
        split_hi_lo(K2, r.k2hi, r.k2lo);
        split_hi_lo(K1, r.k1hi, r.k1lo);
        r.k0 = (float)K0;
        r.sb2pi = (float)SB;
        split_hi_lo(G, r.ghi, r.glo);
    } else {
        r.k2 = K2;
        r.k1 = K1;
        r.k0 = K0;
        r.sb2pi = SB;
        r.g = G;
        r.pad = 0.0;
    }
    *out = r;
}

// one thread per (instance, sub-stage j in [0, nstage]) -- 1D records;
// instance = blockIdx.x, sub-stages strided over blockIdx.y / threadIdx.x
template <typename RecT, int SPLIT>
__global__ void records1d_kernel(const DevInst *__restrict__ inst, SchedConst sc, const double *__restrict__ t_dev,
                                 double t_off, int nstage, const StageFGE *__restrict__ fge, RecT *__restrict__ rec,
                                 unsigned *status)
{
    const int64_t i = blockIdx.x;
    const int64_t nrec = (int64_t)nstage + 1;
    const DevInst p = inst[i];
    const double t0 = *t_dev + t_off;
    // the block's instance factors, computed once (one FP64 division per block, not per record)
    __shared__ RecScale s_c;
    if (threadIdx.x == 0) s_c = rec_scale(p, sc);
    __syncthreads();
    const RecScale c = s_c;
    for (int j = blockIdx.y * blockDim.x + threadIdx.x; j <= nstage; j += gridDim.y * blockDim.x)
        record1d<RecT, SPLIT>(p, sc, c, t0, j, nstage, fge + i * (int64_t)nstage, rec + i * nrec + j, status);
}

// 3D records (symmetric boxes): one per sub-stage, all three axes
template <typename RecT, int SPLIT>
__global__ void records3d_kernel(const DevInst *__restrict__ inst, SchedConst sc, const double *__restrict__ t_dev,
                                 double t_off, int nstage, const StageFGE *__restrict__ fge,
                                 RecT *__restrict__ rec, unsigned *status)
{
    const int j = blockIdx.x * blockDim.x + threadIdx.x;
    if (j > nstage) return;
    const DevInst p = inst[0];
    const double t0 = *t_dev + t_off;
    RecT r;
    double SB = 0.0;
    for (int d = 0; d < 3; ++d) {
        double kappa, bs, g;
        merged_coeffs<SPLIT>(p, 3, d, sc, t0, j, nstage, fge, kappa, bs, g);
        const double K2 = kappa * p.dx[d] * p.dx[d] / (4.0 * kPi);
        const double G = g * kPi / (p.len[d] * p.len[d]);
        SB = bs * sc.h / (2.0 * kPi);
        if (!isfinite(K2) || !isfinite(G)) atomicOr(status, (unsigned)ST_NONFINITE);
        if constexpr (sizeof(r.k2[0]) == sizeof(float)) {
            split_hi_lo(K2, r.k2[d], r.k2lo[d]);
            split_hi_lo(G, r.g[d], r.glo[d]);
        } else {
            r.k2[d] = K2;
            r.g[d] = G;
            r.k2lo[d] = 0.0;
            r.glo[d] = 0.0;
        }
    }
    r.sb2pi = SB;
    rec[j] = r;
}

__global__ void set_time_kernel(double *t_dev, double t) { *t_dev = t; }
__global__ void advance_time_kernel(double *t_dev, double dt) { *t_dev += dt; }

// ---------------------------------------------------------------------------
// host launchers
// ---------------------------------------------------------------------------
static inline unsigned blocks_for(int64_t n, int bs) { return (unsigned)((n + bs - 1) / bs); }

int uniform_law(const hfs_instance *inst, int64_t count)
{
    if (count < 1) return -1;
    for (int64_t i = 1; i < count; ++i)
        if (inst[i].omega_law != inst[0].omega_law) return -1;
    return inst[0].omega_law;
}

bool law_shared(const hfs_instance *inst, int64_t count)
{
    if (uniform_law(inst, count) < 0) return false;
    for (int64_t i = 1; i < count; ++i)
        for (int k = 0; k < 3; ++k)
            if (inst[i].law[k] != inst[0].law[k]) return false;
    return true;
}

size_t law_nodes_bytes(int64_t nstage) { return sizeof(NodeS) * (size_t)nstage; }

template <int FLOW, int LAW>
static void launch_stage_flow_fl(bool shared, dim3 grid, const DevInst *inst, int dim, const SchedConst &sc,
                                 const double *t_dev, double t_off, int nsteps, void *nodes, StageFGE *out,
                                 unsigned *status, cudaStream_t st)
{
    NodeS *nd = static_cast<NodeS *>(nodes);
    if constexpr (LAW >= 0) {
        if (shared && nd) {
            const int nstage = nsteps * sc.m;
            law_nodes_kernel<FLOW, LAW><<<blocks_for(nstage, 128), 128, 0, st>>>(inst, sc, t_dev, t_off, nstage, nd);
            stage_flow_kernel<FLOW, LAW, true><<<grid, 128, 0, st>>>(inst, dim, sc, t_dev, t_off, nsteps, nd, out,
                                                                      status);
            return;
        }
    }
    stage_flow_kernel<FLOW, LAW, false><<<grid, 128, 0, st>>>(inst, dim, sc, t_dev, t_off, nsteps, nullptr, out,
                                                               status);
}

template <int FLOW>
static void launch_stage_flow_law(int law, bool shared, dim3 grid, const DevInst *inst, int dim, const SchedConst &sc,
                                  const double *t_dev, double t_off, int nsteps, void *nodes, StageFGE *out,
                                  unsigned *status, cudaStream_t st)
{
#define HFS_SF(L) launch_stage_flow_fl<FLOW, L>(shared, grid, inst, dim, sc, t_dev, t_off, nsteps, nodes, out, status, st)
    switch (law) {
    case HFS_OMEGA_CONST: HFS_SF(HFS_OMEGA_CONST); break;
    case HFS_OMEGA_SIN: HFS_SF(HFS_OMEGA_SIN); break;
    case HFS_OMEGA_COS_SQ: HFS_SF(HFS_OMEGA_COS_SQ); break;
    case HFS_OMEGA_PULSE: HFS_SF(HFS_OMEGA_PULSE); break;
    default: HFS_SF(-1); break;
    }
#undef HFS_SF
}

cudaError_t launch_stage_flow(const DevInst *inst, int64_t count, int dim, const SchedConst &sc, const double *t_dev,
                              double t_off, int64_t nstage, int uniform_law, bool shared, void *nodes,
                              StageFGE *out, unsigned *status, cudaStream_t st)
{
    if (count == 0 || nstage == 0) return cudaSuccess;
    if (nstage >= INT32_MAX || nstage % sc.m != 0 || count > INT32_MAX) return cudaErrorInvalidValue;
    const int nsteps = (int)(nstage / sc.m);
    const dim3 grid((unsigned)count, std::min(blocks_for(nsteps, 128), 65535u));
    switch (sc.flow) {
    case HFS_FLOW_LEMMA2:
        launch_stage_flow_law<HFS_FLOW_LEMMA2>(uniform_law, shared, grid, inst, dim, sc, t_dev, t_off, nsteps, nodes,
                                               out, status, st);
        break;
    case HFS_FLOW_CF4:
        launch_stage_flow_law<HFS_FLOW_CF4>(uniform_law, shared, grid, inst, dim, sc, t_dev, t_off, nsteps, nodes,
                                            out, status, st);
        break;
    default:
        launch_stage_flow_law<HFS_FLOW_M6>(uniform_law, shared, grid, inst, dim, sc, t_dev, t_off, nsteps, nodes,
                                           out, status, st);
        break;
    }
    return cudaGetLastError();
}

cudaError_t launch_records1d(bool fp64, const DevInst *inst, int64_t count, const SchedConst &sc, const double *t_dev,
                             double t_off, int64_t nstage, const StageFGE *fge, void *rec, unsigned *status,
                             cudaStream_t st)
{
    if (count == 0) return cudaSuccess;
    if (nstage >= INT32_MAX || count > INT32_MAX) return cudaErrorInvalidValue;
    const dim3 grid((unsigned)count, std::min(blocks_for(nstage + 1, 128), 65535u));
    const bool ho = sc.split == HFS_SPLIT_HO;
    if (fp64 && ho)
        records1d_kernel<RecD, HFS_SPLIT_HO><<<grid, 128, 0, st>>>(inst, sc, t_dev, t_off, (int)nstage, fge, (RecD *)rec, status);
    else if (fp64)
        records1d_kernel<RecD, HFS_SPLIT_FOURIER><<<grid, 128, 0, st>>>(inst, sc, t_dev, t_off, (int)nstage, fge, (RecD *)rec, status);
    else if (ho)
        records1d_kernel<RecF, HFS_SPLIT_HO><<<grid, 128, 0, st>>>(inst, sc, t_dev, t_off, (int)nstage, fge, (RecF *)rec, status);
    else
        records1d_kernel<RecF, HFS_SPLIT_FOURIER><<<grid, 128, 0, st>>>(inst, sc, t_dev, t_off, (int)nstage, fge, (RecF *)rec, status);
    return cudaGetLastError();
}

cudaError_t launch_records3d(bool fp64, const DevInst *inst, const SchedConst &sc, const double *t_dev, double t_off,
                             int64_t nstage, const StageFGE *fge, void *rec, unsigned *status, cudaStream_t st)
{
    const int64_t n = nstage + 1;
    if (nstage >= INT32_MAX) return cudaErrorInvalidValue;
    const unsigned b = blocks_for(n, 128);
    const bool ho = sc.split == HFS_SPLIT_HO;
    if (fp64 && ho)
        records3d_kernel<Rec3D, HFS_SPLIT_HO><<<b, 128, 0, st>>>(inst, sc, t_dev, t_off, (int)nstage, fge, (Rec3D *)rec, status);
    else if (fp64)
        records3d_kernel<Rec3D, HFS_SPLIT_FOURIER><<<b, 128, 0, st>>>(inst, sc, t_dev, t_off, (int)nstage, fge, (Rec3D *)rec, status);
    else if (ho)
        records3d_kernel<Rec3F, HFS_SPLIT_HO><<<b, 128, 0, st>>>(inst, sc, t_dev, t_off, (int)nstage, fge, (Rec3F *)rec, status);
    else
        records3d_kernel<Rec3F, HFS_SPLIT_FOURIER><<<b, 128, 0, st>>>(inst, sc, t_dev, t_off, (int)nstage, fge, (Rec3F *)rec, status);
    return cudaGetLastError();
}

cudaError_t launch_set_time(double *t_dev, double t, cudaStream_t st)
{
    set_time_kernel<<<1, 1, 0, st>>>(t_dev, t);
    return cudaGetLastError();
}

cudaError_t launch_advance_time(double *t_dev, double dt, cudaStream_t st)
{
    advance_time_kernel<<<1, 1, 0, st>>>(t_dev, dt);
    return cudaGetLastError();
}

}  // namespace hfs
