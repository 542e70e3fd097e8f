/*
 * hfs_oracle.c -- plain, slow, FP64 CPU oracle for the Hermite-Fourier
 * split step of Bader & Blanes, "Fourier methods for the perturbed harmonic
 * oscillator in linear and nonlinear Schrodinger equations" (arXiv 1007.3470).
 *
 * TEST INFRASTRUCTURE ONLY.  Nothing in the product library links, includes
 * or calls this file; only the tests, the smoke check and the CPU baseline
 * leg of the benchmark do.  It shares no code, header, table or helper with
 * the CUDA path.
 *
 * Everything is applied UNMERGED and in the order the paper applies it:
 * for each stage i of the composition (Sec. 2, Eq. prod-gen, Table
 * "algorithm"): the B sub-flow for b_i h with time frozen at the stage start
 * (Lemma 1), then the A sub-flow over a_i h.  Under the HO split the A flow
 * is the exact (Lemma 2) or Magnus-approximated (Eq. CommutatorFree, Sec. 4.2
 * sixth-order Magnus) harmonic flow, written as  K(f) D(g) K(e)  with the
 * e-kick applied first (Theorems 1 and 2); under the F split it is the plain
 * kinetic drift (Eq. FourierSplit).  A final B sub-flow for b_{m+1} h closes
 * the step (BAB compositions, Table 1).
 *
 * Kick   K(c):  u_j <- exp(-i c x_j^2 / 2) u_j
 * Drift  D(g):  u   <- F^-1 exp(-i g k^2 / 2) F u              (Eq. GP1ODE_T)
 * B(t,s):       u_j <- exp(-i s (eps V_I(x_j) + sigma |u_j|^2)) u_j (Lemma 1)
 *
 * The DFT is either the naive O(N^2) sum or a textbook iterative radix-2
 * Cooley-Tukey FFT; the two are cross-checked by the tests.
 *
 * Parity pins (tests/test_oracle_*.py): brute-force DFT vs FFT and numpy;
 * the 2x2 symplectic identities of Lemma 2 and Theorems 1-2 against
 * scipy.linalg.expm; the one-step ground-state test of Sec. 4; Hermite
 * eigenstate phases; the coherent-state closed form; norm; reversibility;
 * convergence orders; a dense expm check of the discrete linear step; the
 * quadrature conditions of the Table 1 coefficient sets.
 */
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>

#ifdef _OPENMP
#include <omp.h>
#endif

#include "hfs_oracle.h"

#ifndef M_PI
#define M_PI 3.14159265358979323846
#endif

/* ------------------------------------------------------------------ */
/* complex helpers on interleaved (re, im) doubles                     */
/* ------------------------------------------------------------------ */

static void cmul_phase(double *z, double phi)
{
    /* z <- z * exp(-i phi) */
    double c = cos(phi), s = sin(phi);
    double re = z[0], im = z[1];
    z[0] = re * c + im * s;
    z[1] = im * c - re * s;
}

/* ------------------------------------------------------------------ */
/* DFT: naive sum and textbook radix-2 FFT  (Eq. GP1ODE_T)            */
/* ------------------------------------------------------------------ */

/* out_k = sum_j in_j exp(sign * 2 pi i j k / n); no normalisation. */
void or_dft(int n, const double *in, double *out, int sign)
{
    for (int k = 0; k < n; ++k) {
        double sr = 0.0, si = 0.0;
        for (int j = 0; j < n; ++j) {
            /* reduce j*k mod n exactly before forming the angle */
            long long jk = ((long long)j * (long long)k) % n;
            double ang = sign * 2.0 * M_PI * (double)jk / (double)n;
            double c = cos(ang), s = sin(ang);
            sr += in[2 * j] * c - in[2 * j + 1] * s;
            si += in[2 * j] * s + in[2 * j + 1] * c;
        }
        out[2 * k] = sr;
        out[2 * k + 1] = si;
    }
}

static int is_pow2(int n) { return n > 0 && (n & (n - 1)) == 0; }

/* In-place iterative radix-2 decimation-in-time FFT (bit reversal, then
 * log2(n) butterfly sweeps); same sign convention as or_dft.  Returns -1
 * when n is not a power of two. */
int or_fft(int n, double *a, int sign)
{
    if (!is_pow2(n)) return -1;
    /* bit-reversal permutation */
    for (int i = 1, j = 0; i < n; ++i) {
        int bit = n >> 1;
        for (; j & bit; bit >>= 1) j ^= bit;
        j ^= bit;
        if (i < j) {
            double tr = a[2 * i], ti = a[2 * i + 1];
            a[2 * i] = a[2 * j];
            a[2 * i + 1] = a[2 * j + 1];
            a[2 * j] = tr;
            a[2 * j + 1] = ti;
        }
    }
    for (int len = 2; len <= n; len <<= 1) {
        int half = len >> 1;
        for (int k = 0; k < half; ++k) {
            double ang = sign * 2.0 * M_PI * (double)k / (double)len;
            double wr = cos(ang), wi = sin(ang);
            for (int s = 0; s < n; s += len) {
                double *u = a + 2 * (s + k);
                double *v = a + 2 * (s + k + half);
                double tr = v[0] * wr - v[1] * wi;
                double ti = v[0] * wi + v[1] * wr;
                v[0] = u[0] - tr;
                v[1] = u[1] - ti;
                u[0] += tr;
                u[1] += ti;
            }
        }
    }
    return 0;
}

/* forward (sign -1) or inverse (sign +1, scaled by 1/n) 1D transform of a
 * strided line */
static void transform_line(int n, double *base, long stride, int sign, int naive, double *tmp, double *tmp2)
{
    for (int j = 0; j < n; ++j) {
        tmp[2 * j] = base[2 * (long)j * stride];
        tmp[2 * j + 1] = base[2 * (long)j * stride + 1];
    }
    if (naive) {
        or_dft(n, tmp, tmp2, sign);
        memcpy(tmp, tmp2, sizeof(double) * 2 * n);
    } else {
        or_fft(n, tmp, sign);
    }
    double sc = (sign > 0) ? 1.0 / n : 1.0;
    for (int j = 0; j < n; ++j) {
        base[2 * (long)j * stride] = tmp[2 * j] * sc;
        base[2 * (long)j * stride + 1] = tmp[2 * j + 1] * sc;
    }
}

/* ------------------------------------------------------------------ */
/* grid (Eq. GP1ODE: x_i = a + i dx, dx = (b - a)/N; k as in the DFT)  */
/* ------------------------------------------------------------------ */

static long total_points(const or_problem *p)
{
    long n = 1;
    for (int d = 0; d < p->dim; ++d) n *= p->n[d];
    return n;
}

static double grid_x(const or_problem *p, int d, int j)
{
    double dx = (p->b[d] - p->a[d]) / p->n[d];
    return p->a[d] + j * dx;
}

static double grid_k(const or_problem *p, int d, int j)
{
    int n = p->n[d];
    double L = p->b[d] - p->a[d];
    int m = (j < n / 2) ? j : j - n;
    return 2.0 * M_PI / L * (double)m;
}

/* index -> (j0, j1, j2), axis 0 fastest */
static void unravel(const or_problem *p, long idx, int *j)
{
    j[0] = j[1] = j[2] = 0;
    for (int d = 0; d < p->dim; ++d) {
        j[d] = (int)(idx % p->n[d]);
        idx /= p->n[d];
    }
}

/* ------------------------------------------------------------------ */
/* trap laws (Eq. GP1b, Sec. 4.2) and the perturbation V_I             */
/* ------------------------------------------------------------------ */

/* omega^2(t) of the base law (before the per-axis scale c_d) */
double or_omega2(const or_problem *p, double t)
{
    double w;
    switch (p->omega_law) {
    case OR_OMEGA_CONST:
        w = p->w0;
        return w * w;
    case OR_OMEGA_SIN: /* omega = w0 (1 + A sin(W t + phi)) */
        w = p->w0 * (1.0 + p->law[0] * sin(p->law[1] * t + p->law[2]));
        return w * w;
    case OR_OMEGA_COS_SQ: /* omega^2 = w0^2 (1 + A cos(W t)) */
        return p->w0 * p->w0 * (1.0 + p->law[0] * cos(p->law[1] * t));
    case OR_OMEGA_PULSE: { /* omega = w0 (1 + A t / cosh^2(B (t - t_c))) */
        double ch = cosh(p->law[1] * (t - p->law[2]));
        w = p->w0 * (1.0 + p->law[0] * t / (ch * ch));
        return w * w;
    }
    default:
        return NAN;
    }
}

static double axis_omega2(const or_problem *p, int d, double t)
{
    double c = (p->dim == 1) ? 1.0 : p->axis_scale[d];
    return c * c * or_omega2(p, t);
}

/* V_I at a point: separable sum over axes of v(x_d) */
static double vi_at(const or_problem *p, const int *j)
{
    double v = 0.0;
    for (int d = 0; d < p->dim; ++d) {
        double x = grid_x(p, d, j[d]);
        switch (p->vi_kind) {
        case OR_VI_NONE: break;
        case OR_VI_X4: v += x * x * x * x; break;
        case OR_VI_COS: v += cos(p->vi_k * x); break;
        default: v += NAN;
        }
    }
    return v;
}

/* ------------------------------------------------------------------ */
/* sub-flows                                                           */
/* ------------------------------------------------------------------ */

/* B sub-flow (Lemma 1) for a time s with time frozen at t:
 * u_j <- exp(-i s (eps V_I(x_j) + sigma |u_j|^2)) u_j
 * Under the F split B also carries the trap: + mu omega_d^2(t) x_d^2 / 2. */
static void flow_B(const or_problem *p, double *u, double t, double s)
{
    long np = total_points(p);
    for (long q = 0; q < np; ++q) {
        int j[3];
        unravel(p, q, j);
        double dens = u[2 * q] * u[2 * q] + u[2 * q + 1] * u[2 * q + 1];
        double F = p->eps * vi_at(p, j) + p->sigma * dens;
        if (p->split == OR_SPLIT_FOURIER) {
            for (int d = 0; d < p->dim; ++d) {
                double x = grid_x(p, d, j[d]);
                F += 0.5 * p->mu * axis_omega2(p, d, t) * x * x;
            }
        }
        cmul_phase(u + 2 * q, s * F);
    }
}

/* Kick K(c) along axis d: u <- exp(-i c x_d^2 / 2) u */
static void flow_kick(const or_problem *p, double *u, int d, double c)
{
    long np = total_points(p);
    for (long q = 0; q < np; ++q) {
        int j[3];
        unravel(p, q, j);
        double x = grid_x(p, d, j[d]);
        cmul_phase(u + 2 * q, 0.5 * c * x * x);
    }
}

/* Drift D(g) along axis d (Eq. GP1ODE_T): forward DFT along that axis,
 * multiply by exp(-i g k^2 / 2), inverse DFT. */
static void flow_drift(const or_problem *p, double *u, int d, double g)
{
    int n = p->n[d];
    long stride = 1;
    for (int e = 0; e < d; ++e) stride *= p->n[e];
    long np = total_points(p);
    long nlines = np / n;
    double *tmp = (double *)malloc(sizeof(double) * 2 * n);
    double *tmp2 = (double *)malloc(sizeof(double) * 2 * n);
    double *ph = (double *)malloc(sizeof(double) * n);
    for (int k = 0; k < n; ++k) {
        double kk = grid_k(p, d, k);
        ph[k] = 0.5 * g * kk * kk;
    }
    for (long line = 0; line < nlines; ++line) {
        /* base index of the line: decompose line into (below d, above d) */
        long lo = line % stride, hi = line / stride;
        double *base = u + 2 * (lo + hi * stride * n);
        transform_line(n, base, stride, -1, p->naive_dft, tmp, tmp2);
        for (int k = 0; k < n; ++k) cmul_phase(base + 2 * (long)k * stride, ph[k]);
        transform_line(n, base, stride, +1, p->naive_dft, tmp, tmp2);
    }
    free(tmp);
    free(tmp2);
    free(ph);
}

/* ------------------------------------------------------------------ */
/* harmonic-oscillator flow coefficients                               */
/* ------------------------------------------------------------------ */

/* 1 - cos(th), without cancellation for small th */
static double one_minus_cos(double th)
{
    double s = sin(0.5 * th);
    return 2.0 * s * s;
}

/* Lemma 2 (with mu, omega):  g = sin(omega t)/(mu omega),
 * f = e = mu omega tan(omega t / 2).  Valid for |t| < pi/omega. */
void or_coef_lemma2(double mu, double omega, double t, double *f, double *g, double *e)
{
    *g = sin(omega * t) / (mu * omega);
    *f = mu * omega * tan(0.5 * omega * t);
    *e = *f;
}

/* cos / (sin x / x)-type quantities of a half step with squared frequency w:
 * c = cos(sqrt(w) tau), s = sin(sqrt(w) tau), and the ratios s/omega,
 * omega*s, continued to w <= 0 by cosh / sinh. */
static void half_flow(double w, double tau, double *c, double *s_over_om, double *om_s, double *omc)
{
    if (w > 0.0) {
        double om = sqrt(w);
        double th = om * tau;
        *c = cos(th);
        *s_over_om = sin(th) / om;
        *om_s = om * sin(th);
        *omc = one_minus_cos(th);
    } else if (w < 0.0) {
        double om = sqrt(-w);
        double th = om * tau;
        double sh = sinh(0.5 * th);
        *c = cosh(th);
        *s_over_om = sinh(th) / om;
        *om_s = -om * sinh(th);
        *omc = -2.0 * sh * sh;
    } else {
        *c = 1.0;
        *s_over_om = tau;
        *om_s = 0.0;
        *omc = 0.0;
    }
}

/* Theorem 2: e^{-i t/2 (p^2/2 + w_L x^2/2)} e^{-i t/2 (p^2/2 + w_R x^2/2)}
 *          = K(f) D(g) K(e)  with (c_k, s_k) = (cos, sin)(omega_k t / 2):
 *   g = s_L c_R / om_L + c_L s_R / om_R
 *   f = (1 - c_L c_R + (om_L/om_R) s_L s_R) / g
 *   e = (1 - c_L c_R + (om_R/om_L) s_L s_R) / g
 * (om_L/om_R) s_L s_R is written as (om_L s_L)(s_R/om_R), and
 * 1 - c_L c_R = (1 - c_L) + c_L (1 - c_R), so that the small-t limit and
 * w <= 0 are handled.  Then mu enters as f,e -> mu f, mu e and g -> g/mu
 * (conjugation by diag(1, mu) of the classical 2x2 flow). */
void or_coef_thm2(double mu, double wL, double wR, double t, double *f, double *g, double *e)
{
    double cL, sLo, oSL, omcL, cR, sRo, oSR, omcR;
    half_flow(wL, 0.5 * t, &cL, &sLo, &oSL, &omcL);
    half_flow(wR, 0.5 * t, &cR, &sRo, &oSR, &omcR);
    double gg = sLo * cR + cL * sRo;
    double one_m_cc = omcL + cL * omcR;
    double ff = (one_m_cc + oSL * sRo) / gg;
    double ee = (one_m_cc + oSR * sLo) / gg;
    *f = mu * ff;
    *g = gg / mu;
    *e = mu * ee;
}

/* Theorem 1: e^{-i t/2 (alpha x^2 + beta (xp+px) + gamma p^2)} = K(f) D(g) K(e)
 *   eta = sqrt(alpha gamma - beta^2),  g = gamma sin(eta t)/eta,
 *   f = (1 - cos(eta t) + beta sin(eta t)/eta) / g,
 *   e = (1 - cos(eta t) - beta sin(eta t)/eta) / g.
 * eta^2 <= 0 is continued by sinh / cosh. */
void or_coef_thm1(double alpha, double beta, double gamma, double t, double *f, double *g, double *e)
{
    double eta2 = alpha * gamma - beta * beta;
    double c, so, os, omc;
    half_flow(eta2, t, &c, &so, &os, &omc);
    (void)c;
    (void)os;
    *g = gamma * so;
    *f = (omc + beta * so) / *g;
    *e = (omc - beta * so) / *g;
}

/* Gauss-Legendre nodes of the fourth-order commutator-free Magnus
 * (Eq. CommutatorFree) and its weights alpha, beta. */
static const double CF4_C1 = 0.5 - 0.28867513459481288225; /* 1/2 - sqrt(3)/6 */
static const double CF4_C2 = 0.5 + 0.28867513459481288225;

/* The A flow of one stage over [t0, t0 + s] on axis d under the HO split:
 * returns (f, g, e) of K(f) D(g) K(e). */
int or_stage_coeffs(const or_problem *p, int d, double t0, double s, double *f, double *g, double *e)
{
    double cd = (p->dim == 1) ? 1.0 : p->axis_scale[d];
    switch (p->ho_flow) {
    case OR_FLOW_LEMMA2: {
        double om = sqrt(axis_omega2(p, d, t0));
        or_coef_lemma2(p->mu, om, s, f, g, e);
        return 0;
    }
    case OR_FLOW_CF4: {
        double alpha = 0.5 - 1.0 / sqrt(3.0);
        double beta = 1.0 - alpha;
        double w1 = axis_omega2(p, d, t0 + CF4_C1 * s);
        double w2 = axis_omega2(p, d, t0 + CF4_C2 * s);
        double wL = alpha * w1 + beta * w2;
        double wR = beta * w1 + alpha * w2;
        or_coef_thm2(p->mu, wL, wR, s, f, g, e);
        return 0;
    }
    case OR_FLOW_M6: {
        /* sixth-order Magnus of Sec. 4.2, nodes 1/2 -+ sqrt(15)/10, 1/2;
         * the printed omega_i are read as omega^2 at the nodes. */
        double r = sqrt(15.0) / 10.0;
        double w1 = axis_omega2(p, d, t0 + (0.5 - r) * s);
        double w2 = axis_omega2(p, d, t0 + 0.5 * s);
        double w3 = axis_omega2(p, d, t0 + (0.5 + r) * s);
        double s2 = s * s;
        double al = (5.0 * w1 + 8.0 * w2 + 5.0 * w3) / 18.0
                  + s2 / 486.0 * (17.0 / 4.0 * (w1 * w1 + w3 * w3) + 8.0 * w2 * w2 + w1 * w2 + w2 * w3
                                  - 37.0 / 2.0 * w1 * w3);
        double be = s * sqrt(5.0 / 3.0) * (w3 - w1) * (1.0 / 12.0 + s2 / 3240.0 * (5.0 * w1 + 8.0 * w2 + 5.0 * w3));
        double ga = 1.0 + s2 / 54.0 * (w1 - 2.0 * w2 + w3);
        double ff, gg, ee;
        or_coef_thm1(al, be, ga, s, &ff, &gg, &ee);
        *f = p->mu * ff;
        *g = gg / p->mu;
        *e = p->mu * ee;
        (void)cd;
        return 0;
    }
    default:
        return -1;
    }
}

/* ------------------------------------------------------------------ */
/* one step and the driver                                             */
/* ------------------------------------------------------------------ */

/* One step t -> t + h of the composition (Eq. prod-gen) by the algorithm
 * of Table "algorithm"; BAB form with m A-stages and m+1 B-stages. */
static int one_step(const or_problem *p, double *u, double t)
{
    double tau = t;
    for (int i = 0; i < p->m; ++i) {
        double s_b = p->bcoef[i] * p->h;
        double s_a = p->acoef[i] * p->h;
        flow_B(p, u, tau, s_b);
        if (p->split == OR_SPLIT_HO) {
            for (int d = 0; d < p->dim; ++d) {
                double f, g, e;
                if (or_stage_coeffs(p, d, tau, s_a, &f, &g, &e)) return -1;
                flow_kick(p, u, d, e);
                flow_drift(p, u, d, g);
                flow_kick(p, u, d, f);
            }
        } else {
            for (int d = 0; d < p->dim; ++d) flow_drift(p, u, d, s_a / p->mu);
        }
        tau += s_a;
    }
    flow_B(p, u, tau, p->bcoef[p->m] * p->h);
    return 0;
}

int or_run(const or_problem *p, double *psi, long nsteps)
{
    if (p->dim != 1 && p->dim != 3) return -2;
    for (int d = 0; d < p->dim; ++d)
        if (!is_pow2(p->n[d]) && !p->naive_dft) return -3;
    for (long s = 0; s < nsteps; ++s) {
        double t = p->t0 + (double)s * p->h;
        if (one_step(p, psi, t)) return -1;
    }
    return 0;
}

int or_run_batch(const or_problem *probs, double *const *psis, long count, long nsteps, int nthreads)
{
    int err = 0;
#ifdef _OPENMP
    if (nthreads > 0) omp_set_num_threads(nthreads);
#pragma omp parallel for schedule(dynamic, 1) reduction(| : err)
#endif
    for (long i = 0; i < count; ++i) err |= (or_run(&probs[i], psis[i], nsteps) != 0);
    (void)nthreads;
    return err ? -1 : 0;
}

int or_max_threads(void)
{
#ifdef _OPENMP
    return omp_get_max_threads();
#else
    return 1;
#endif
}

/* ------------------------------------------------------------------ */
/* diagnostics                                                         */
/* ------------------------------------------------------------------ */

static double cell_volume(const or_problem *p)
{
    double v = 1.0;
    for (int d = 0; d < p->dim; ++d) v *= (p->b[d] - p->a[d]) / p->n[d];
    return v;
}

/* discrete norm  dV sum_j |u_j|^2 */
double or_norm(const or_problem *p, const double *psi)
{
    long np = total_points(p);
    double s = 0.0;
    for (long q = 0; q < np; ++q) s += psi[2 * q] * psi[2 * q] + psi[2 * q + 1] * psi[2 * q + 1];
    return s * cell_volume(p);
}

/* energy at time t (not defined in the paper; the GPE functional):
 * dV sum_j [ sum_d |(F^-1 i k_d F u)_j|^2 / (2 mu) + V(x_j, t)|u_j|^2 + sigma/2 |u_j|^4 ],
 * V = sum_d mu omega_d^2(t) x_d^2 / 2 + eps V_I. */
double or_energy(const or_problem *p, const double *psi, double t)
{
    long np = total_points(p);
    double *w = (double *)malloc(sizeof(double) * 2 * np);
    double kin = 0.0;
    for (int d = 0; d < p->dim; ++d) {
        int n = p->n[d];
        long stride = 1;
        for (int e = 0; e < d; ++e) stride *= p->n[e];
        long nlines = np / n;
        double *tmp = (double *)malloc(sizeof(double) * 2 * n);
        double *tmp2 = (double *)malloc(sizeof(double) * 2 * n);
        memcpy(w, psi, sizeof(double) * 2 * np);
        for (long line = 0; line < nlines; ++line) {
            long lo = line % stride, hi = line / stride;
            double *base = w + 2 * (lo + hi * stride * n);
            transform_line(n, base, stride, -1, p->naive_dft, tmp, tmp2);
            for (int k = 0; k < n; ++k) {
                double kk = grid_k(p, d, k);
                double *z = base + 2 * (long)k * stride;
                double re = z[0], im = z[1];
                z[0] = -kk * im; /* i k z */
                z[1] = kk * re;
            }
            transform_line(n, base, stride, +1, p->naive_dft, tmp, tmp2);
        }
        for (long q = 0; q < np; ++q) kin += w[2 * q] * w[2 * q] + w[2 * q + 1] * w[2 * q + 1];
        free(tmp);
        free(tmp2);
    }
    free(w);
    double pot = 0.0, inter = 0.0;
    for (long q = 0; q < np; ++q) {
        int j[3];
        unravel(p, q, j);
        double dens = psi[2 * q] * psi[2 * q] + psi[2 * q + 1] * psi[2 * q + 1];
        double V = p->eps * vi_at(p, j);
        for (int d = 0; d < p->dim; ++d) {
            double x = grid_x(p, d, j[d]);
            V += 0.5 * p->mu * axis_omega2(p, d, t) * x * x;
        }
        pot += V * dens;
        inter += 0.5 * p->sigma * dens * dens;
    }
    return cell_volume(p) * (kin / (2.0 * p->mu) + pot + inter);
}
