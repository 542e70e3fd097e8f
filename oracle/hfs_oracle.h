/*
 * hfs_oracle.h -- interface of the FP64 CPU oracle (test infrastructure
 * only; the product library never includes this header).
 */
#ifndef HFS_ORACLE_H
#define HFS_ORACLE_H

#ifdef __cplusplus
extern "C" {
#endif

enum { OR_OMEGA_CONST = 0, OR_OMEGA_SIN = 1, OR_OMEGA_COS_SQ = 2, OR_OMEGA_PULSE = 3 };
enum { OR_VI_NONE = 0, OR_VI_X4 = 1, OR_VI_COS = 2 };
enum { OR_SPLIT_HO = 0, OR_SPLIT_FOURIER = 1 };
enum { OR_FLOW_LEMMA2 = 0, OR_FLOW_CF4 = 1, OR_FLOW_M6 = 2 };

/* One problem instance: a 1D or 3D periodic grid, the trap, the
 * perturbation and the composition.  Field order is mirrored by the ctypes
 * structure in oracle/oracle.py. */
typedef struct {
    int dim;              /* 1 or 3 */
    int n[3];             /* points per axis (axis 0 fastest in memory) */
    double a[3], b[3];    /* periodic box [a_d, b_d) */
    double mu;
    int omega_law;        /* OR_OMEGA_* */
    double w0;            /* base frequency */
    double law[3];        /* law parameters (A, W, phi) or (A, B, t_c) */
    double axis_scale[3]; /* per-axis c_d (3D): omega_d = c_d omega */
    double eps;
    int vi_kind;          /* OR_VI_* */
    double vi_k;          /* wavenumber of the cosine perturbation */
    double sigma;
    int split;            /* OR_SPLIT_* */
    int ho_flow;          /* OR_FLOW_* */
    int m;                /* number of A stages; bcoef has m + 1 entries */
    const double *acoef;
    const double *bcoef;
    double h;             /* time step (may be negative) */
    double t0;            /* start time */
    int naive_dft;        /* 1: O(N^2) DFT, 0: radix-2 FFT */
} or_problem;

void or_dft(int n, const double *in, double *out, int sign);
int or_fft(int n, double *a, int sign);
double or_omega2(const or_problem *p, double t);
void or_coef_lemma2(double mu, double omega, double t, double *f, double *g, double *e);
void or_coef_thm2(double mu, double wL, double wR, double t, double *f, double *g, double *e);
void or_coef_thm1(double alpha, double beta, double gamma, double t, double *f, double *g, double *e);
int or_stage_coeffs(const or_problem *p, int d, double t0, double s, double *f, double *g, double *e);
int or_run(const or_problem *p, double *psi, long nsteps);
int or_run_batch(const or_problem *probs, double *const *psis, long count, long nsteps, int nthreads);
int or_max_threads(void);
double or_norm(const or_problem *p, const double *psi);
double or_energy(const or_problem *p, const double *psi, double t);

#ifdef __cplusplus
}
#endif
#endif
