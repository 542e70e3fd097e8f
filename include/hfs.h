/*
 * hfs.h -- C ABI of the GB300 (sm_103a) Hermite-Fourier split-step library.
 *
 * The library advances the 1D or 3D Gross-Pitaevskii / linear Schrodinger
 * equation with a perturbed, possibly time-dependent harmonic trap,
 *     i psi_t = ( p^2/(2 mu) + mu omega^2(t) x^2 / 2 ) psi
 *               + ( eps V_I(x) + sigma |psi|^2 ) psi                (Eq. GP1, GP1b)
 * on a periodic grid x_j = lo + j dx, dx = (hi - lo)/N (Eq. GP1ODE), by the
 * Hermite-Fourier splitting of Bader & Blanes (arXiv 1007.3470, Sec. 3):
 * each A stage (the harmonic flow, exact by Lemma 2 or Magnus-approximated
 * by Eq. CommutatorFree / the sixth-order Magnus of Sec. 4.2) is written as
 * chirp . kinetic . chirp (Theorems 1, 2), and composed with the pointwise
 * flow of eps V_I + sigma |psi|^2 (Lemma 1) by the m-stage compositions of
 * Eq. prod-gen / Table 1 with the frozen-time algorithm of Table
 * "algorithm"; adjacent chirps and B flows are merged as in
 * Eq. prod-genHarmOsc, so one step costs m forward + m inverse FFTs.
 *
 * Conventions for every entry point:
 *  - All functions return an int status (HFS_OK == 0); nothing throws or
 *    aborts across the ABI.  hfs_error_string() names a status.
 *  - The library performs NO device allocation.  The caller owns the state
 *    buffer psi and the workspace (e.g. torch tensors) and binds them with
 *    hfs_bind(); their sizes come from hfs_state_size() and
 *    hfs_workspace_size().  Both must stay valid until hfs_destroy() or the
 *    next hfs_bind().  The context itself is a small host allocation.
 *  - Device work is enqueued asynchronously on the stream given to
 *    hfs_set_stream() (default: the legacy default stream).  Calls that
 *    return host data (hfs_norm, hfs_energy, hfs_get_psi to host,
 *    hfs_sync_status) synchronise that stream.
 *  - psi is interleaved complex: complex64 (2 x float) for HFS_C64 or
 *    complex128 (2 x double) for HFS_C128.  A 1D batch is the concatenation
 *    of its instances in order (offsets from hfs_instance_offset()); a 3D
 *    instance is row-major with axis 0 (x) fastest.
 *  - Asynchronous device-side problems (non-finite coefficients, an
 *    exhausted bounded wait) are recorded in a device status word that
 *    hfs_sync_status() reads and clears.
 */
#ifndef HFS_H
#define HFS_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

#define HFS_API_VERSION 1

/* ---- status codes ------------------------------------------------------ */
#define HFS_OK 0
#define HFS_ERR_INVALID_ARG 1    /* null pointer, bad enum, bad size */
#define HFS_ERR_UNSUPPORTED 2    /* grid size / dim / precision not built */
#define HFS_ERR_STEP_TOO_LARGE 3 /* |a_i h| omega_max >= pi: outside the validity of Lemma 2 / Thms 1-2 */
#define HFS_ERR_CUDA 4           /* a CUDA runtime call failed */
#define HFS_ERR_NONFINITE 5      /* non-finite coefficient or state detected */
#define HFS_ERR_NOT_READY 6      /* buffers not bound or schedule not set */
#define HFS_ERR_ALIGNMENT 7      /* psi or workspace not 256-byte aligned */
#define HFS_ERR_WORKSPACE 8      /* bound workspace smaller than required */
#define HFS_ERR_DEVICE_TIMEOUT 9 /* a bounded device-side wait ran out */

/* ---- enums ------------------------------------------------------------- */
#define HFS_C64 0  /* complex64 state, FP32 bulk arithmetic */
#define HFS_C128 1 /* complex128 state, FP64 throughout (parity mode) */

/* omega(t) of Eq. GP1b; per axis omega_d = axis_scale[d] * omega in 3D */
#define HFS_OMEGA_CONST 0  /* omega = w0 */
#define HFS_OMEGA_SIN 1    /* omega = w0 (1 + law[0] sin(law[1] t + law[2])) */
#define HFS_OMEGA_COS_SQ 2 /* omega^2 = w0^2 (1 + law[0] cos(law[1] t))   (Sec. 4.2) */
#define HFS_OMEGA_PULSE 3  /* omega = w0 (1 + law[0] t / cosh^2(law[1] (t - law[2])))  (Sec. 4.2) */

/* perturbation V_I(x), separable: sum over axes of v(x_d) */
#define HFS_VI_NONE 0
#define HFS_VI_X4 1  /* v(x) = x^4 */
#define HFS_VI_COS 2 /* v(x) = cos(vi_k x) */

/* splittings (Sec. 2.1) */
#define HFS_SPLIT_HO 0      /* A = p^2/2mu + mu omega^2 x^2/2, B = eps V_I + sigma|psi|^2 (Eq. HermiteSplit) */
#define HFS_SPLIT_FOURIER 1 /* A = p^2/2mu, B = mu omega^2 x^2/2 + eps V_I + sigma|psi|^2 (Eq. FourierSplit) */

/* harmonic flow of one A stage under the HO split */
#define HFS_FLOW_LEMMA2 0 /* exact flow for constant omega (Lemma 2) */
#define HFS_FLOW_CF4 1    /* 4th-order commutator-free Magnus (Eq. CommutatorFree) + Theorem 2 */
#define HFS_FLOW_M6 2     /* 6th-order Magnus (Sec. 4.2) + Theorem 1 */

/* compositions (BAB form: m A-stages, m+1 B-stages; Eq. LeapFrogB, Table 1) */
#define HFS_COMP_STRANG 0
#define HFS_COMP_SRKN6_4 1
#define HFS_COMP_NI4_82 2
#define HFS_COMP_NI5_84 3
#define HFS_COMP_CUSTOM 4

/* execution modes of the 1D batched step */
#define HFS_MODE_RESIDENT 0  /* every step of a call on-chip: one load + one store per instance */
#define HFS_MODE_STREAMING 1 /* steps_per_launch steps per launch, one global round trip each */

/* ---- problem description ----------------------------------------------- */
typedef struct {
    int32_t n[3];          /* grid points per axis (power of two); 1D uses n[0] */
    double lo[3], hi[3];   /* periodic box [lo_d, hi_d) */
    double mu;             /* mass (mu > 0) */
    int32_t omega_law;     /* HFS_OMEGA_* */
    double w0;             /* base frequency */
    double law[3];         /* law parameters, see HFS_OMEGA_* */
    double axis_scale[3];  /* 3D: omega_d = axis_scale[d] * omega(t); ignored in 1D */
    double eps;            /* perturbation strength */
    int32_t vi_kind;       /* HFS_VI_* */
    double vi_k;           /* wavenumber for HFS_VI_COS */
    double sigma;          /* nonlinearity (>0 repulsive, <0 attractive) */
} hfs_instance;

typedef struct hfs_ctx_s *hfs_ctx_t;

/* ---- lifecycle --------------------------------------------------------- */

/* Create a context for `count` 1D instances (dim == 1; each n[0] in
 * {128, ..., 4096}) or for one 3D instance (dim == 3, count == 1, n = 128^3
 * or 32^3 / 64^3 per axis, all axes equal).  `inst` is a host array that is
 * copied.  precision: HFS_C64 or HFS_C128.  Needs a current CUDA device.
 * Errors: HFS_ERR_INVALID_ARG, HFS_ERR_UNSUPPORTED, HFS_ERR_CUDA. */
int hfs_create(hfs_ctx_t *ctx, int dim, int precision, const hfs_instance *inst, int64_t count);

/* Release the context (host memory only; caller-owned buffers untouched). */
void hfs_destroy(hfs_ctx_t ctx);

/* Stream for all later device work (a cudaStream_t, or NULL). */
int hfs_set_stream(hfs_ctx_t ctx, void *cuda_stream);

/* Total complex elements of the state and its size in bytes. */
int hfs_state_size(hfs_ctx_t ctx, int64_t *elems, size_t *bytes);

/* Element offset of instance i inside the state buffer. */
int hfs_instance_offset(hfs_ctx_t ctx, int64_t i, int64_t *elem_offset);

/* Workspace bytes needed when hfs_step() processes at most `chunk_steps`
 * steps per schedule chunk (longer calls are split into chunks). */
int hfs_workspace_size(hfs_ctx_t ctx, int64_t chunk_steps, size_t *bytes);

/* Bind caller-owned device buffers: psi (state_size bytes) and a workspace
 * of work_bytes (>= hfs_workspace_size for the chunk length given).  Both
 * 256-byte aligned.  Initialises the workspace tables on the stream.
 * Errors: HFS_ERR_INVALID_ARG, HFS_ERR_ALIGNMENT, HFS_ERR_WORKSPACE. */
int hfs_bind(hfs_ctx_t ctx, void *psi_dev, void *work_dev, size_t work_bytes, int64_t chunk_steps);

/* ---- schedule (Sec. 2, Table "algorithm"; Sec. 3) ---------------------- */

/* Choose the splitting, the harmonic flow and the composition, and the time
 * step dt (may be negative).  For HFS_COMP_CUSTOM pass a[na], b[nb] with
 * nb == na + 1 (b_1 applied first); otherwise a/b may be NULL.  The
 * validity |a_i dt| omega_max < pi is checked per instance at hfs_step().
 * Errors: HFS_ERR_INVALID_ARG. */
int hfs_set_schedule(hfs_ctx_t ctx, int split, int ho_flow, int composition, const double *a, int na,
                     const double *b, int nb, double dt);

/* Execution mode of the 1D step (default HFS_MODE_RESIDENT) and, for
 * HFS_MODE_STREAMING, the number of steps fused per launch (>= 1). */
int hfs_set_mode(hfs_ctx_t ctx, int mode, int steps_per_launch);

/* Norm projection of the 1D complex64 step (enable != 0; default off).  The
 * exact scheme conserves the discrete norm dx sum |psi_j|^2 (every sub-flow is
 * a pure phase in x or k: Lemma 1, Eq. GP1ODE_T), but FP32 rounding in the
 * FFT passes and phases changes it by small unbiased amounts that add up as
 * a random walk (rms ~ 8e-7 after 500 steps for a state covering ~15 grid
 * points).  With projection on, each sub-stage rescales every instance by
 * sqrt(N0 / N_j), N_0 the sum of |psi|^2 at the start of the hfs_step() call
 * and N_j the current one (both measured in FP32 inside the fused kernel),
 * which removes the radial component of the rounding error instead of
 * letting it accumulate; the paper's method itself has no such step.  With
 * the projection the step kernels read plain FP32 twiddles (the compensated
 * table only stops a systematic norm bias, which the projection removes).
 * 3D (complex64, 128 points per axis): each plane pass sums |psi|^2 in its
 * x-phase and the z-pass that follows applies the factor, the target being
 * the sum at the start of the hfs_step() call.
 * Errors: HFS_ERR_UNSUPPORTED for complex128 contexts (drift ~1e-14) and 3D
 * grids other than 128^3. */
int hfs_set_norm_projection(hfs_ctx_t ctx, int enable);

/* Engine of the radix-16 DFT stages of the 3D z-transform (the first pass of
 * each forward and inverse FFT along z, Eq. GP1ODE_T), complex64 with n = 64
 * or 128 per axis:
 *   HFS_DFT_SIMT          butterflies on the FP32 pipes (default);
 *   HFS_DFT_TENSOR_3XTF32 each CTA's 256 length-16 DFTs as one real matrix
 *                         product on the tensor cores (tcgen05), operands
 *                         split into two TF32 parts, three products
 *                         accumulated in FP32.
 * Errors: HFS_ERR_INVALID_ARG (unknown engine), HFS_ERR_UNSUPPORTED (1D,
 * complex128, or another grid size). */
#define HFS_DFT_SIMT 0
#define HFS_DFT_TENSOR_3XTF32 1
int hfs_set_dft_engine(hfs_ctx_t ctx, int engine);

/* Capture each hfs_step(nsteps) launch sequence in a CUDA graph and replay
 * it on later calls with the same nsteps (enable != 0).  Capture needs a
 * stream other than the legacy default stream: hfs_step() returns
 * HFS_ERR_INVALID_ARG when graphs are enabled and the stream is NULL. */
int hfs_set_graphs(hfs_ctx_t ctx, int enable);

/* Schedule reuse for 1D contexts (enable != 0; default off).  The phase
 * records of a call (the FP64 stage flows of Lemma 2 / Theorems 1-2 merged
 * as in Eq. prod-genHarmOsc) depend only on the call's start time, its step
 * count and the schedule, so with reuse on the context keeps two record
 * buffers, each tagged with the call it holds: a call of at most one chunk
 * whose records are held skips the FP64 schedule kernels, and each call
 * computes the records of the call that would follow it (start time
 * t + nsteps dt) on an internal stream, in parallel with its fused step
 * kernel, which it launches at the device's highest scheduling priority so
 * that the schedule fills only the SMs that the step kernel leaves.  The
 * records, and so the results, are bit-identical to those computed in line.
 * Any change of schedule, instances, plans, stream or buffers drops the held
 * records.  The second buffer enlarges the workspace (hfs_workspace_size
 * reports the size with the current setting): when the bound workspace is too
 * small the context is left unbound and HFS_ERR_WORKSPACE is returned; bind
 * again with a workspace of the new size.
 * Errors: HFS_ERR_UNSUPPORTED (3D), HFS_ERR_WORKSPACE, HFS_ERR_CUDA. */
int hfs_set_schedule_reuse(hfs_ctx_t ctx, int enable);

/* Current time t_n (host copy; advanced by hfs_step). */
int hfs_set_time(hfs_ctx_t ctx, double t);
int hfs_get_time(hfs_ctx_t ctx, double *t);

/* ---- state ------------------------------------------------------------- */

/* Copy a full state (state_size bytes) into / out of the bound psi buffer.
 * on_device != 0: src/dst is device memory, else host memory. */
int hfs_set_psi(hfs_ctx_t ctx, const void *src, int src_on_device);
int hfs_get_psi(hfs_ctx_t ctx, void *dst, int dst_on_device);

/* Advance every instance by nsteps steps of the schedule from the current
 * time (asynchronous).  Errors: HFS_ERR_NOT_READY, HFS_ERR_STEP_TOO_LARGE,
 * HFS_ERR_CUDA. */
int hfs_step(hfs_ctx_t ctx, int64_t nsteps);

/* ---- diagnostics ------------------------------------------------------- */

/* Discrete norm dV sum_j |psi_j|^2 per instance (FP64 accumulation), into
 * the host array out[count]. */
int hfs_norm(hfs_ctx_t ctx, double *out);

/* Energy per instance at the current time:
 * dV sum_j [ |grad psi|^2/(2 mu) + V(x_j,t)|psi_j|^2 + sigma/2 |psi_j|^4 ],
 * V = mu omega^2(t) x^2 / 2 + eps V_I; gradient spectral.  Host out[count]. */
int hfs_energy(hfs_ctx_t ctx, double *out);

/* Wait for the stream, then read and clear the device status word. */
int hfs_sync_status(hfs_ctx_t ctx);

/* ---- plans / autotuning (1D) ------------------------------------------- */

/* Plan of the grid size n: plan = elements per thread (16, 8 for n <= 2048,
 * 4 for n <= 1024), | HFS_PLAN_ALT_ORDER for the alternative order of the
 * Stockham radices with 16 values per thread (radix 8 throughout at n = 4096,
 * the small radix first otherwise).  4 values per thread and the alternative
 * order are complex64 only.  Affects later hfs_step calls.
 * Errors: HFS_ERR_UNSUPPORTED. */
#define HFS_PLAN_ALT_ORDER 0x100
int hfs_set_plan(hfs_ctx_t ctx, int n, int plan);

/* CTAs per SM of the persistent 1D step grid (0: as many as fit, the
 * default; values above that are clamped). */
int hfs_set_occupancy(hfs_ctx_t ctx, int ctas_per_sm);

/* Search the 1D plans with CUDA-event timings of trial_steps steps of the
 * whole batch in the current mode (resident or streaming): coordinate
 * descent from 8 values per thread for n <= 1024 and 16 above, two rounds
 * over the grid sizes present, each trying every
 * admissible plan of that size (16, 8, 4 values per thread, the alternative
 * radix order) with the others fixed, keeping the fastest batch time; then
 * one CTA per SM against as many as fit.  Overwrites the state: call before
 * hfs_set_psi.  best_plans[6] (host, may be NULL) receives the chosen plan
 * (as for hfs_set_plan) for n = 128 ... 4096, 0 where the size is absent. */
int hfs_autotune(hfs_ctx_t ctx, int trial_steps, int32_t *best_plans);

/* hfs_autotune with a persistent cache: the JSON file at `path` holds tuned
 * plans keyed by the GPU name and SM count, the precision, a hash of the
 * library's sources, the perturbation-kind variant, the norm projection, the
 * mode, the schedule (flow, split, stages) and the batch's count of
 * instances per grid size.  A matching entry is applied without timing
 * anything (*hit = 1); otherwise the search runs, its plans take effect and
 * its result is added to the file (*hit = 0; written to path.tmp and renamed;
 * a file that cannot be written is left as it is).
 * Errors: as hfs_autotune. */
int hfs_autotune_cache(hfs_ctx_t ctx, const char *path, int trial_steps, int32_t *best_plans, int *hit);

/* ---- profiling -------------------------------------------------------- */

/* enable != 0: record CUDA events on the context's stream around the fused
 * step-kernel launches of every hfs_step() (also inside captured graphs). */
int hfs_set_profiling(hfs_ctx_t ctx, int enable);

/* Device time in ms from the first to the last fused step-kernel launch of
 * the most recent hfs_step() (synchronises on its end event).  Errors:
 * HFS_ERR_NOT_READY when profiling is off or no step ran. */
int hfs_last_step_kernel_ms(hfs_ctx_t ctx, float *ms);

/* ---- allocation-free batched step -------------------------------------- */

/* The paper has no counterpart to this entry point; it exists for callers
 * that cannot allocate device memory -- code that runs where cudaMalloc is
 * not allowed or not wanted (allocator or memory-pool callbacks, a device
 * memory budget fixed at start-up, a host library that is only handed a
 * device pointer to the state) and therefore cannot provide the workspace
 * that hfs_bind() needs.
 *
 * Advances `count` 1D instances (host array inst, n[0] in 128..4096) whose
 * states are concatenated in the device buffer psi (complex64 for HFS_C64,
 * complex128 for HFS_C128, 8/16-byte aligned; read and overwritten in place)
 * by nsteps steps of size dt from time t0, with the given split, harmonic
 * flow and built-in composition (HFS_COMP_CUSTOM is not accepted), on the
 * given stream (NULL: legacy default stream).  Results equal, bit for bit,
 * those of hfs_step() with a 16-step schedule chunk and the context's
 * defaults (16 values per thread, norm projection off).
 *
 * No device memory is allocated or freed: all scratch lives in one
 * file-scope __device__ array of HFS_NOALLOC_SCRATCH_BYTES that every GPU
 * loading the library keeps until process exit.  The first call on a device
 * resolves the array's address and fills its twiddle tables, synchronising
 * the stream.  Every call
 * reuses the same array, which keeps the previous call's contents (the call
 * clears what must start at zero): calls whose GPU work overlaps -- on
 * different streams, or from different host threads -- race on it and must
 * be serialised by the caller.
 *
 * wait != 0: synchronise the stream before returning and report a non-finite
 * state as HFS_ERR_NONFINITE.  With wait == 0 the call returns once the work
 * is enqueued, and device-side problems (a non-finite state) are not
 * reported to the caller: the status word that records them lives in the
 * shared array and is cleared by the next call.  Errors: HFS_ERR_WORKSPACE when count exceeds
 * HFS_NOALLOC_MAX_INSTANCES; HFS_ERR_INVALID_ARG, HFS_ERR_UNSUPPORTED,
 * HFS_ERR_ALIGNMENT, HFS_ERR_STEP_TOO_LARGE, HFS_ERR_CUDA as for the
 * context API. */
#define HFS_NOALLOC_MAX_INSTANCES 512
#define HFS_NOALLOC_SCRATCH_BYTES (6u << 20)
int hfs_step1d_noalloc(void *psi, int precision, const hfs_instance *inst, int64_t count, int split, int ho_flow,
                       int composition, double dt, double t0, int64_t nsteps, void *stream, int wait);

const char *hfs_error_string(int status);

#ifdef __cplusplus
}
#endif
#endif
