/*
 * hfs_fno.h -- C ABI of the Fourier-neural-operator surrogate of the
 * split-step solver (the learned map from an initial state and the problem
 * parameters to the state at a fixed final time; the paper has no learned
 * component -- the surrogate is trained on trajectories of this library's
 * Hermite-Fourier solver, which stays the fallback and the reference for its
 * error).
 *
 * Architecture (channels last, one sample = `grid` points):
 *   H0  = X P_in + b_in                                    lift, in_ch -> width
 *   for each of `layers` layers:
 *       S   = DFT of H over x, truncated to the `modes` lowest wavenumbers
 *       Y_k = S_k R_k   (complex width x width weights per retained mode)
 *       U   = real inverse DFT of Y from those modes (1/grid, factor 2 for k > 0)
 *       Z   = H W + b + U;  H = GELU(Z) (last layer: H = Z)
 *   Q = GELU(H P1 + c1);  O = Q P2 + c2                     projection width -> proj -> out_ch
 *   loss = mean over samples of ||O - Y|| / ||Y||            relative L2
 * Every contraction is a BF16 tensor-core GEMM (mma.sync m16n8k16) with FP32
 * accumulation; master weights, Adam moments and loss are FP32.
 *
 * Parameter vector (FP32, caller-owned, `param_count` floats, in order):
 *   P_in[in_ch][width], b_in[width], then per layer R_re[modes][width][width],
 *   R_im[modes][width][width], W[width][width], b[width]; then
 *   P1[width][proj], c1[proj], P2[proj][out_ch], c2[out_ch].
 * Tensors: x [batch][grid][in_ch] FP32 (device), y [batch][grid][out_ch] FP32.
 *
 * Conventions as in hfs.h: int status returns, no device allocation (caller
 * binds the parameters and a workspace sized by hfs_fno_workspace_size),
 * asynchronous on the stream from hfs_fno_set_stream (NULL: legacy stream).
 */
#ifndef HFS_FNO_H
#define HFS_FNO_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef struct {
    int32_t grid;   /* points per sample (L >= 16) */
    int32_t width;  /* channels of the spectral layers */
    int32_t modes;  /* retained wavenumbers (2 modes <= grid) */
    int32_t layers; /* spectral layers */
    int32_t in_ch;  /* input channels (<= 8) */
    int32_t proj;   /* hidden width of the projection */
    int32_t out_ch; /* output channels */
} hfs_fno_config;

typedef struct hfs_fno_s *hfs_fno_t;

/* Create a model for batches of up to max_batch samples; train != 0 also
 * sizes the backward / optimizer buffers.  Host-only. */
int hfs_fno_create(hfs_fno_t *out, const hfs_fno_config *cfg, int32_t max_batch, int32_t train);
void hfs_fno_destroy(hfs_fno_t f);
int hfs_fno_set_stream(hfs_fno_t f, void *cuda_stream);
int hfs_fno_param_count(hfs_fno_t f, int64_t *count);
int hfs_fno_workspace_size(hfs_fno_t f, size_t *bytes);

/* Bind the FP32 parameter vector and the workspace (both device, 256-byte
 * aligned); builds the DFT matrices and the BF16 weight copies and resets
 * the optimizer state.  Errors: HFS_ERR_ALIGNMENT, HFS_ERR_WORKSPACE. */
int hfs_fno_bind(hfs_fno_t f, float *params_dev, void *work_dev, size_t work_bytes);

/* Deterministic initial parameters from a seed (uniform, fan-in scaled). */
int hfs_fno_init_params(hfs_fno_t f, uint64_t seed);

/* y = model(x) for `batch` samples. */
int hfs_fno_forward(hfs_fno_t f, const float *x_dev, float *y_dev, int32_t batch);

/* Loss of model(x) against y and its gradient with respect to every
 * parameter (FP32, parameter-vector layout) into grad_dev (device, may be
 * NULL to keep it internal); loss_host (may be NULL) receives the loss and
 * makes the call synchronous.  Needs train != 0. */
int hfs_fno_loss_grad(hfs_fno_t f, const float *x_dev, const float *y_dev, int32_t batch, float *grad_dev,
                      float *loss_host);

/* One Adam step (beta1 0.9, beta2 0.999, eps 1e-8, learning rate lr) on the
 * loss of one batch; loss_host as above. */
int hfs_fno_train_step(hfs_fno_t f, const float *x_dev, const float *y_dev, int32_t batch, float lr,
                       float *loss_host);

/* GEMM engine of the row-streaming products (rows >= 8192, K and N of 64 or
 * 128: the pointwise layers, the projection and their backward products).
 * HFS_FNO_GEMM_MMA_SYNC (default): cp.async tile ring and mma.sync.m16n8k16.
 * HFS_FNO_GEMM_TCGEN05: persistent CTAs keep op(B) in shared memory, stream
 * 128-row tiles of A, and run the products on the tcgen05 tensor cores (BF16
 * operands through shared-memory descriptors, FP32 accumulators in tensor
 * memory, one tile's products issued while the previous tile's epilogue
 * runs); at batch 512 it measures slower than the default (its per-tile
 * phases are latency bound with few warps per SM).  Other shapes always use
 * mma.sync.  Errors: HFS_ERR_INVALID_ARG. */
#define HFS_FNO_GEMM_MMA_SYNC 0
#define HFS_FNO_GEMM_TCGEN05 1
int hfs_fno_set_gemm_engine(hfs_fno_t f, int engine);

/* Wait for the context's stream and report device-side problems since the
 * last call: HFS_ERR_DEVICE_TIMEOUT when a tensor-core GEMM's bounded wait
 * for its matrix products ran out (that launch's results were not written);
 * the word is cleared. */
int hfs_fno_sync_status(hfs_fno_t f);

#ifdef __cplusplus
}
#endif
#endif
