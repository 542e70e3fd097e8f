// hfs_fno.cu -- Fourier-neural-operator surrogate of the split-step solver:
// forward, relative-L2 loss, backward and Adam, all in this library's CUDA
// kernels (BF16 tensor-core GEMMs with FP32 accumulation, FP32 master
// weights).  See include/hfs_fno.h for the architecture and the ABI.
#include <math.h>
#include <string.h>

#include <algorithm>
#include <new>
#include <vector>

#include "hfs.h"
#include "hfs_fno.h"
#include "hfs_fno_kernels.cuh"
#include "hfs_fno_tc.cuh"

using namespace hfs::fno;

namespace {

inline size_t al256(size_t v) { return (v + 255) / 256 * 256; }
inline unsigned blocks(int64_t n, int bs = 256) { return (unsigned)((n + bs - 1) / bs); }

struct ParamOffsets {
    int64_t Pin, bin, P1, c1, P2, c2, total;
    std::vector<int64_t> Rre, Rim, W, b;
};

}  // namespace

struct hfs_fno_s {
    hfs_fno_config cfg{};
    int max_batch = 0, train = 0;
    int64_t nparams = 0;
    ParamOffsets po;
    cudaStream_t stream = nullptr;
    float *params = nullptr;
    unsigned char *work = nullptr;
    size_t work_bytes = 0;
    int64_t step = 0;
    int gemm_engine = HFS_FNO_GEMM_MMA_SYNC;  // hfs_fno_set_gemm_engine
    // workspace sections (byte offsets)
    struct {
        size_t X8, Hf, Hb, pre, S, Yf, Yb, U, Qpre, Qb, O, dO, dOb, dQ, dQb, dH, dZ, dZb, dYb, dSb, dR1, dR2, grad, m,
            v, sums, loss, Pinb, Wb, Rb1, Rb2, P1b, P2b, F2, Gre, Gim, status, total;
    } off{};
};

namespace {

constexpr int kInPad = 8;

ParamOffsets param_offsets(const hfs_fno_config &c)
{
    ParamOffsets p;
    int64_t o = 0;
    const int64_t C = c.width, M = c.modes;
    p.Pin = o;
    o += (int64_t)c.in_ch * C;
    p.bin = o;
    o += C;
    for (int l = 0; l < c.layers; ++l) {
        p.Rre.push_back(o);
        o += M * C * C;
        p.Rim.push_back(o);
        o += M * C * C;
        p.W.push_back(o);
        o += C * C;
        p.b.push_back(o);
        o += C;
    }
    p.P1 = o;
    o += C * c.proj;
    p.c1 = o;
    o += c.proj;
    p.P2 = o;
    o += (int64_t)c.proj * c.out_ch;
    p.c2 = o;
    o += c.out_ch;
    p.total = o;
    return p;
}

void layout(hfs_fno_s *f)
{
    const hfs_fno_config &c = f->cfg;
    const int64_t B = f->max_batch, L = c.grid, C = c.width, M = c.modes, P = c.proj, NL = c.layers;
    const int64_t rows = B * L;
    size_t o = 0;
    auto take = [&](size_t bytes) {
        size_t at = o;
        o = al256(o + bytes);
        return at;
    };
    auto &w = f->off;
    w.X8 = take(2 * rows * kInPad);
    w.Hf = take(4 * rows * C * (NL + 1));
    w.Hb = take(2 * rows * C * (NL + 1));
    w.pre = take(4 * rows * C * NL);
    w.S = take(2 * B * 2 * M * C * NL);
    w.Yf = take(4 * M * B * 2 * C);
    w.Yb = take(2 * M * B * 2 * C);
    w.U = take(4 * rows * C);
    w.Qpre = take(4 * rows * P);
    w.Qb = take(2 * rows * P);
    w.O = take(4 * rows * c.out_ch);
    if (f->train) {
        w.dO = take(4 * rows * c.out_ch);
        w.dOb = take(2 * rows * c.out_ch);
        w.dQ = take(4 * rows * P);
        w.dQb = take(2 * rows * P);
        w.dH = take(4 * rows * C);
        w.dZ = take(4 * rows * C);
        w.dZb = take(2 * rows * C);
        w.dYb = take(2 * M * B * 2 * C);
        w.dSb = take(2 * B * 2 * M * C);
        w.dR1 = take(4 * M * C * 2 * C);
        w.dR2 = take(4 * M * C * 2 * C);
        w.grad = take(4 * f->nparams);
        w.m = take(4 * f->nparams);
        w.v = take(4 * f->nparams);
        w.sums = take(4 * 2 * B);
        w.loss = take(4);
    }
    w.Pinb = take(2 * kInPad * C);
    w.Wb = take(2 * C * C * NL);
    w.Rb1 = take(2 * M * C * 2 * C * NL);
    w.Rb2 = take(2 * M * C * 2 * C * NL);
    w.P1b = take(2 * C * P);
    w.P2b = take(2 * P * c.out_ch);
    w.F2 = take(2 * 2 * M * L);
    w.Gre = take(2 * L * M);
    w.Gim = take(2 * L * M);
    w.status = take(4);
    w.total = o;
}

template <typename T> T *at(hfs_fno_s *f, size_t off) { return reinterpret_cast<T *>(f->work + off); }

#define FCK(expr)                                                                                                 \
    do {                                                                                                          \
        if ((expr) != cudaSuccess) return HFS_ERR_CUDA;                                                           \
    } while (0)

GemmArgs gemm(int M, int N, int K, const bf16 *A, int64_t lda, const bf16 *B, int64_t ldb)
{
    GemmArgs g;
    memset(&g, 0, sizeof(g));
    g.M = M;
    g.N = N;
    g.K = K;
    g.A = A;
    g.lda = lda;
    g.B = B;
    g.ldb = ldb;
    g.alpha = 1.0f;
    g.splitk = 1;
    g.batch = 1;
    return g;
}

// tensor-core form (hfs_fno_tc.cuh): persistent, as many CTAs per SM as the
// shared and tensor memory hold
template <bool TB, int NT, int KT> cudaError_t run_tc(const GemmArgs &g, cudaStream_t st)
{
    static int ctas = 0;  // CTAs of the grid per batch slice (SMs x resident CTAs), set once
    auto k = gemm_bf16_tc_kernel<TB, NT, KT>;
    constexpr int smem = tc_smem_bytes<NT, KT>();
    if (ctas == 0) {
        cudaError_t e = cudaFuncSetAttribute(k, cudaFuncAttributeMaxDynamicSharedMemorySize, smem);
        int dev = 0, sms = 0, per = 0;
        if (e == cudaSuccess) e = cudaGetDevice(&dev);
        if (e == cudaSuccess) e = cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
        if (e == cudaSuccess) e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per, k, 128, smem);
        if (e != cudaSuccess) return e;
        ctas = sms * std::max(1, std::min(per, 512 / (2 * NT)));  // tensor memory: two NT-column accumulators
    }
    const int tiles = (g.M + TC_M - 1) / TC_M;
    k<<<dim3((unsigned)std::min(tiles, ctas), (unsigned)g.batch), 128, smem, st>>>(g);
    return cudaGetLastError();
}

// status: the tensor-core form's status word; null selects the mma.sync forms
cudaError_t run(const GemmArgs &g0, bool ta, bool tb, cudaStream_t st, unsigned *status = nullptr)
{
    GemmArgs g = g0;
    g.status = status;
    if (status && gemm_tc_ok(g, ta)) {
        const int key = (tb ? 4 : 0) + (g.N == 128 ? 2 : 0) + (g.K == 128 ? 1 : 0);
        switch (key) {
        case 0: return run_tc<false, 64, 64>(g, st);
        case 1: return run_tc<false, 64, 128>(g, st);
        case 2: return run_tc<false, 128, 64>(g, st);
        case 3: return run_tc<false, 128, 128>(g, st);
        case 4: return run_tc<true, 64, 64>(g, st);
        case 5: return run_tc<true, 64, 128>(g, st);
        case 6: return run_tc<true, 128, 64>(g, st);
        default: return run_tc<true, 128, 128>(g, st);
        }
    }
    const dim3 grid((g.N + GT_N - 1) / GT_N, (g.M + GT_M - 1) / GT_M, g.batch * g.splitk);
    if (gemm_pipe_ok(g, ta, tb)) {
        if (!ta && !tb) gemm_bf16_pipe_kernel<false, false><<<grid, 128, 0, st>>>(g);
        else if (ta && !tb) gemm_bf16_pipe_kernel<true, false><<<grid, 128, 0, st>>>(g);
        else if (!ta && tb) gemm_bf16_pipe_kernel<false, true><<<grid, 128, 0, st>>>(g);
        else gemm_bf16_pipe_kernel<true, true><<<grid, 128, 0, st>>>(g);
        return cudaGetLastError();
    }
    if (!ta && !tb) gemm_bf16_kernel<false, false><<<grid, 128, 0, st>>>(g);
    else if (ta && !tb) gemm_bf16_kernel<true, false><<<grid, 128, 0, st>>>(g);
    else if (!ta && tb) gemm_bf16_kernel<false, true><<<grid, 128, 0, st>>>(g);
    else gemm_bf16_kernel<true, true><<<grid, 128, 0, st>>>(g);
    return cudaGetLastError();
}

// row-split of the column sums: about 64 rows per block
inline unsigned colsum_blocks(int64_t rows) { return (unsigned)std::max<int64_t>(1, std::min<int64_t>(4096, rows / 64)); }

// split-K weight gradient dW (+)= A^T B over `rows` (both row-major, K = rows)
cudaError_t weight_grad(int M, int N, int64_t rows, const bf16 *A, int64_t lda, const bf16 *B, int64_t ldb, float *dW,
                        cudaStream_t st)
{
    GemmArgs g = gemm(M, N, (int)rows, A, lda, B, ldb);
    g.C = dW;
    g.ldc = N;
    const int64_t tiles = (int64_t)((M + GT_M - 1) / GT_M) * ((N + GT_N - 1) / GT_N);
    int64_t split = std::max<int64_t>(1, std::min<int64_t>(1024 / std::max<int64_t>(tiles, 1), rows / 256));
    g.splitk = (int)split;
    return run(g, true, false, st);
}

int refresh_weights(hfs_fno_s *f)
{
    const hfs_fno_config &c = f->cfg;
    const int64_t C = c.width, M = c.modes, P = c.proj;
    cudaStream_t st = f->stream;
    to_bf16_pad_kernel<<<blocks((int64_t)kInPad * C), 256, 0, st>>>(f->params + f->po.Pin, c.in_ch, (int)C,
                                                                     at<bf16>(f, f->off.Pinb), (int)C);
    // P_in is [in_ch][C]: pad rows in_ch..7 with zeros
    if (c.in_ch < kInPad)
        FCK(cudaMemsetAsync(at<bf16>(f, f->off.Pinb) + (int64_t)c.in_ch * C, 0, 2 * (kInPad - c.in_ch) * C, st));
    for (int l = 0; l < c.layers; ++l) {
        to_bf16_kernel<<<blocks(C * C), 256, 0, st>>>(f->params + f->po.W[l], at<bf16>(f, f->off.Wb) + l * C * C, C * C);
        mixing_weights_kernel<<<blocks(M * C * 2 * C), 256, 0, st>>>(
            f->params + f->po.Rre[l], f->params + f->po.Rim[l], (int)M, (int)C,
            at<bf16>(f, f->off.Rb1) + l * M * C * 2 * C, at<bf16>(f, f->off.Rb2) + l * M * C * 2 * C);
    }
    to_bf16_kernel<<<blocks(C * P), 256, 0, st>>>(f->params + f->po.P1, at<bf16>(f, f->off.P1b), C * P);
    to_bf16_kernel<<<blocks(P * c.out_ch), 256, 0, st>>>(f->params + f->po.P2, at<bf16>(f, f->off.P2b), P * c.out_ch);
    FCK(cudaGetLastError());
    return HFS_OK;
}

int forward(hfs_fno_s *f, const float *x, int B)
{
    const hfs_fno_config &c = f->cfg;
    const int64_t L = c.grid, C = c.width, M = c.modes, P = c.proj, NL = c.layers;
    const int64_t rows = (int64_t)B * L, Bm = f->max_batch, rowsM = Bm * L;
    cudaStream_t st = f->stream;
    // the tensor-core GEMMs' bounded-wait status word; null keeps every GEMM on mma.sync
    unsigned *fst = f->gemm_engine == HFS_FNO_GEMM_TCGEN05 ? at<unsigned>(f, f->off.status) : nullptr;
    const auto &w = f->off;
    bf16 *X8 = at<bf16>(f, w.X8);
    to_bf16_pad_kernel<<<blocks(rows * kInPad), 256, 0, st>>>(x, rows, c.in_ch, X8, kInPad);
    float *Hf = at<float>(f, w.Hf);
    bf16 *Hb = at<bf16>(f, w.Hb);
    // lift: H0 = X P_in + b_in
    {
        GemmArgs g = gemm((int)rows, (int)C, kInPad, X8, kInPad, at<bf16>(f, w.Pinb), C);
        g.bias = f->params + f->po.bin;
        g.C = Hf;
        g.ldc = C;
        g.Cb = Hb;
        g.ldcb = C;
        FCK(run(g, false, false, st, fst));
    }
    for (int l = 0; l < NL; ++l) {
        const bf16 *Hinb = Hb + l * rowsM * C;
        bf16 *S = at<bf16>(f, w.S) + l * Bm * 2 * M * C;
        // S_b = F2 H_b   (2M x C per sample)
        {
            GemmArgs g = gemm((int)(2 * M), (int)C, (int)L, at<bf16>(f, w.F2), L, Hinb, C);
            g.sA = 0;
            g.sB = L * C;
            g.Cb = S;
            g.ldcb = C;
            g.sCb = 2 * M * C;
            g.batch = B;
            FCK(run(g, false, false, st, fst));
        }
        // Y_k = S_re,k R1_k + S_im,k R2_k   (B x 2C per mode)
        float *Yf = at<float>(f, w.Yf);
        bf16 *Yb = at<bf16>(f, w.Yb);
        for (int part = 0; part < 2; ++part) {
            GemmArgs g = gemm(B, (int)(2 * C), (int)C, S + part * M * C, 2 * M * C,
                              at<bf16>(f, part == 0 ? w.Rb1 : w.Rb2) + l * M * C * 2 * C, 2 * C);
            g.sA = C;
            g.sB = C * 2 * C;
            g.C = Yf;
            g.ldc = 2 * C;
            g.sC = Bm * 2 * C;
            g.beta = part;
            if (part == 1) {
                g.Cb = Yb;
                g.ldcb = 2 * C;
                g.sCb = Bm * 2 * C;
            }
            g.batch = (int)M;
            FCK(run(g, false, false, st, fst));
        }
        // U_b = Gre Yre_b + Gim Yim_b   (L x C per sample)
        float *U = at<float>(f, w.U);
        for (int part = 0; part < 2; ++part) {
            GemmArgs g = gemm((int)L, (int)C, (int)M, at<bf16>(f, part == 0 ? w.Gre : w.Gim), M, Yb + part * C,
                              Bm * 2 * C);
            g.sA = 0;
            g.sB = 2 * C;
            g.C = U;
            g.ldc = C;
            g.sC = L * C;
            g.beta = part;
            g.batch = B;
            FCK(run(g, false, false, st, fst));
        }
        // Z = H W + b + U; H_next = GELU(Z) (identity on the last layer)
        {
            GemmArgs g = gemm((int)rows, (int)C, (int)C, Hinb, C, at<bf16>(f, w.Wb) + l * C * C, C);
            g.bias = f->params + f->po.b[l];
            g.add = U;
            g.ldadd = C;
            g.pre = at<float>(f, w.pre) + l * rowsM * C;
            g.ldp = C;
            g.gelu = (l < NL - 1) ? 1 : 0;
            g.C = Hf + (l + 1) * rowsM * C;
            g.ldc = C;
            g.Cb = Hb + (l + 1) * rowsM * C;
            g.ldcb = C;
            FCK(run(g, false, false, st, fst));
        }
    }
    // projection: Q = GELU(H P1 + c1); O = Q P2 + c2
    {
        GemmArgs g = gemm((int)rows, (int)P, (int)C, Hb + NL * rowsM * C, C, at<bf16>(f, w.P1b), P);
        g.bias = f->params + f->po.c1;
        g.pre = at<float>(f, w.Qpre);
        g.ldp = P;
        g.gelu = 1;
        g.Cb = at<bf16>(f, w.Qb);
        g.ldcb = P;
        FCK(run(g, false, false, st, fst));
    }
    {
        GemmArgs g = gemm((int)rows, c.out_ch, (int)P, at<bf16>(f, w.Qb), P, at<bf16>(f, w.P2b), c.out_ch);
        g.bias = f->params + f->po.c2;
        g.C = at<float>(f, w.O);
        g.ldc = c.out_ch;
        FCK(run(g, false, false, st, fst));
    }
    return HFS_OK;
}

int backward(hfs_fno_s *f, const float *y, int B, float *grad)
{
    const hfs_fno_config &c = f->cfg;
    const int64_t L = c.grid, C = c.width, M = c.modes, P = c.proj, NL = c.layers, OC = c.out_ch;
    const int64_t rows = (int64_t)B * L, Bm = f->max_batch, rowsM = Bm * L;
    cudaStream_t st = f->stream;
    // the tensor-core GEMMs' bounded-wait status word; null keeps every GEMM on mma.sync
    unsigned *fst = f->gemm_engine == HFS_FNO_GEMM_TCGEN05 ? at<unsigned>(f, f->off.status) : nullptr;
    const auto &w = f->off;
    FCK(cudaMemsetAsync(grad, 0, 4 * f->nparams, st));
    // loss and dO
    float *O = at<float>(f, w.O), *dO = at<float>(f, w.dO), *sums = at<float>(f, w.sums);
    bf16 *dOb = at<bf16>(f, w.dOb);
    loss_sums_kernel<<<B, 256, 0, st>>>(O, y, L * OC, sums);
    loss_grad_kernel<<<blocks(rows * OC), 256, 0, st>>>(O, y, sums, L * OC, B, dO, dOb);
    loss_value_kernel<<<1, 256, 0, st>>>(sums, B, at<float>(f, w.loss));
    FCK(cudaGetLastError());
    // projection
    bf16 *Qb = at<bf16>(f, w.Qb), *dQb = at<bf16>(f, w.dQb);
    float *dQ = at<float>(f, w.dQ);
    FCK(weight_grad((int)P, (int)OC, rows, Qb, P, dOb, OC, grad + f->po.P2, st));
    colsum_kernel<<<colsum_blocks(rows), (unsigned)OC, 0, st>>>(dO, rows, (int)OC, grad + f->po.c2);
    {
        GemmArgs g = gemm((int)rows, (int)P, (int)OC, dOb, OC, at<bf16>(f, w.P2b), OC);  // dQ = dO P2^T
        g.C = dQ;
        g.ldc = P;
        FCK(run(g, false, true, st, fst));
    }
    gelu_bwd_kernel<<<blocks(rows * P), 256, 0, st>>>(dQ, at<float>(f, w.Qpre), 1, dQ, dQb, rows * P);
    bf16 *Hb = at<bf16>(f, w.Hb);
    FCK(weight_grad((int)C, (int)P, rows, Hb + NL * rowsM * C, C, dQb, P, grad + f->po.P1, st));
    colsum_kernel<<<colsum_blocks(rows), (unsigned)P, 0, st>>>(dQ, rows, (int)P, grad + f->po.c1);
    float *dH = at<float>(f, w.dH), *dZ = at<float>(f, w.dZ);
    bf16 *dZb = at<bf16>(f, w.dZb);
    {
        GemmArgs g = gemm((int)rows, (int)C, (int)P, dQb, P, at<bf16>(f, w.P1b), P);  // dH = dQpre P1^T
        g.C = dH;
        g.ldc = C;
        FCK(run(g, false, true, st, fst));
    }
    bf16 *dYb = at<bf16>(f, w.dYb), *dSb = at<bf16>(f, w.dSb);
    float *dR1 = at<float>(f, w.dR1), *dR2 = at<float>(f, w.dR2);
    for (int l = NL - 1; l >= 0; --l) {
        gelu_bwd_kernel<<<blocks(rows * C), 256, 0, st>>>(dH, at<float>(f, w.pre) + l * rowsM * C,
                                                          (l < NL - 1) ? 1 : 0, dZ, dZb, rows * C);
        const bf16 *Hinb = Hb + l * rowsM * C;
        FCK(weight_grad((int)C, (int)C, rows, Hinb, C, dZb, C, grad + f->po.W[l], st));
        colsum_kernel<<<colsum_blocks(rows), (unsigned)C, 0, st>>>(dZ, rows, (int)C, grad + f->po.b[l]);
        {
            GemmArgs g = gemm((int)rows, (int)C, (int)C, dZb, C, at<bf16>(f, w.Wb) + l * C * C, C);  // dZ W^T
            g.C = dH;
            g.ldc = C;
            FCK(run(g, false, true, st, fst));
        }
        // dYre_b = Gre^T dU_b, dYim_b = Gim^T dU_b  -> dY[k][b][part C + o]
        for (int part = 0; part < 2; ++part) {
            GemmArgs g = gemm((int)M, (int)C, (int)L, at<bf16>(f, part == 0 ? w.Gre : w.Gim), M, dZb, C);
            g.sA = 0;
            g.sB = L * C;
            g.Cb = dYb + part * C;
            g.ldcb = Bm * 2 * C;
            g.sCb = 2 * C;
            g.batch = B;
            FCK(run(g, true, false, st, fst));
        }
        const bf16 *S = at<bf16>(f, w.S) + l * Bm * 2 * M * C;
        for (int part = 0; part < 2; ++part) {
            // dR{1,2}_k = S_{re,im},k^T dY_k   (C x 2C per mode, K = B)
            GemmArgs g = gemm((int)C, (int)(2 * C), B, S + part * M * C, 2 * M * C, dYb, 2 * C);
            g.sA = C;
            g.sB = Bm * 2 * C;
            g.C = part == 0 ? dR1 : dR2;
            g.ldc = 2 * C;
            g.sC = C * 2 * C;
            g.batch = (int)M;
            FCK(run(g, true, false, st, fst));
            // dS_{re,im},k = dY_k R{1,2}_k^T   -> dS[b][part M + k][c]
            GemmArgs h = gemm(B, (int)C, (int)(2 * C), dYb, 2 * C,
                              at<bf16>(f, part == 0 ? w.Rb1 : w.Rb2) + l * M * C * 2 * C, 2 * C);
            h.sA = Bm * 2 * C;
            h.sB = C * 2 * C;
            h.Cb = dSb + part * M * C;
            h.ldcb = 2 * M * C;
            h.sCb = C;
            h.batch = (int)M;
            FCK(run(h, false, true, st, fst));
        }
        mixing_grad_kernel<<<blocks(M * C * C), 256, 0, st>>>(dR1, dR2, (int)M, (int)C, grad + f->po.Rre[l],
                                                                grad + f->po.Rim[l]);
        // dH_in += F2^T dS_b
        {
            GemmArgs g = gemm((int)L, (int)C, (int)(2 * M), at<bf16>(f, w.F2), L, dSb, C);
            g.sA = 0;
            g.sB = 2 * M * C;
            g.C = dH;
            g.ldc = C;
            g.sC = L * C;
            g.beta = 1;
            g.batch = B;
            FCK(run(g, true, false, st, fst));
        }
    }
    // lift
    gelu_bwd_kernel<<<blocks(rows * C), 256, 0, st>>>(dH, nullptr, 0, nullptr, dZb, rows * C);
    // dP_in over the padded input rows into scratch, then keep the first in_ch rows
    FCK(cudaMemsetAsync(at<float>(f, w.dR1), 0, 4 * kInPad * C, st));
    FCK(weight_grad(kInPad, (int)C, rows, at<bf16>(f, w.X8), kInPad, dZb, C, at<float>(f, w.dR1), st));
    colsum_kernel<<<colsum_blocks(rows), (unsigned)C, 0, st>>>(dH, rows, (int)C, grad + f->po.bin);
    FCK(cudaMemcpyAsync(grad + f->po.Pin, at<float>(f, w.dR1), 4 * c.in_ch * C, cudaMemcpyDeviceToDevice, st));
    FCK(cudaGetLastError());
    return HFS_OK;
}

}  // namespace

extern "C" {

int hfs_fno_create(hfs_fno_t *out, const hfs_fno_config *cfg, int32_t max_batch, int32_t train)
{
    if (!out || !cfg || max_batch < 1) return HFS_ERR_INVALID_ARG;
    *out = nullptr;
    const hfs_fno_config &c = *cfg;
    if (c.grid < 16 || c.width < 8 || c.modes < 1 || 2 * c.modes > c.grid || c.layers < 1 || c.in_ch < 1 ||
        c.in_ch > kInPad || c.proj < 1 || c.out_ch < 1 || c.proj > 1024 || c.width > 1024 || c.out_ch > 1024)
        return HFS_ERR_INVALID_ARG;
    hfs_fno_s *f = new (std::nothrow) hfs_fno_s();
    if (!f) return HFS_ERR_INVALID_ARG;
    f->cfg = c;
    f->max_batch = max_batch;
    f->train = train ? 1 : 0;
    f->po = param_offsets(c);
    f->nparams = f->po.total;
    layout(f);
    *out = f;
    return HFS_OK;
}

void hfs_fno_destroy(hfs_fno_t f) { delete f; }

int hfs_fno_set_stream(hfs_fno_t f, void *stream)
{
    if (!f) return HFS_ERR_INVALID_ARG;
    f->stream = (cudaStream_t)stream;
    return HFS_OK;
}

int hfs_fno_param_count(hfs_fno_t f, int64_t *count)
{
    if (!f || !count) return HFS_ERR_INVALID_ARG;
    *count = f->nparams;
    return HFS_OK;
}

int hfs_fno_workspace_size(hfs_fno_t f, size_t *bytes)
{
    if (!f || !bytes) return HFS_ERR_INVALID_ARG;
    *bytes = f->off.total;
    return HFS_OK;
}

int hfs_fno_bind(hfs_fno_t f, float *params, void *work, size_t work_bytes)
{
    if (!f || !params || !work) return HFS_ERR_INVALID_ARG;
    if (((uintptr_t)params & 255) || ((uintptr_t)work & 255)) return HFS_ERR_ALIGNMENT;
    if (work_bytes < f->off.total) return HFS_ERR_WORKSPACE;
    f->params = params;
    f->work = (unsigned char *)work;
    f->work_bytes = work_bytes;
    const hfs_fno_config &c = f->cfg;
    (void)cudaGetLastError();
    dft_consts_kernel<<<blocks((int64_t)c.grid * c.modes), 256, 0, f->stream>>>(
        c.grid, c.modes, at<bf16>(f, f->off.F2), at<bf16>(f, f->off.Gre), at<bf16>(f, f->off.Gim));
    FCK(cudaGetLastError());
    if (f->train) {
        FCK(cudaMemsetAsync(at<float>(f, f->off.m), 0, 4 * f->nparams, f->stream));
        FCK(cudaMemsetAsync(at<float>(f, f->off.v), 0, 4 * f->nparams, f->stream));
    }
    f->step = 0;
    FCK(cudaMemsetAsync(at<unsigned>(f, f->off.status), 0, sizeof(unsigned), f->stream));
    return refresh_weights(f);
}

int hfs_fno_set_gemm_engine(hfs_fno_t f, int engine)
{
    if (!f || (engine != HFS_FNO_GEMM_MMA_SYNC && engine != HFS_FNO_GEMM_TCGEN05)) return HFS_ERR_INVALID_ARG;
    f->gemm_engine = engine;
    return HFS_OK;
}

int hfs_fno_sync_status(hfs_fno_t f)
{
    if (!f || !f->work) return HFS_ERR_NOT_READY;
    unsigned word = 0;
    unsigned *dev = at<unsigned>(f, f->off.status);
    FCK(cudaMemcpyAsync(&word, dev, sizeof(unsigned), cudaMemcpyDeviceToHost, f->stream));
    FCK(cudaStreamSynchronize(f->stream));
    if (word) FCK(cudaMemsetAsync(dev, 0, sizeof(unsigned), f->stream));
    return word ? HFS_ERR_DEVICE_TIMEOUT : HFS_OK;
}

int hfs_fno_init_params(hfs_fno_t f, uint64_t seed)
{
    if (!f || !f->params) return HFS_ERR_NOT_READY;
    const hfs_fno_config &c = f->cfg;
    const int64_t C = c.width;
    cudaStream_t st = f->stream;
    (void)cudaGetLastError();
    auto uni = [&](int64_t off, int64_t n, float scale, uint64_t s) {
        init_uniform_kernel<<<blocks(n), 256, 0, st>>>(f->params + off, n, scale, seed * 1000003ull + s);
    };
    FCK(cudaMemsetAsync(f->params, 0, 4 * f->nparams, st));
    uni(f->po.Pin, (int64_t)c.in_ch * C, 1.0f / sqrtf((float)c.in_ch), 1);
    for (int l = 0; l < c.layers; ++l) {
        uni(f->po.Rre[l], (int64_t)c.modes * C * C, 1.0f / (float)C, 10 + 4 * l);
        uni(f->po.Rim[l], (int64_t)c.modes * C * C, 1.0f / (float)C, 11 + 4 * l);
        uni(f->po.W[l], C * C, 1.0f / sqrtf((float)C), 12 + 4 * l);
    }
    uni(f->po.P1, C * c.proj, 1.0f / sqrtf((float)C), 2);
    uni(f->po.P2, (int64_t)c.proj * c.out_ch, 1.0f / sqrtf((float)c.proj), 3);
    FCK(cudaGetLastError());
    return refresh_weights(f);
}

int hfs_fno_forward(hfs_fno_t f, const float *x, float *y, int32_t batch)
{
    if (!f || !x || !y) return HFS_ERR_INVALID_ARG;
    if (!f->params || !f->work) return HFS_ERR_NOT_READY;
    if (batch < 1 || batch > f->max_batch) return HFS_ERR_INVALID_ARG;
    (void)cudaGetLastError();
    int s = forward(f, x, batch);
    if (s) return s;
    FCK(cudaMemcpyAsync(y, at<float>(f, f->off.O), 4 * (size_t)batch * f->cfg.grid * f->cfg.out_ch,
                        cudaMemcpyDeviceToDevice, f->stream));
    return HFS_OK;
}

int hfs_fno_loss_grad(hfs_fno_t f, const float *x, const float *y, int32_t batch, float *grad, float *loss_host)
{
    if (!f || !x || !y) return HFS_ERR_INVALID_ARG;
    if (!f->params || !f->work || !f->train) return HFS_ERR_NOT_READY;
    if (batch < 1 || batch > f->max_batch) return HFS_ERR_INVALID_ARG;
    (void)cudaGetLastError();
    int s = forward(f, x, batch);
    if (s) return s;
    float *g = grad ? grad : at<float>(f, f->off.grad);
    s = backward(f, y, batch, g);
    if (s) return s;
    if (loss_host) {
        FCK(cudaMemcpyAsync(loss_host, at<float>(f, f->off.loss), 4, cudaMemcpyDeviceToHost, f->stream));
        FCK(cudaStreamSynchronize(f->stream));
    }
    return HFS_OK;
}

int hfs_fno_train_step(hfs_fno_t f, const float *x, const float *y, int32_t batch, float lr, float *loss_host)
{
    int s = hfs_fno_loss_grad(f, x, y, batch, nullptr, nullptr);
    if (s) return s;
    f->step += 1;
    const float b1 = 0.9f, b2 = 0.999f;
    const float c1 = 1.0f - powf(b1, (float)f->step), c2 = 1.0f - powf(b2, (float)f->step);
    adam_kernel<<<blocks(f->nparams), 256, 0, f->stream>>>(f->params, at<float>(f, f->off.grad),
                                                            at<float>(f, f->off.m), at<float>(f, f->off.v),
                                                            f->nparams, lr, b1, b2, 1e-8f, c1, c2);
    FCK(cudaGetLastError());
    s = refresh_weights(f);
    if (s) return s;
    if (loss_host) {
        FCK(cudaMemcpyAsync(loss_host, at<float>(f, f->off.loss), 4, cudaMemcpyDeviceToHost, f->stream));
        FCK(cudaStreamSynchronize(f->stream));
    }
    return HFS_OK;
}

}  // extern "C"
