/*
 * fno.h -- C ABI of the Fourier-neural-operator kernels in libwave: the
 * learned preconditioner that maps an RTM gradient to a velocity update.
 *
 * The paper uses Fourier neural operators (Li et al. 2020) as learned
 * surrogates (arxiv 2304.05592, section "Fourier neural operator surrogates")
 * and trains them with reverse-mode AD; here the same architecture is trained
 * on (gradient, true velocity perturbation) pairs, with every forward and
 * backward step in these kernels.  One Fourier layer on v[B][C][Nz][Nx] is
 *   v <- act(W v + b + S(R * T(v))),
 * T the truncated DFT  X[kz,kx] = sum_{z,x} v[z,x] exp(-i psi),
 *   psi = 2 pi (kz z/Nz + kx x/Nx), kz rows {0..mz-1, Nz-mz..Nz-1} (in that
 *   order, KZ = 2 mz of them), kx in {0..mx-1};
 * R * X the per-mode complex channel mix Y[o,k] = sum_i X[i,k] R[i,o,k];
 * S the truncated real inverse y = (1/(Nz Nx)) sum_k w_kx Re(Y[k] exp(+i psi)),
 *   w_0 = 1, w_kx = 2 (kx > 0).
 * T and S are evaluated as two small dense transforms each: along x (the
 * contiguous axis) against a table of [Nx][mx] complex factors, along z
 * against the table E[z][kz] = exp(+i phi), phi = 2 pi kz z / Nz.  The same two
 * kernels, with other x tables, give the adjoints used by the backward pass:
 *   table  fwd = (cos th, -sin th)                 x part of T
 *          inv = (w cos th, w sin th) / (Nz Nx)     x part of S (fno_combine)
 *          bwd = (w cos th, -w sin th) / (Nz Nx)    x part of S' (fno_dft_x)
 *          adj = (cos th, sin th)                   x part of T' (fno_combine)
 *   with th = 2 pi kx x / Nx.
 *
 * Layouts (C order, x fastest):
 *   activations        [B][C][Nz][Nx], float (or bf16 where stated)
 *   x-transformed      [rows][mx][2]     (re, im), rows = B C Nz
 *   spectra            [B C][KZ][mx][2]
 *   z-inverted         [B C][Nz][mx][2]
 *   spectral weights R [Ci][Co][KZ][mx][2]
 *   pointwise weights  M [Co][Ci] (or [Ci][Co] with m_trans = 1), bias [Co]
 *   x tables           [Nx][mx][2], z table [Nz][KZ][2]
 * Limits: 1 <= mx <= 16, 1 <= mz, 2 mz <= Nz, mx <= Nx / 2, channel counts
 * 1..64.  All pointers are device pointers owned by the caller; nothing is
 * allocated.  Work is queued on `stream` (a cudaStream_t, NULL = legacy
 * default stream) and the calls return without synchronising.  Return value:
 * WAVE_OK, WAVE_ERR_ARG for a null pointer or a size outside the limits
 * (nothing launched), WAVE_ERR_CUDA if a launch failed.
 */
#ifndef FNO_H
#define FNO_H

#include <stddef.h>

#include "wave.h"

#ifdef __cplusplus
extern "C" {
#endif

/* Activation applied by fno_combine. */
typedef enum { FNO_ACT_NONE = 0, FNO_ACT_GELU = 1 } fno_act_t;

/* The four x tables ([Nx][mx][2] each) and the z table ([Nz][2 mz][2]) above,
 * computed in double precision on the device and rounded to float. */
wave_status_t fno_tables(int Nz, int Nx, int mz, int mx, float* tx_fwd, float* tx_inv, float* tx_bwd,
                         float* tx_adj, float* tz, void* stream);

/* out[r][kx] = sum_x in[r][x] * (table[x][kx].re + i table[x][kx].im) for
 * rows r < rows; in is float, or bf16 when in_bf16 != 0. */
wave_status_t fno_dft_x(long long rows, int Nx, int mx, const void* in, int in_bf16, const float* table,
                        float* out, void* stream);

/* Along z, per batch b < nb: out[b][kz][kx] = sum_z in[b][z][kx] conj(E[z][kz])
 * (the forward direction; in is [nb][Nz][mx][2], out [nb][2mz][mx][2]). */
wave_status_t fno_dft_z(int nb, int Nz, int mz, int mx, const float* in, const float* tz, float* out,
                        void* stream);

/* Along z, inverse direction: out[b][z][kx] = sum_kz in[b][kz][kx] E[z][kz]
 * (in [nb][2mz][mx][2], out [nb][Nz][mx][2]). */
wave_status_t fno_idft_z(int nb, int Nz, int mz, int mx, const float* in, const float* tz, float* out,
                         void* stream);

/* Per-mode channel mix Y[b][o][m] = sum_i X[b][i][m] R[i][o][m] over
 * nmode = 2 mz mx complex modes. */
wave_status_t fno_mix(int B, int Ci, int Co, int nmode, const float* X, const float* R, float* Y,
                      void* stream);

/* fno_mix followed by fno_idft_z in one pass, the mixed spectrum Y kept on chip:
 *   out[b][o][z][kx] = sum_a Y[b][o][a][kx] E[z][a],
 *   Y[b][o][a][kx]   = sum_i X[b][i][a][kx] R[i][o][a][kx]
 * with a over the 2 mz kept z modes (X [B][Ci][2mz][mx][2], R as in fno_mix,
 * out [B][Co][Nz][mx][2]).  Both sums run in the order of the separate calls. */
wave_status_t fno_mix_idft_z(int B, int Ci, int Co, int Nz, int mz, int mx, const float* X, const float* R,
                             const float* tz, float* out, void* stream);

/* Its backward: dX[b][i][m] = sum_o dY[b][o][m] conj(R[i][o][m]) and
 * dR[i][o][m] = sum_b conj(X[b][i][m]) dY[b][o][m] (dR overwritten; the sum
 * over b runs in a fixed order).  Either output may be NULL. */
wave_status_t fno_mix_backward(int B, int Ci, int Co, int nmode, const float* X, const float* R, const float* dY,
                               float* dX, float* dR, void* stream);

/* Pointwise channel mix with an optional spectral term and activation:
 *   pre[b][o][z][x] = sum_i M[o][i] in[b][i][z][x] + bias[o]
 *                     + sum_kx (T[b][o][z][kx].re table[x][kx].re - T[b][o][z][kx].im table[x][kx].im)
 *   out = act(pre).
 * bias, T (then table is unused) and pre (stored only when non-NULL) may be
 * NULL; in is float or bf16 (in_bf16), out float or bf16 (out_bf16). */
wave_status_t fno_combine(int B, int Ci, int Co, int Nz, int Nx, int mx, const void* in, int in_bf16,
                          const float* M, int m_trans, const float* bias, const float* T, const float* table,
                          int act, float* pre, void* out, int out_bf16, void* stream);

/* The projection head Q of the FNO (two pointwise layers, GELU between them)
 * in one pass, for inference:
 *   out[b][0][z][x] = q2 + sum_h Q2[h] GELU(q1[h] + sum_i Q1[h][i] in[b][i][z][x])
 * with Q1 [H][Ci], q1 [H] (may be NULL), Q2 [1][H], q2 [1] (may be NULL); in is
 * float or bf16 (in_bf16), out float [B][1][Nz][Nx].  The H hidden channels
 * never leave the chip (fno_combine followed by a second fno_combine writes and
 * reads them).  With bf16 input, Ci = 32 and H = 32 or 64 it runs on the
 * tensor cores (the hidden layer as in fno_combine, the second layer in the
 * epilogue in float), otherwise on the CUDA cores. */
wave_status_t fno_project(int B, int Ci, int H, int Nz, int Nx, const void* in, int in_bf16, const float* Q1,
                          const float* q1, const float* Q2, const float* q2, float* out, void* stream);

/* With the tensor cores allowed (fno_set_tensor_cores(1), the default), the BF16
 * inference path runs on them (tcgen05.mma, BF16 operands, FP32 accumulation in
 * tensor memory): fno_combine when in and out are bf16, pre is NULL, m_trans = 0,
 * Ci = 32 and Co is 32 or 64; fno_project under the conditions stated there;
 * fno_dft_x when in is bf16.  The weights, the tables and the spectral
 * coefficients are rounded to BF16 on their way into shared memory, the bias to
 * two BF16 parts (about 16 significant bits), and GELU there evaluates erf by
 * Abramowitz and Stegun's formula 7.1.26 (|error| <= 1.5e-7).
 * fno_set_tensor_cores(0) keeps the CUDA-core kernels everywhere.
 * fno_tensor_core_status synchronises the device, returns WAVE_ERR_TIMEOUT if a
 * tensor-core launch since the last call gave up waiting for its MMAs (its
 * results are then invalid), and clears the flag. */
wave_status_t fno_set_tensor_cores(int on);
wave_status_t fno_tensor_core_status(void);

/* Weight gradients of a pointwise layer: dM[o][i] = sum_{b,p} dU[b][o][p] in[b][i][p],
 * dbias[o] = sum_{b,p} dU[b][o][p] (npix = Nz Nx pixels per sample), both
 * overwritten.  `work` holds fno_wgrad_work_floats(B, Ci, Co, npix) floats;
 * partial sums are combined in a fixed order, so results are repeatable on a
 * given GPU (the pixel chunks are sized to the GPU's resident blocks, so the
 * grouping of the sums, and with it the last bits, can differ between GPU
 * models).  dbias may be NULL. */
size_t fno_wgrad_work_floats(int B, int Ci, int Co, long long npix);
wave_status_t fno_wgrad(int B, int Ci, int Co, long long npix, const float* dU, const float* in, float* dM,
                        float* dbias, float* work, void* stream);

/* dpre = dout * GELU'(pre) (GELU(x) = x Phi(x)), n elements. */
wave_status_t fno_gelu_backward(long long n, const float* dout, const float* pre, float* dpre, void* stream);

/* Mean squared error (1/n) sum (pred - target)^2 into *loss (device double)
 * and its gradient 2 (pred - target) / n into dpred (may be NULL); `work`
 * holds 1024 doubles. */
wave_status_t fno_mse(long long n, const float* pred, const float* target, float* dpred, double* loss,
                      double* work, void* stream);

/* One Adam step (Kingma and Ba 2015) on n parameters, step number t >= 1:
 * m = b1 m + (1-b1) g, v = b2 v + (1-b2) g^2,
 * p -= lr (m / (1-b1^t)) / (sqrt(v / (1-b2^t)) + eps).  The hyper-parameters
 * are doubles so that 1-b1, 1-b2 and the bias corrections are formed before
 * rounding to float; the update itself runs in float. */
wave_status_t fno_adam(long long n, float* p, const float* g, float* m, float* v, double lr, double b1, double b2,
                       double eps, int t, void* stream);

#ifdef __cplusplus
}
#endif

#endif /* FNO_H */
