/* caxsi_nn.h -- building blocks of the learned warm start.
 *
 * The paper has no learned component: these kernels serve an extension that
 * predicts the reconstruction's starting image f^0 from the first EM-type
 * iterate (Sec. VI, Algorithm 4) with a 2-D U-Net over the object's (i, j)
 * plane, whose 128 channels are the q bins; the EM-type iterations then continue
 * from f^0.  Activations are FP32 in NHWC order ([n][H][W][C], channels
 * fastest; the object f = [X][J][Q] is one such image); the convolutions are
 * GEMMs on tensor cores with bf16 operands and FP32 accumulation (the tcgen05
 * kernel of the table paths).  bf16 buffers are passed as uint16_t (IEEE
 * bfloat16 bits).  All pointers are device pointers owned by the caller; every
 * call is asynchronous on `stream` (a cudaStream_t, NULL = default stream) and
 * runs on the current device.  Reductions run in a fixed order (deterministic).
 * Errors: CAXSI_ERR_INVALID for null pointers, non-positive sizes or a layout
 * condition stated below; CAXSI_ERR_CUDA for a failed launch.
 */
#ifndef CAXSI_NN_H
#define CAXSI_NN_H

#include <stdint.h>

#include "caxsi.h"

#ifdef __cplusplus
extern "C" {
#endif

/* col[p][(ky*3 + kx)*C + c] = x[n][h+ky-1][w+kx-1][c] (0 outside the image) for
 * pixel p = (n, h, w): the 3x3 "same" convolution as a GEMM operand, bf16.
 * col: [n*H*W][9*C].  C must be a multiple of 8. */
caxsi_status caxsi_nn_im2col3x3(const float *x, int n, int H, int W, int C, uint16_t *col, void *stream);

/* The adjoint of im2col: dx[n][h][w][c] = sum over (ky, kx) of
 * dcol[(n, h-ky+1, w-kx+1)][(ky*3 + kx)*C + c] (gather, no atomics). */
caxsi_status caxsi_nn_col2im3x3(const float *dcol, int n, int H, int W, int C, float *dx, void *stream);

/* C[M][N] = A[M][K] * B[N][K]^T, A and B bf16 row-major (K contiguous), C FP32
 * row-major.  K*2 bytes and N*4 bytes must be multiples of 16 bytes, pointers
 * 16-byte aligned.  err_dev: one device int set to 1 if a copy wait of the
 * kernel timed out (then C is incomplete). */
caxsi_status caxsi_nn_gemm_bf16(int M, int N, int K, const uint16_t *A, const uint16_t *B, float *C,
                                int *err_dev, void *stream);

/* y[i] = bf16(x[i]) (round to nearest even). */
caxsi_status caxsi_nn_to_bf16(const float *x, uint16_t *y, int64_t n, void *stream);

/* y[c][r] = bf16(x[r][c]) for x [rows][cols]; x is FP32 if x_is_f32, else bf16. */
caxsi_status caxsi_nn_transpose_bf16(const void *x, int x_is_f32, int rows, int cols, uint16_t *y, void *stream);

/* y[p][c] += bias[c] (bias may be NULL), then max(y, 0) if relu. */
caxsi_status caxsi_nn_bias_act(float *y, const float *bias, int64_t P, int C, int relu, void *stream);

/* dy[i] = y[i] > 0 ? dy[i] : 0 (the ReLU backward, y the ReLU output). */
caxsi_status caxsi_nn_relu_bwd(float *dy, const float *y, int64_t n, void *stream);

/* db[c] = sum over p of dy[p][c]. */
caxsi_status caxsi_nn_bias_grad(const float *dy, int64_t P, int C, float *db, void *stream);

/* 2x2 average pooling x [n][H][W][C] -> y [n][H/2][W/2][C] (H, W even), and its
 * adjoint dx = dy / 4 on each 2x2 block. */
caxsi_status caxsi_nn_pool2(const float *x, int n, int H, int W, int C, float *y, void *stream);
caxsi_status caxsi_nn_pool2_bwd(const float *dy, int n, int H, int W, int C, float *dx, void *stream);

/* Nearest 2x upsampling x [n][h][w][C] -> y [n][2h][2w][C], and its adjoint
 * (dx = the sum over each 2x2 block of dy). */
caxsi_status caxsi_nn_up2(const float *x, int n, int h, int w, int C, float *y, void *stream);
caxsi_status caxsi_nn_up2_bwd(const float *dy, int n, int h, int w, int C, float *dx, void *stream);

/* dst[p][dst_off + c] = src[p][src_off + c] for c < Cs (channel concatenation and
 * its split); src_ld, dst_ld: channels per pixel of each buffer. */
caxsi_status caxsi_nn_copy_channels(const float *src, int64_t P, int Cs, int src_off, int src_ld, float *dst,
                                    int dst_off, int dst_ld, void *stream);

/* y[i] = max(a * x[i], lo) (scaling in and out of the network's units; lo = -inf
 * for none). */
caxsi_status caxsi_nn_scale_clamp(const float *x, float a, float lo, float *y, int64_t n, void *stream);

/* Adam step (t >= 1, bias-corrected): m = b1 m + (1-b1) g; v = b2 v + (1-b2) g^2;
 * w -= lr (m / (1-b1^t)) / (sqrt(v / (1-b2^t)) + eps). */
caxsi_status caxsi_nn_adam(float *w, const float *g, float *m, float *v, int64_t n, float lr, float b1, float b2,
                           float eps, int t, void *stream);

/* y[i] += a * x[i] (gradients meeting at a skip connection). */
caxsi_status caxsi_nn_axpy(float a, const float *x, float *y, int64_t n, void *stream);

/* Mean squared error: loss_dev[0] = sum_i (y_i - t_i)^2 / n accumulated in FP64
 * (fixed-order partial sums kept in loss_dev[1 .. CAXSI_NN_MSE_PARTS]),
 * grad_i = 2 (y_i - t_i) / n.  loss_dev holds 1 + CAXSI_NN_MSE_PARTS doubles. */
#define CAXSI_NN_MSE_PARTS 512
caxsi_status caxsi_nn_mse(const float *y, const float *t, int64_t n, float *grad, double *loss_dev, void *stream);

/* out[i] ~ Poisson(scale * mean[i]) as an integer-valued float (0 where the mean
 * is not positive): training counts drawn on the device.  Uniforms come from the
 * counter-based generator Philox4x32-10 with key `seed` and counter (i, block),
 * so each element's draw depends only on (seed, i), not on the launch; means
 * below 10 are drawn by inversion of the cumulative distribution, larger ones
 * by Hormann's transformed rejection with squeeze (1993).  scale >= 0. */
caxsi_status caxsi_nn_poisson(const float *mean, float scale, int64_t n, uint64_t seed, float *out, void *stream);

#ifdef __cplusplus
}
#endif

#endif
