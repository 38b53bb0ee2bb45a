// Building blocks of the learned warm start (include/caxsi_nn.h): a U-Net over
// the object's (i, j) plane with the q bins as channels.  Convolutions are
// im2col gathers to bf16 plus the tcgen05 GEMM of the table paths (bf16
// operands, FP32 accumulation); everything else is elementwise, pooling,
// upsampling or a fixed-order reduction.  NHWC FP32 activations throughout.
#include <cuda_bf16.h>
#include <math.h>

#include "caxsi_nn.h"
#include "internal.cuh"
#include "table.cuh"

namespace {

constexpr int NT = 256;

inline unsigned nblocks(int64_t n) { return (unsigned)((n + NT - 1) / NT); }

__global__ void k_im2col3x3(const float *__restrict__ x, int n, int H, int W, int C,
                            __nv_bfloat16 *__restrict__ col) {
    // one thread per (pixel, tap, 8 channels)
    const int C8 = C >> 3;
    const int64_t total = (int64_t)n * H * W * 9 * C8;
    const int64_t idx = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (idx >= total) return;
    const int c8 = (int)(idx % C8);
    const int64_t r = idx / C8;
    const int tap = (int)(r % 9);
    const int64_t p = r / 9;
    const int w = (int)(p % W);
    const int h = (int)((p / W) % H);
    const int b = (int)(p / ((int64_t)W * H));
    const int hh = h + tap / 3 - 1, ww = w + tap % 3 - 1;
    float4 v0 = make_float4(0.f, 0.f, 0.f, 0.f), v1 = v0;
    if (hh >= 0 && hh < H && ww >= 0 && ww < W) {
        const float4 *src = reinterpret_cast<const float4 *>(x + (((int64_t)b * H + hh) * W + ww) * C + c8 * 8);
        v0 = src[0];
        v1 = src[1];
    }
    __nv_bfloat162 q[4] = {__floats2bfloat162_rn(v0.x, v0.y), __floats2bfloat162_rn(v0.z, v0.w),
                           __floats2bfloat162_rn(v1.x, v1.y), __floats2bfloat162_rn(v1.z, v1.w)};
    *reinterpret_cast<uint4 *>(col + p * 9 * C + tap * C + c8 * 8) = *reinterpret_cast<uint4 *>(q);
}

__global__ void k_col2im3x3(const float *__restrict__ dcol, int n, int H, int W, int C, float *__restrict__ dx) {
    const int64_t total = (int64_t)n * H * W * C;
    const int64_t idx = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (idx >= total) return;
    const int c = (int)(idx % C);
    const int64_t p = idx / C;
    const int w = (int)(p % W);
    const int h = (int)((p / W) % H);
    const int b = (int)(p / ((int64_t)W * H));
    float acc = 0.f;
#pragma unroll
    for (int tap = 0; tap < 9; ++tap) {
        const int ho = h - tap / 3 + 1, wo = w - tap % 3 + 1;   // the output pixel that read x[h][w] at this tap
        if (ho < 0 || ho >= H || wo < 0 || wo >= W) continue;
        acc += dcol[(((int64_t)b * H + ho) * W + wo) * 9 * C + tap * C + c];
    }
    dx[idx] = acc;
}

__global__ void k_to_bf16(const float *__restrict__ x, __nv_bfloat16 *__restrict__ y, int64_t n) {
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i < n) y[i] = __float2bfloat16_rn(x[i]);
}

template <typename T>
__global__ void k_transpose_bf16(const T *__restrict__ x, int rows, int cols, __nv_bfloat16 *__restrict__ y) {
    __shared__ float tile[32][33];
    const int c0 = blockIdx.x * 32, r0 = blockIdx.y * 32;
    for (int k = threadIdx.y; k < 32; k += blockDim.y) {
        const int r = r0 + k, c = c0 + threadIdx.x;
        tile[k][threadIdx.x] = (r < rows && c < cols) ? (float)x[(int64_t)r * cols + c] : 0.f;
    }
    __syncthreads();
    for (int k = threadIdx.y; k < 32; k += blockDim.y) {
        const int c = c0 + k, r = r0 + threadIdx.x;
        if (c < cols && r < rows) y[(int64_t)c * rows + r] = __float2bfloat16_rn(tile[threadIdx.x][k]);
    }
}

__global__ void k_bias_act(float *__restrict__ y, const float *__restrict__ bias, int64_t P, int C, int relu) {
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= P * C) return;
    float v = y[i] + (bias ? bias[i % C] : 0.f);
    if (relu) v = fmaxf(v, 0.f);
    y[i] = v;
}

__global__ void k_relu_bwd(float *__restrict__ dy, const float *__restrict__ y, int64_t n) {
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i < n && !(y[i] > 0.f)) dy[i] = 0.f;
}

// one block per channel; fixed strided partition then a fixed tree
__global__ void k_bias_grad(const float *__restrict__ dy, int64_t P, int C, float *__restrict__ db) {
    __shared__ float sh[NT];
    const int c = blockIdx.x;
    float acc = 0.f;
    for (int64_t p = threadIdx.x; p < P; p += NT) acc += dy[p * C + c];
    sh[threadIdx.x] = acc;
    __syncthreads();
    for (int s = NT / 2; s > 0; s >>= 1) {
        if (threadIdx.x < s) sh[threadIdx.x] += sh[threadIdx.x + s];
        __syncthreads();
    }
    if (threadIdx.x == 0) db[c] = sh[0];
}

__global__ void k_pool2(const float *__restrict__ x, int n, int H, int W, int C, float *__restrict__ y) {
    const int h2 = H / 2, w2 = W / 2;
    const int64_t total = (int64_t)n * h2 * w2 * C;
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= total) return;
    const int c = (int)(i % C);
    const int64_t p = i / C;
    const int w = (int)(p % w2), h = (int)((p / w2) % h2), b = (int)(p / ((int64_t)w2 * h2));
    const float *s = x + (((int64_t)b * H + 2 * h) * W + 2 * w) * C + c;
    y[i] = 0.25f * (s[0] + s[C] + s[(int64_t)W * C] + s[(int64_t)W * C + C]);
}

__global__ void k_pool2_bwd(const float *__restrict__ dy, int n, int H, int W, int C, float *__restrict__ dx) {
    const int64_t total = (int64_t)n * H * W * C;
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= total) return;
    const int c = (int)(i % C);
    const int64_t p = i / C;
    const int w = (int)(p % W), h = (int)((p / W) % H), b = (int)(p / ((int64_t)W * H));
    dx[i] = 0.25f * dy[(((int64_t)b * (H / 2) + h / 2) * (W / 2) + w / 2) * C + c];
}

__global__ void k_up2(const float *__restrict__ x, int n, int h, int w, int C, float *__restrict__ y) {
    const int H = 2 * h, W = 2 * w;
    const int64_t total = (int64_t)n * H * W * C;
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= total) return;
    const int c = (int)(i % C);
    const int64_t p = i / C;
    const int ww = (int)(p % W), hh = (int)((p / W) % H), b = (int)(p / ((int64_t)W * H));
    y[i] = x[(((int64_t)b * h + hh / 2) * w + ww / 2) * C + c];
}

__global__ void k_up2_bwd(const float *__restrict__ dy, int n, int h, int w, int C, float *__restrict__ dx) {
    const int64_t total = (int64_t)n * h * w * C;
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= total) return;
    const int c = (int)(i % C);
    const int64_t p = i / C;
    const int ww = (int)(p % w), hh = (int)((p / w) % h), b = (int)(p / ((int64_t)w * h));
    const int W = 2 * w;
    const float *s = dy + (((int64_t)b * 2 * h + 2 * hh) * W + 2 * ww) * C + c;
    dx[i] = (s[0] + s[C]) + (s[(int64_t)W * C] + s[(int64_t)W * C + C]);
}

__global__ void k_copy_channels(const float *__restrict__ src, int64_t P, int Cs, int so, int sld,
                                float *__restrict__ dst, int dof, int dld) {
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= P * Cs) return;
    const int c = (int)(i % Cs);
    const int64_t p = i / Cs;
    dst[p * dld + dof + c] = src[p * sld + so + c];
}

__global__ void k_scale_clamp(const float *__restrict__ x, float a, float lo, float *__restrict__ y, int64_t n) {
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i < n) y[i] = fmaxf(a * x[i], lo);
}

__global__ void k_adam(float *__restrict__ w, const float *__restrict__ g, float *__restrict__ m, float *__restrict__ v,
                       int64_t n, float lr, float b1, float b2, float eps, float c1, float c2) {
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    const float gi = g[i];
    const float mi = b1 * m[i] + (1.f - b1) * gi;
    const float vi = b2 * v[i] + (1.f - b2) * gi * gi;
    m[i] = mi;
    v[i] = vi;
    w[i] -= lr * (mi / c1) / (sqrtf(vi / c2) + eps);
}

// per-block FP64 partials in a fixed order, then one block sums the partials
__global__ void k_mse(const float *__restrict__ y, const float *__restrict__ t, int64_t n, float *__restrict__ grad,
                      double *__restrict__ part) {
    __shared__ double sh[NT];
    double acc = 0.0;
    const float s = 2.f / (float)n;
    for (int64_t i = (int64_t)blockIdx.x * NT + threadIdx.x; i < n; i += (int64_t)gridDim.x * NT) {
        const float d = y[i] - t[i];
        grad[i] = s * d;
        acc += (double)d * (double)d;
    }
    sh[threadIdx.x] = acc;
    __syncthreads();
    for (int k = NT / 2; k > 0; k >>= 1) {
        if (threadIdx.x < k) sh[threadIdx.x] += sh[threadIdx.x + k];
        __syncthreads();
    }
    if (threadIdx.x == 0) part[blockIdx.x] = sh[0];
}

__global__ void k_mse_final(const double *__restrict__ part, int nb, int64_t n, double *__restrict__ out) {
    if (threadIdx.x == 0 && blockIdx.x == 0) {
        double s = 0.0;
        for (int b = 0; b < nb; ++b) s += part[b];
        out[0] = s / (double)n;
    }
}

int device_sms() {
    static int cache[CAXSI_MAX_DEVICES] = {0};
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= CAXSI_MAX_DEVICES) return 0;
    if (!cache[dev]) cudaDeviceGetAttribute(&cache[dev], cudaDevAttrMultiProcessorCount, dev);
    return cache[dev];
}

caxsi_status launched() { return cudaGetLastError() == cudaSuccess ? CAXSI_OK : CAXSI_ERR_CUDA; }

// ---- Poisson draws from a counter-based generator ---------------------------------
// Philox4x32-10 (Salmon, Moraes, Dror and Shaw, "Parallel random numbers: as easy
// as 1, 2, 3", SC 2011): ten rounds of two 32 x 32 -> 64-bit multiplications
// whose halves are xored with the other counter words and the key, the key
// advanced by the Weyl constants between rounds.  Counter (element, block of
// four uniforms, 0, 0), key = the seed: every element's stream is independent of
// the launch shape.
struct Philox {
    uint32_t k0, k1, i0, i1, blk;
    uint32_t buf[4];
    int used;
    __device__ Philox(uint64_t seed, uint64_t idx)
        : k0((uint32_t)seed), k1((uint32_t)(seed >> 32)), i0((uint32_t)idx), i1((uint32_t)(idx >> 32)), blk(0),
          used(4) {}
    __device__ void refill() {
        uint32_t c0 = i0, c1 = i1, c2 = blk++, c3 = 0u, a = k0, b = k1;
#pragma unroll
        for (int r = 0; r < 10; ++r) {
            if (r > 0) {
                a += 0x9E3779B9u;
                b += 0xBB67AE85u;
            }
            const uint32_t lo0 = 0xD2511F53u * c0, hi0 = __umulhi(0xD2511F53u, c0);
            const uint32_t lo1 = 0xCD9E8D57u * c2, hi1 = __umulhi(0xCD9E8D57u, c2);
            const uint32_t n0 = hi1 ^ c1 ^ a, n2 = hi0 ^ c3 ^ b;
            c0 = n0;
            c1 = lo1;
            c2 = n2;
            c3 = lo0;
        }
        buf[0] = c0;
        buf[1] = c1;
        buf[2] = c2;
        buf[3] = c3;
        used = 0;
    }
    // uniform in the open interval (0, 1) with 24 random bits
    __device__ float uniform() {
        if (used == 4) refill();
        return ((float)(buf[used++] >> 8) + 0.5f) * 5.9604645e-8f;
    }
};

// k ~ Poisson(lam).  lam < 10: inversion by sequential search over the
// cumulative distribution (one uniform).  lam >= 10: the transformed rejection
// method with squeeze of Hormann ("The transformed rejection method for
// generating Poisson random variables", Insurance: Mathematics and Economics 12,
// 1993), whose acceptance test is taken in FP64.  Both loops are bounded; the
// bounds are far beyond any draw with a probability above 1e-30.
__device__ float poisson_draw(Philox &rng, float lam) {
    if (!(lam > 0.f)) return 0.f;
    if (lam < 10.f) {
        const float u = rng.uniform();
        float p = expf(-lam), F = p;
        int k = 0;
        while (u > F && k < 128) {
            ++k;
            p *= lam / (float)k;
            F += p;
        }
        return (float)k;
    }
    const double L = (double)lam, sl = sqrt(L), logl = log(L);
    const double b = 0.931 + 2.53 * sl, a = -0.059 + 0.02483 * b;
    const double inv_alpha = 1.1239 + 1.1328 / (b - 3.4), vr = 0.9277 - 3.6224 / (b - 2.0);
    for (int it = 0; it < 256; ++it) {
        const double U = (double)rng.uniform() - 0.5, V = (double)rng.uniform();
        const double us = 0.5 - fabs(U);
        const double k = floor((2.0 * a / us + b) * U + L + 0.43);
        if (us >= 0.07 && V <= vr) return (float)k;
        if (k < 0.0 || (us < 0.013 && V > us)) continue;
        if (log(V) + log(inv_alpha) - log(a / (us * us) + b) <= -L + k * logl - lgamma(k + 1.0)) return (float)k;
    }
    return rintf(lam);
}

__global__ void k_poisson(const float *__restrict__ mean, float scale, int64_t n, uint64_t seed,
                          float *__restrict__ out) {
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
        Philox rng(seed, (uint64_t)i);
        out[i] = poisson_draw(rng, scale * mean[i]);
    }
}

constexpr int MSE_BLOCKS = CAXSI_NN_MSE_PARTS;

__global__ void k_axpy(float a, const float *__restrict__ x, float *__restrict__ y, int64_t n) {
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i < n) y[i] = fmaf(a, x[i], y[i]);
}

}  // namespace

extern "C" {

caxsi_status caxsi_nn_im2col3x3(const float *x, int n, int H, int W, int C, uint16_t *col, void *stream) {
    if (!x || !col || n < 1 || H < 1 || W < 1 || C < 8 || C % 8) return CAXSI_ERR_INVALID;
    const int64_t total = (int64_t)n * H * W * 9 * (C / 8);
    k_im2col3x3<<<nblocks(total), NT, 0, (cudaStream_t)stream>>>(x, n, H, W, C,
                                                                  reinterpret_cast<__nv_bfloat16 *>(col));
    return launched();
}

caxsi_status caxsi_nn_col2im3x3(const float *dcol, int n, int H, int W, int C, float *dx, void *stream) {
    if (!dcol || !dx || n < 1 || H < 1 || W < 1 || C < 1) return CAXSI_ERR_INVALID;
    k_col2im3x3<<<nblocks((int64_t)n * H * W * C), NT, 0, (cudaStream_t)stream>>>(dcol, n, H, W, C, dx);
    return launched();
}

caxsi_status caxsi_nn_gemm_bf16(int M, int N, int K, const uint16_t *A, const uint16_t *B, float *C, int *err_dev,
                                void *stream) {
    if (!A || !B || !C || !err_dev || M < 1 || N < 1 || K < 1) return CAXSI_ERR_INVALID;
    if ((K * 2) % 16 || (N * 4) % 16 || ((uintptr_t)A | (uintptr_t)B | (uintptr_t)C) & 15) return CAXSI_ERR_INVALID;
    const int sms = device_sms();
    if (sms < 1) return CAXSI_ERR_CUDA;
    const cudaError_t e = tc_gemm(1, N > 128 ? 256 : 128, M, N, K, A, nullptr, K, B, nullptr, K, C, N, err_dev, sms,
                                  (cudaStream_t)stream);
    return e == cudaSuccess ? CAXSI_OK : CAXSI_ERR_CUDA;
}

caxsi_status caxsi_nn_to_bf16(const float *x, uint16_t *y, int64_t n, void *stream) {
    if (!x || !y || n < 1) return CAXSI_ERR_INVALID;
    k_to_bf16<<<nblocks(n), NT, 0, (cudaStream_t)stream>>>(x, reinterpret_cast<__nv_bfloat16 *>(y), n);
    return launched();
}

caxsi_status caxsi_nn_transpose_bf16(const void *x, int x_is_f32, int rows, int cols, uint16_t *y, void *stream) {
    if (!x || !y || rows < 1 || cols < 1) return CAXSI_ERR_INVALID;
    const dim3 grid((unsigned)((cols + 31) / 32), (unsigned)((rows + 31) / 32)), block(32, 8);
    if (x_is_f32)
        k_transpose_bf16<float><<<grid, block, 0, (cudaStream_t)stream>>>(
            static_cast<const float *>(x), rows, cols, reinterpret_cast<__nv_bfloat16 *>(y));
    else
        k_transpose_bf16<__nv_bfloat16><<<grid, block, 0, (cudaStream_t)stream>>>(
            static_cast<const __nv_bfloat16 *>(x), rows, cols, reinterpret_cast<__nv_bfloat16 *>(y));
    return launched();
}

caxsi_status caxsi_nn_bias_act(float *y, const float *bias, int64_t P, int C, int relu, void *stream) {
    if (!y || P < 1 || C < 1) return CAXSI_ERR_INVALID;
    k_bias_act<<<nblocks(P * C), NT, 0, (cudaStream_t)stream>>>(y, bias, P, C, relu);
    return launched();
}

caxsi_status caxsi_nn_relu_bwd(float *dy, const float *y, int64_t n, void *stream) {
    if (!dy || !y || n < 1) return CAXSI_ERR_INVALID;
    k_relu_bwd<<<nblocks(n), NT, 0, (cudaStream_t)stream>>>(dy, y, n);
    return launched();
}

caxsi_status caxsi_nn_bias_grad(const float *dy, int64_t P, int C, float *db, void *stream) {
    if (!dy || !db || P < 1 || C < 1) return CAXSI_ERR_INVALID;
    k_bias_grad<<<(unsigned)C, NT, 0, (cudaStream_t)stream>>>(dy, P, C, db);
    return launched();
}

caxsi_status caxsi_nn_pool2(const float *x, int n, int H, int W, int C, float *y, void *stream) {
    if (!x || !y || n < 1 || H < 2 || W < 2 || H % 2 || W % 2 || C < 1) return CAXSI_ERR_INVALID;
    k_pool2<<<nblocks((int64_t)n * (H / 2) * (W / 2) * C), NT, 0, (cudaStream_t)stream>>>(x, n, H, W, C, y);
    return launched();
}

caxsi_status caxsi_nn_pool2_bwd(const float *dy, int n, int H, int W, int C, float *dx, void *stream) {
    if (!dy || !dx || n < 1 || H < 2 || W < 2 || H % 2 || W % 2 || C < 1) return CAXSI_ERR_INVALID;
    k_pool2_bwd<<<nblocks((int64_t)n * H * W * C), NT, 0, (cudaStream_t)stream>>>(dy, n, H, W, C, dx);
    return launched();
}

caxsi_status caxsi_nn_up2(const float *x, int n, int h, int w, int C, float *y, void *stream) {
    if (!x || !y || n < 1 || h < 1 || w < 1 || C < 1) return CAXSI_ERR_INVALID;
    k_up2<<<nblocks((int64_t)n * 4 * h * w * C), NT, 0, (cudaStream_t)stream>>>(x, n, h, w, C, y);
    return launched();
}

caxsi_status caxsi_nn_up2_bwd(const float *dy, int n, int h, int w, int C, float *dx, void *stream) {
    if (!dy || !dx || n < 1 || h < 1 || w < 1 || C < 1) return CAXSI_ERR_INVALID;
    k_up2_bwd<<<nblocks((int64_t)n * h * w * C), NT, 0, (cudaStream_t)stream>>>(dy, n, h, w, C, dx);
    return launched();
}

caxsi_status caxsi_nn_copy_channels(const float *src, int64_t P, int Cs, int src_off, int src_ld, float *dst,
                                    int dst_off, int dst_ld, void *stream) {
    if (!src || !dst || P < 1 || Cs < 1 || src_off < 0 || dst_off < 0 || src_off + Cs > src_ld ||
        dst_off + Cs > dst_ld)
        return CAXSI_ERR_INVALID;
    k_copy_channels<<<nblocks(P * Cs), NT, 0, (cudaStream_t)stream>>>(src, P, Cs, src_off, src_ld, dst, dst_off,
                                                                    dst_ld);
    return launched();
}

caxsi_status caxsi_nn_scale_clamp(const float *x, float a, float lo, float *y, int64_t n, void *stream) {
    if (!x || !y || n < 1 || !isfinite(a)) return CAXSI_ERR_INVALID;
    k_scale_clamp<<<nblocks(n), NT, 0, (cudaStream_t)stream>>>(x, a, lo, y, n);
    return launched();
}

caxsi_status caxsi_nn_adam(float *w, const float *g, float *m, float *v, int64_t n, float lr, float b1, float b2,
                           float eps, int t, void *stream) {
    if (!w || !g || !m || !v || n < 1 || t < 1 || !(lr > 0.f) || !(b1 >= 0.f && b1 < 1.f) ||
        !(b2 >= 0.f && b2 < 1.f) || !(eps > 0.f))
        return CAXSI_ERR_INVALID;
    const float c1 = 1.f - powf(b1, (float)t), c2 = 1.f - powf(b2, (float)t);
    k_adam<<<nblocks(n), NT, 0, (cudaStream_t)stream>>>(w, g, m, v, n, lr, b1, b2, eps, c1, c2);
    return launched();
}

caxsi_status caxsi_nn_axpy(float a, const float *x, float *y, int64_t n, void *stream) {
    if (!x || !y || n < 1 || !isfinite(a)) return CAXSI_ERR_INVALID;
    k_axpy<<<nblocks(n), NT, 0, (cudaStream_t)stream>>>(a, x, y, n);
    return launched();
}

caxsi_status caxsi_nn_poisson(const float *mean, float scale, int64_t n, uint64_t seed, float *out, void *stream) {
    if (!mean || !out || n < 1 || !isfinite(scale) || scale < 0.f) return CAXSI_ERR_INVALID;
    const int64_t nb = (n + NT - 1) / NT;
    k_poisson<<<(unsigned)(nb < 4096 ? nb : 4096), NT, 0, (cudaStream_t)stream>>>(mean, scale, n, seed, out);
    return launched();
}

caxsi_status caxsi_nn_mse(const float *y, const float *t, int64_t n, float *grad, double *loss_dev, void *stream) {
    if (!y || !t || !grad || !loss_dev || n < 1) return CAXSI_ERR_INVALID;
    k_mse<<<MSE_BLOCKS, NT, 0, (cudaStream_t)stream>>>(y, t, n, grad, loss_dev + 1);
    if (cudaGetLastError() != cudaSuccess) return CAXSI_ERR_CUDA;
    k_mse_final<<<1, 32, 0, (cudaStream_t)stream>>>(loss_dev + 1, MSE_BLOCKS, n, loss_dev);
    return launched();
}

}  // extern "C"
