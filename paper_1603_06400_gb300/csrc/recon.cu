// Elementwise parts of one EM-type iteration (Sec. V-VI, Algorithm 4,
// Appendices B-C): the likelihood ratio y / (A f + r) with the negative
// log-likelihood accumulated in FP64, and the closed-form update of Eq. 10
// with the Huber edge-preserving penalty on the 4 spatial neighbours.
#include <math.h>

#include "internal.cuh"

namespace {

constexpr int NLL_THREADS = 256;

// ratio_i = y_i / z_i with z = g + r (FP32); per-block FP64 partial sums of
// d_i = z_i - y_i ln z_i + ln y_i!.  y_i = 0 with z_i <= 0 contributes 0 and
// ratio 0; y_i > 0 with z_i <= 0 raises the plan's error word.
__global__ void __launch_bounds__(NLL_THREADS)
k_ratio_nll(const float *__restrict__ g, const float *__restrict__ y, const float *__restrict__ r,
            const int *__restrict__ sub, int subset, float *__restrict__ ratio, double *__restrict__ part,
            int *err, int64_t n) {
    __shared__ double sh[NLL_THREADS / 32];
    double local = 0.0;
    for (int64_t idx = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; idx < n;
         idx += (int64_t)gridDim.x * blockDim.x) {
        const float z = r ? g[idx] + r[idx] : g[idx];
        const float yy = y[idx];
        float rt = 0.f;
        if (sub && sub[idx] != subset) {
            // outside the subset: no ratio, no likelihood term
        } else if (z > 0.f) {
            rt = yy / z;
            const double zd = (double)z, yd = (double)yy;
            local += zd - (yd > 0.0 ? yd * log(zd) : 0.0) + lgamma(yd + 1.0);
        } else if (yy > 0.f) {
            *err = 1;
        }
        ratio[idx] = rt;
    }
    for (int o = 16; o > 0; o >>= 1) local += __shfl_down_sync(0xffffffffu, local, o);
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    if (lane == 0) sh[warp] = local;
    __syncthreads();
    if (threadIdx.x == 0) {
        double s = 0.0;
        for (int w = 0; w < NLL_THREADS / 32; ++w) s += sh[w];
        part[blockIdx.x] = s;
    }
}

// Fixed-order sum of the block partials (deterministic).
__global__ void k_sum_nll(const double *__restrict__ part, int nb, double *__restrict__ out) {
    if (blockIdx.x == 0 && threadIdx.x == 0) {
        double s = 0.0;
        for (int b = 0; b < nb; ++b) s += part[b];
        *out = s;
    }
}

// chi1 = beta (b3 + b4), chi2 = b1 + beta (-f (b3 + b4) + b5 + b6), chi3 = f b2,
// b3 = b4 = 2 sum_k omega(f_j - f_k), b5 = b6 = sum_k psi_dot(f_j - f_k) over the
// 4 spatial neighbours (symmetric neighbourhood, unit weights); the update is
// the positive root of chi1 x^2 + chi2 x - chi3 = 0 (the Lemma), written without
// cancellation for chi2 > 0.
__global__ void k_update(DevGeo g, const float *__restrict__ f, const float *__restrict__ b1,
                         const float *__restrict__ b2, float beta, float delta,
                         float *__restrict__ fnew) {
    const int64_t n = (int64_t)g.R * g.Q;
    const int64_t idx = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (idx >= n) return;
    const int l = (int)(idx % g.Q);
    const int v = (int)(idx / g.Q);
    const int i = v / g.J, j = v - i * g.J;
    const float fh = f[idx];
    float b3 = 0.f, b5 = 0.f;
    if (beta != 0.f) {
        const int di[4] = {-1, 1, 0, 0};
        const int dj[4] = {0, 0, -1, 1};
#pragma unroll
        for (int q = 0; q < 4; ++q) {
            const int ii = i + di[q], jj = j + dj[q];
            if (ii < 0 || ii >= g.X || jj < 0 || jj >= g.J) continue;
            const float d = fh - f[((int64_t)ii * g.J + jj) * g.Q + l];
            const float ad = fabsf(d);
            b3 += 2.f * (ad <= delta ? 1.f : delta / ad);
            b5 += fminf(fmaxf(d, -delta), delta);
        }
    }
    const float chi1 = beta * (2.f * b3);
    const float chi2 = b1[idx] + beta * (-fh * (2.f * b3) + 2.f * b5);
    const float chi3 = fh * b2[idx];
    float x;
    if (chi1 > 0.f) {
        const float disc = sqrtf(fmaf(chi2, chi2, 4.f * chi1 * chi3));
        x = chi2 > 0.f ? (2.f * chi3) / (chi2 + disc) : (disc - chi2) / (2.f * chi1);
    } else if (chi2 > 0.f) {
        x = chi3 / chi2;
    } else {
        x = fh;
    }
    fnew[idx] = x;
}

}  // namespace

caxsi_status recon_ratio(caxsi_plan *p, const float *y, const float *r, const int *sub, int subset,
                         cudaStream_t s) {
    const int64_t n = (int64_t)p->dg.M * p->dg.N;
    {
        CAXSI_PROF(p, "ratio_nll", s);
        k_ratio_nll<<<p->nll_blocks, NLL_THREADS, 0, s>>>(p->gtmp, y, r, sub, subset, p->ratio,
                                                          p->nll_part, p->err_flag, n);
    }
    CAXSI_LAUNCH_CHECK(p);
    {
        CAXSI_PROF(p, "sum_nll", s);
        k_sum_nll<<<1, 32, 0, s>>>(p->nll_part, p->nll_blocks, p->nll_dev);
    }
    CAXSI_LAUNCH_CHECK(p);
    return CAXSI_OK;
}

caxsi_status recon_update(caxsi_plan *p, const float *f_old, float beta, float delta,
                          const float *b1, cudaStream_t s) {
    const int64_t n = (int64_t)p->dg.R * p->dg.Q;
    {
        CAXSI_PROF(p, "em_update", s);
        k_update<<<(unsigned)ceil_div64(n, 256), 256, 0, s>>>(p->dg, f_old, b1, p->b2, beta, delta, p->fnew);
    }
    CAXSI_LAUNCH_CHECK(p);
    return CAXSI_OK;
}

caxsi_status recon_nll_fetch(caxsi_plan *p, double *out, cudaStream_t s) {
    int err[2] = {0, 0};
    CAXSI_CUDA_TRY(cudaMemcpyAsync(out, p->nll_dev, sizeof(double), cudaMemcpyDeviceToHost, s));
    CAXSI_CUDA_TRY(cudaMemcpyAsync(err, p->err_flag, 2 * sizeof(int), cudaMemcpyDeviceToHost, s));
    CAXSI_CUDA_TRY(cudaStreamSynchronize(s));
    if (err[0] || err[1]) {
        CAXSI_CUDA_TRY(cudaMemsetAsync(p->err_flag, 0, 2 * sizeof(int), s));
        CAXSI_CUDA_TRY(cudaStreamSynchronize(s));
        return err[1] ? CAXSI_ERR_INTERNAL : CAXSI_ERR_NONPOS_MEAN;
    }
    return CAXSI_OK;
}
