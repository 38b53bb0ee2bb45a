// Elementwise parts of one EM-type iteration (Sec. V-VI, Algorithm 4,
// Appendices B-C): the likelihood ratio y / (A f + r) with the negative
// log-likelihood accumulated in FP64, and the closed-form update of Eq. 10
// with the Huber edge-preserving penalty on the 4 spatial neighbours.
#include <float.h>
#include <math.h>

#include "internal.cuh"

namespace {

// ratio_i = y_i / z_i with z = g + r (FP32); per-block FP64 partial sums of
// d_i = z_i - y_i ln z_i + ln y_i!, and their sum in block order by the block
// that finishes last (a completion counter, reset by that block), so the total
// is deterministic.  y_i = 0 with z_i <= 0 contributes 0 and ratio 0; y_i > 0
// with z_i <= 0 raises the plan's error word.  Small blocks spread the FP64
// log / lgamma work over every SM.
__global__ void __launch_bounds__(NLL_THREADS)
k_ratio_nll(const float *__restrict__ g, const float *__restrict__ y, const float *__restrict__ r,
            const int *__restrict__ sub, int subset, float *__restrict__ ratio, double *__restrict__ part,
            unsigned *done, double *__restrict__ total, int *err, int64_t n) {
    __shared__ double sh[NLL_THREADS];
    __shared__ bool last;
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
        __threadfence();
        last = atomicAdd(done, 1u) == gridDim.x - 1;   // every partial is written
    }
    __syncthreads();
    if (!last) return;   // block-uniform
    // the last block: thread t sums partials t, t + NLL_THREADS, ... in order (read
    // through L2), then a fixed tree over the threads
    __threadfence();
    double t = 0.0;
    for (unsigned b = threadIdx.x; b < gridDim.x; b += NLL_THREADS) t += __ldcg(part + b);
    sh[threadIdx.x] = t;
    __syncthreads();
    for (int h = NLL_THREADS / 2; h > 0; h >>= 1) {
        if (threadIdx.x < h) sh[threadIdx.x] += sh[threadIdx.x + h];
        __syncthreads();
    }
    if (threadIdx.x == 0) {
        *total = sh[0];
        *done = 0u;
    }
}

// The ratio alone, for calls that do not ask for the likelihood: the same
// quotient as k_ratio_nll and the same error word, without the FP64 log and
// lgamma terms (slow on this part's FP64 units).
__global__ void k_ratio(const float *__restrict__ g, const float *__restrict__ y, const float *__restrict__ r,
                        const int *__restrict__ sub, int subset, float *__restrict__ ratio, int *err, int64_t n) {
    for (int64_t idx = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; idx < n;
         idx += (int64_t)gridDim.x * blockDim.x) {
        const float z = r ? g[idx] + r[idx] : g[idx];
        const float yy = y[idx];
        float rt = 0.f;
        if (sub && sub[idx] != subset) {
            // outside the subset: no ratio
        } else if (z > 0.f) {
            rt = yy / z;
        } else if (yy > 0.f) {
            *err = 1;
        }
        ratio[idx] = rt;
    }
}

// The ratio y / (g + r) over n elements of caller buffers (any number of
// detector images back to back), with the edge rules of k_ratio, and its
// reverse mode: d ratio / d g = -y / z^2 = -(y / z) / z where z > 0, 0 elsewhere
// (the ratio is 0 there whatever g is).
__global__ void k_ratio_ext(const float *__restrict__ g, const float *__restrict__ y, const float *__restrict__ r,
                            float *__restrict__ ratio, int *err, int64_t n) {
    for (int64_t idx = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; idx < n;
         idx += (int64_t)gridDim.x * blockDim.x) {
        const float z = r ? g[idx] + r[idx] : g[idx];
        const float yy = y[idx];
        float rt = 0.f;
        if (z > 0.f) rt = yy / z;
        else if (yy > 0.f) *err = 1;
        ratio[idx] = rt;
    }
}

__global__ void k_ratio_vjp(const float *__restrict__ g, const float *__restrict__ y, const float *__restrict__ r,
                            const float *__restrict__ gr, float *__restrict__ gg, int64_t n) {
    for (int64_t idx = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; idx < n;
         idx += (int64_t)gridDim.x * blockDim.x) {
        const float z = r ? g[idx] + r[idx] : g[idx];
        gg[idx] = z > 0.f ? -(gr[idx] * (y[idx] / z)) / z : 0.f;
    }
}

// chi1 = beta (b3 + b4), chi2 = b1 + beta (-f (b3 + b4) + b5 + b6), chi3 = f b2,
// b3 = b4 = 2 sum_k omega(f_j - f_k), b5 = b6 = sum_k psi_dot(f_j - f_k) over the
// 4 spatial neighbours (symmetric neighbourhood, unit weights); the update is
// the positive root of chi1 x^2 + chi2 x - chi3 = 0 (the Lemma), written without
// cancellation for chi2 > 0.  n = nobj * R * Q: objects of the same geometry
// back to back, each with its own neighbourhoods.
// omega(d) = psi_dot(d) / d of the Huber penalty, from |d| and delta: 1 within
// delta, delta / |d| beyond.  Beyond delta with delta normal, |d| is normal too
// and the hardware quotient (within 2 ulp) serves; a zero or subnormal delta
// keeps the IEEE quotient.  The IEEE form, evaluated for every neighbour as the
// select compiles it, divides by |d| = 0 wherever the image is flat, and that
// case runs its slow path: the update took twice as long on a flat image.
__device__ __forceinline__ float huber_omega(float ad, float delta) {
    if (ad <= delta) return 1.f;
    return delta >= FLT_MIN ? __fdividef(delta, ad) : delta / ad;
}

struct UpdTerms {
    float fh, b3, b5, chi1, chi2, chi3, x;
    int kind;   // 0: root with chi1 > 0, 1: chi3 / chi2, 2: value kept
};

__device__ __forceinline__ int64_t nb_index(const DevGeo &g, int64_t idx, int q, bool &ok) {
    const int l = (int)(idx % g.Q);
    const int64_t vv = idx / g.Q;
    const int v = (int)(vv % g.R);
    const int64_t base = (vv - v) * g.Q;   // the object's first element
    const int i = v / g.J, j = v - i * g.J;
    const int ii = i + (q == 0 ? -1 : q == 1 ? 1 : 0), jj = j + (q == 2 ? -1 : q == 3 ? 1 : 0);
    ok = ii >= 0 && ii < g.X && jj >= 0 && jj < g.J;
    return base + ((int64_t)ii * g.J + jj) * g.Q + l;
}

__device__ __forceinline__ UpdTerms upd_terms(const DevGeo &g, const float *__restrict__ f,
                                              const float *__restrict__ b1, const float *__restrict__ b2,
                                              float beta, float delta, int64_t idx) {
    UpdTerms u;
    u.fh = f[idx];
    u.b3 = 0.f;
    u.b5 = 0.f;
    if (beta != 0.f) {
#pragma unroll
        for (int q = 0; q < 4; ++q) {
            bool ok;
            const int64_t k = nb_index(g, idx, q, ok);
            if (!ok) continue;
            const float d = u.fh - f[k];
            const float ad = fabsf(d);
            u.b3 += 2.f * huber_omega(ad, delta);
            u.b5 += fminf(fmaxf(d, -delta), delta);
        }
    }
    u.chi1 = beta * (2.f * u.b3);
    u.chi2 = b1[idx] + beta * (-u.fh * (2.f * u.b3) + 2.f * u.b5);
    u.chi3 = u.fh * b2[idx];
    if (u.chi1 > 0.f) {
        const float disc = sqrtf(fmaf(u.chi2, u.chi2, 4.f * u.chi1 * u.chi3));
        u.x = u.chi2 > 0.f ? (2.f * u.chi3) / (u.chi2 + disc) : (disc - u.chi2) / (2.f * u.chi1);
        u.kind = 0;
    } else if (u.chi2 > 0.f) {
        u.x = u.chi3 / u.chi2;
        u.kind = 1;
    } else {
        u.x = u.fh;
        u.kind = 2;
    }
    return u;
}

// The update of one element from its value fh, its 4 neighbours nb (ok: inside
// the object), b1 and b2 (the same arithmetic as upd_terms).
__device__ __forceinline__ float update_value(float fh, const float (&nb)[4], const bool (&ok)[4], float b1v,
                                              float b2v, float beta, float delta) {
    float b3 = 0.f, b5 = 0.f;
    if (beta != 0.f) {
#pragma unroll
        for (int q = 0; q < 4; ++q) {
            if (!ok[q]) continue;
            const float d = fh - nb[q];
            const float ad = fabsf(d);
            b3 += 2.f * huber_omega(ad, delta);
            b5 += fminf(fmaxf(d, -delta), delta);
        }
    }
    const float chi1 = beta * (2.f * b3);
    const float chi2 = b1v + beta * (-fh * (2.f * b3) + 2.f * b5);
    const float chi3 = fh * b2v;
    if (chi1 > 0.f) {
        const float disc = sqrtf(fmaf(chi2, chi2, 4.f * chi1 * chi3));
        return chi2 > 0.f ? (2.f * chi3) / (chi2 + disc) : (disc - chi2) / (2.f * chi1);
    }
    if (chi2 > 0.f) return chi3 / chi2;
    return fh;
}

// One block per voxel (blockIdx.x over nobj * R voxels), the q channels across
// the threads: the neighbours are +-Q and +-J*Q away, no index divisions per element.
__global__ void k_update(DevGeo g, const float *__restrict__ f, const float *__restrict__ b1,
                         const float *__restrict__ b2, float beta, float delta,
                         float *__restrict__ fnew) {
    const int vv = blockIdx.x;
    const int v = vv % g.R;
    const int i = v / g.J, j = v - i * g.J;
    const int64_t JQ = (int64_t)g.J * g.Q;
    const bool ok[4] = {i > 0, i + 1 < g.X, j > 0, j + 1 < g.J};
    for (int l = threadIdx.x; l < g.Q; l += blockDim.x) {
        const int64_t idx = (int64_t)vv * g.Q + l;
        float nb[4] = {0.f, 0.f, 0.f, 0.f};
        if (beta != 0.f) {
            nb[0] = ok[0] ? f[idx - JQ] : 0.f;
            nb[1] = ok[1] ? f[idx + JQ] : 0.f;
            nb[2] = ok[2] ? f[idx - g.Q] : 0.f;
            nb[3] = ok[3] ? f[idx + g.Q] : 0.f;
        }
        fnew[idx] = update_value(f[idx], nb, ok, b1[idx], b2[idx], beta, delta);
    }
}

// The same with four q channels per thread and 16-byte accesses (Q % 4 == 0 and
// 16-byte aligned arrays): block (Q/4, voxels per block); thread (x, y) takes
// channels 4x .. 4x + 3 of voxel blockIdx.x * blockDim.y + y, nv voxels in all.
__global__ void k_update4(DevGeo g, const float4 *__restrict__ f, const float4 *__restrict__ b1,
                          const float4 *__restrict__ b2, float beta, float delta, float4 *__restrict__ fnew,
                          int nv) {
    const int QV = (int)blockDim.x;
    const int vv = (int)(blockIdx.x * blockDim.y + threadIdx.y);
    if (vv >= nv) return;
    const int64_t e = (int64_t)vv * QV + threadIdx.x;
    const int v = vv % g.R;
    const int i = v / g.J, j = v - i * g.J;
    const int64_t JQ = (int64_t)g.J * QV;
    const bool ok[4] = {i > 0, i + 1 < g.X, j > 0, j + 1 < g.J};
    const float4 z4 = make_float4(0.f, 0.f, 0.f, 0.f);
    float4 n4[4] = {z4, z4, z4, z4};
    if (beta != 0.f) {
        n4[0] = ok[0] ? f[e - JQ] : z4;
        n4[1] = ok[1] ? f[e + JQ] : z4;
        n4[2] = ok[2] ? f[e - QV] : z4;
        n4[3] = ok[3] ? f[e + QV] : z4;
    }
    const float4 fh = f[e], c1 = b1[e], c2 = b2[e];
    float4 out;
    {
        const float nb[4] = {n4[0].x, n4[1].x, n4[2].x, n4[3].x};
        out.x = update_value(fh.x, nb, ok, c1.x, c2.x, beta, delta);
    }
    {
        const float nb[4] = {n4[0].y, n4[1].y, n4[2].y, n4[3].y};
        out.y = update_value(fh.y, nb, ok, c1.y, c2.y, beta, delta);
    }
    {
        const float nb[4] = {n4[0].z, n4[1].z, n4[2].z, n4[3].z};
        out.z = update_value(fh.z, nb, ok, c1.z, c2.z, beta, delta);
    }
    {
        const float nb[4] = {n4[0].w, n4[1].w, n4[2].w, n4[3].w};
        out.w = update_value(fh.w, nb, ok, c1.w, c2.w, beta, delta);
    }
    fnew[e] = out;
}

// Launch the update over n elements (n / Q voxels, objects back to back).
cudaError_t launch_update(const DevGeo &g, const float *f, const float *b1, const float *b2, float beta,
                          float delta, float *out, int64_t n, cudaStream_t s) {
    const int64_t nv = n / g.Q;
    const bool v4 = g.Q % 4 == 0 && g.Q / 4 <= 1024 && nv < INT32_MAX &&
                    ((reinterpret_cast<uintptr_t>(f) | reinterpret_cast<uintptr_t>(b1) |
                      reinterpret_cast<uintptr_t>(b2) | reinterpret_cast<uintptr_t>(out)) & 15) == 0;
    if (v4) {
        const int qv = g.Q / 4, vpb = qv >= 256 ? 1 : 256 / qv;
        k_update4<<<(unsigned)ceil_div64(nv, vpb), dim3((unsigned)qv, (unsigned)vpb), 0, s>>>(
            g, reinterpret_cast<const float4 *>(f), reinterpret_cast<const float4 *>(b1),
            reinterpret_cast<const float4 *>(b2), beta, delta, reinterpret_cast<float4 *>(out), (int)nv);
    } else {
        const unsigned thr = (unsigned)(g.Q >= 128 ? 128 : (g.Q + 31) / 32 * 32);
        k_update<<<(unsigned)(n / g.Q), thr, 0, s>>>(g, f, b1, b2, beta, delta, out);
    }
    return cudaGetLastError();
}


// Reverse mode of the update.  Implicit differentiation of the root:
// (2 chi1 x + chi2) dx = dchi3 - x dchi2 - x^2 dchi1.  Pass 1, per element j: the
// gradients of chi1..3, hence of b2_j, of f_j through chi2 and chi3, and of b3_j
// and b5_j (kept in gb3, gb5) with their derivatives with respect to f_j itself
// (omega'(d) = -delta sign(d) / d^2 beyond delta, psi_dot'(d) = 1 within it).
// Element idx of arrays that start at an object's first element (objects of g's
// geometry back to back).
__device__ __forceinline__ void update_vjp1_elem(const DevGeo &g, const float *__restrict__ f,
                                                 const float *__restrict__ b1, const float *__restrict__ b2,
                                                 float beta, float delta, const float *__restrict__ gx,
                                                 float *__restrict__ gf, float *__restrict__ gb2,
                                                 float *__restrict__ gb3, float *__restrict__ gb5, int64_t idx) {
    const UpdTerms u = upd_terms(g, f, b1, b2, beta, delta, idx);
    const float gxi = gx[idx];
    if (u.kind == 2) {
        gf[idx] = gxi;
        gb2[idx] = 0.f;
        gb3[idx] = 0.f;
        gb5[idx] = 0.f;
        return;
    }
    const float D = 2.f * u.chi1 * u.x + u.chi2;
    if (!(D > 0.f)) {   // a double root at x = 0 (f = 0 and chi2 = 0): no derivative, taken as 0
        gf[idx] = 0.f;
        gb2[idx] = 0.f;
        gb3[idx] = 0.f;
        gb5[idx] = 0.f;
        return;
    }
    const float g3 = gxi / D, g2 = -gxi * u.x / D, g1 = -gxi * u.x * u.x / D;
    const float gB3 = 2.f * beta * g1 - 2.f * beta * u.fh * g2;
    const float gB5 = 2.f * beta * g2;
    float own = g3 * b2[idx] + g2 * (-2.f * beta * u.b3);
    if (beta != 0.f) {
#pragma unroll
        for (int q = 0; q < 4; ++q) {
            bool ok;
            const int64_t k = nb_index(g, idx, q, ok);
            if (!ok) continue;
            const float d = u.fh - f[k];
            const float ad = fabsf(d);
            const float domega = ad <= delta ? 0.f : -delta * copysignf(1.f, d) / (d * d);
            own += gB3 * 2.f * domega + gB5 * (ad < delta ? 1.f : 0.f);
        }
    }
    gf[idx] = own;
    gb2[idx] = g3 * u.fh;
    gb3[idx] = gB3;
    gb5[idx] = gB5;
}

// Pass 2: each neighbour k of j adds -(gb3_k 2 omega'(f_k - f_j) + gb5_k psi_dot'(f_k - f_j)).
__device__ __forceinline__ void update_vjp2_elem(const DevGeo &g, const float *__restrict__ f, float delta,
                                                 const float *__restrict__ gb3, const float *__restrict__ gb5,
                                                 float *__restrict__ gf, int64_t idx) {
    const float fj = f[idx];
    float acc = gf[idx];
#pragma unroll
    for (int q = 0; q < 4; ++q) {
        bool ok;
        const int64_t k = nb_index(g, idx, q, ok);
        if (!ok) continue;
        const float d = f[k] - fj;
        const float ad = fabsf(d);
        const float domega = ad <= delta ? 0.f : -delta * copysignf(1.f, d) / (d * d);
        acc -= gb3[k] * 2.f * domega + gb5[k] * (ad < delta ? 1.f : 0.f);
    }
    gf[idx] = acc;
}

__global__ void k_update_vjp1(DevGeo g, const float *__restrict__ f, const float *__restrict__ b1,
                              const float *__restrict__ b2, float beta, float delta,
                              const float *__restrict__ gx, float *__restrict__ gf, float *__restrict__ gb2,
                              float *__restrict__ gb3, float *__restrict__ gb5, int64_t n) {
    const int64_t idx = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (idx >= n) return;
    update_vjp1_elem(g, f, b1, b2, beta, delta, gx, gf, gb2, gb3, gb5, idx);
}

__global__ void k_update_vjp2(DevGeo g, const float *__restrict__ f, float delta, const float *__restrict__ gb3,
                              const float *__restrict__ gb5, float *__restrict__ gf, int64_t n) {
    const int64_t idx = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (idx >= n) return;
    update_vjp2_elem(g, f, delta, gb3, gb5, gf, idx);
}

// ---- objects of different geometries packed back to back ------------------------
// Object b's elements are [foff[b], foff[b+1]) with the geometry geos[b]; its
// voxels are [vox0[b], vox0[b+1]) in the packed voxel order.

__device__ __forceinline__ int multi_object(const int64_t *__restrict__ first, int n, int64_t it) {
    int lo = 0, hi = n - 1;
    while (lo < hi) {
        const int mid = (lo + hi + 1) >> 1;
        if (first[mid] <= it) lo = mid;
        else hi = mid - 1;
    }
    return lo;
}

// One block per packed voxel, the q channels across the threads (as k_update).
__global__ void k_update_multi(const DevGeo *__restrict__ geos, const int64_t *__restrict__ vox0,
                               const int64_t *__restrict__ foff, int nobj, const float *__restrict__ f,
                               const float *__restrict__ b1, const float *__restrict__ b2, float beta, float delta,
                               float *__restrict__ fnew) {
    const int b = multi_object(vox0, nobj, blockIdx.x);
    const DevGeo g = geos[b];
    const int v = (int)(blockIdx.x - vox0[b]);
    const int i = v / g.J, j = v - i * g.J;
    const int64_t JQ = (int64_t)g.J * g.Q;
    const bool ok[4] = {i > 0, i + 1 < g.X, j > 0, j + 1 < g.J};
    const int64_t o = foff[b];
    for (int l = threadIdx.x; l < g.Q; l += blockDim.x) {
        const int64_t idx = o + (int64_t)v * g.Q + l;
        float nb[4] = {0.f, 0.f, 0.f, 0.f};
        if (beta != 0.f) {
            nb[0] = ok[0] ? f[idx - JQ] : 0.f;
            nb[1] = ok[1] ? f[idx + JQ] : 0.f;
            nb[2] = ok[2] ? f[idx - g.Q] : 0.f;
            nb[3] = ok[3] ? f[idx + g.Q] : 0.f;
        }
        fnew[idx] = update_value(f[idx], nb, ok, b1[idx], b2[idx], beta, delta);
    }
}

__global__ void k_update_vjp1_multi(const DevGeo *__restrict__ geos, const int64_t *__restrict__ foff, int nobj,
                                    const float *__restrict__ f, const float *__restrict__ b1,
                                    const float *__restrict__ b2, float beta, float delta,
                                    const float *__restrict__ gx, float *__restrict__ gf, float *__restrict__ gb2,
                                    float *__restrict__ gb3, float *__restrict__ gb5, int64_t n) {
    const int64_t idx = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (idx >= n) return;
    const int b = multi_object(foff, nobj, idx);
    const int64_t o = foff[b];
    update_vjp1_elem(geos[b], f + o, b1 + o, b2 + o, beta, delta, gx + o, gf + o, gb2 + o, gb3 + o, gb5 + o,
                     idx - o);
}

__global__ void k_update_vjp2_multi(const DevGeo *__restrict__ geos, const int64_t *__restrict__ foff, int nobj,
                                    const float *__restrict__ f, float delta, const float *__restrict__ gb3,
                                    const float *__restrict__ gb5, float *__restrict__ gf, int64_t n) {
    const int64_t idx = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (idx >= n) return;
    const int b = multi_object(foff, nobj, idx);
    const int64_t o = foff[b];
    update_vjp2_elem(geos[b], f + o, delta, gb3 + o, gb5 + o, gf + o, idx - o);
}

}  // namespace

caxsi_status recon_ratio(caxsi_plan *p, const float *y, const float *r, const int *sub, int subset, bool nll,
                         cudaStream_t s) {
    const int64_t n = (int64_t)p->dg.M * p->dg.N;
    if (!nll) {
        {
            CAXSI_PROF(p, "ratio", s);
            const int64_t nb = ceil_div64(n, 256);
            k_ratio<<<(unsigned)(nb < 4 * p->num_sms ? nb : 4 * p->num_sms), 256, 0, s>>>(
                p->gtmp, y, r, sub, subset, p->ratio, p->err_flag, n);
        }
        CAXSI_LAUNCH_CHECK(p);
        return CAXSI_OK;
    }
    {
        CAXSI_PROF(p, "ratio_nll", s);
        k_ratio_nll<<<p->nll_blocks, NLL_THREADS, 0, s>>>(p->gtmp, y, r, sub, subset, p->ratio, p->nll_part,
                                                          reinterpret_cast<unsigned *>(p->err_flag + 2),
                                                          p->nll_dev, p->err_flag, n);
    }
    CAXSI_LAUNCH_CHECK(p);
    return CAXSI_OK;
}

caxsi_status recon_update(caxsi_plan *p, const float *f_old, float beta, float delta,
                          const float *b1, cudaStream_t s) {
    const int64_t n = (int64_t)p->dg.R * p->dg.Q;
    {
        CAXSI_PROF(p, "em_update", s);
        CAXSI_CUDA_TRY(launch_update(p->dg, f_old, b1, p->b2, beta, delta, p->fnew, n, s));
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

caxsi_status recon_update_ext(caxsi_plan *p, const float *f, const float *b1, const float *b2, float beta,
                              float delta, float *out, int64_t n, cudaStream_t s) {
    {
        CAXSI_PROF(p, "em_update", s);
        CAXSI_CUDA_TRY(launch_update(p->dg, f, b1, b2, beta, delta, out, n, s));
    }
    CAXSI_LAUNCH_CHECK(p);
    return CAXSI_OK;
}

caxsi_status recon_update_vjp(caxsi_plan *p, const float *f, const float *b1, const float *b2, float beta,
                              float delta, const float *gx, float *gf, float *gb2, int64_t n, cudaStream_t s) {
    if (n > p->vjp_cap) {
        cudaFree(p->vjp_scratch);
        p->vjp_scratch = nullptr;
        p->vjp_cap = 0;
        CAXSI_CUDA_TRY(cudaMalloc(&p->vjp_scratch, 2 * (size_t)n * sizeof(float)));
        p->vjp_cap = n;
    }
    float *gb3 = p->vjp_scratch, *gb5 = p->vjp_scratch + n;
    const unsigned nb = (unsigned)ceil_div64(n, 256);
    {
        CAXSI_PROF(p, "em_update_vjp1", s);
        k_update_vjp1<<<nb, 256, 0, s>>>(p->dg, f, b1, b2, beta, delta, gx, gf, gb2, gb3, gb5, n);
    }
    CAXSI_LAUNCH_CHECK(p);
    {
        CAXSI_PROF(p, "em_update_vjp2", s);
        k_update_vjp2<<<nb, 256, 0, s>>>(p->dg, f, delta, gb3, gb5, gf, n);
    }
    CAXSI_LAUNCH_CHECK(p);
    return CAXSI_OK;
}

caxsi_status recon_ratio_ext(caxsi_plan *p, const float *g, const float *y, const float *r, float *ratio, int64_t n,
                             cudaStream_t s) {
    const int64_t nb = ceil_div64(n, 256);
    {
        CAXSI_PROF(p, "ratio", s);
        k_ratio_ext<<<(unsigned)(nb < 4 * p->num_sms ? nb : 4 * p->num_sms), 256, 0, s>>>(g, y, r, ratio,
                                                                                        p->err_flag, n);
    }
    CAXSI_LAUNCH_CHECK(p);
    return CAXSI_OK;
}

caxsi_status recon_ratio_vjp(caxsi_plan *p, const float *g, const float *y, const float *r, const float *gr,
                             float *gg, int64_t n, cudaStream_t s) {
    const int64_t nb = ceil_div64(n, 256);
    {
        CAXSI_PROF(p, "ratio_vjp", s);
        k_ratio_vjp<<<(unsigned)(nb < 4 * p->num_sms ? nb : 4 * p->num_sms), 256, 0, s>>>(g, y, r, gr, gg, n);
    }
    CAXSI_LAUNCH_CHECK(p);
    return CAXSI_OK;
}

caxsi_status multi_update(const DevGeo *geos, const int64_t *vox0, const int64_t *foff, int nobj, int64_t n_vox,
                          int qmax, const float *f, const float *b1, const float *b2, float beta, float delta,
                          float *out, cudaStream_t s) {
    const unsigned thr = (unsigned)(qmax >= 128 ? 128 : (qmax + 31) / 32 * 32);
    k_update_multi<<<(unsigned)n_vox, thr, 0, s>>>(geos, vox0, foff, nobj, f, b1, b2, beta, delta, out);
    CAXSI_CUDA_TRY(cudaGetLastError());
    return CAXSI_OK;
}

caxsi_status multi_update_vjp(const DevGeo *geos, const int64_t *foff, int nobj, const float *f, const float *b1,
                              const float *b2, float beta, float delta, const float *gx, float *gf, float *gb2,
                              float *scratch, int64_t n, cudaStream_t s) {
    float *gb3 = scratch, *gb5 = scratch + n;
    const unsigned nb = (unsigned)ceil_div64(n, 256);
    k_update_vjp1_multi<<<nb, 256, 0, s>>>(geos, foff, nobj, f, b1, b2, beta, delta, gx, gf, gb2, gb3, gb5, n);
    CAXSI_CUDA_TRY(cudaGetLastError());
    k_update_vjp2_multi<<<nb, 256, 0, s>>>(geos, foff, nobj, f, delta, gb3, gb5, gf, n);
    CAXSI_CUDA_TRY(cudaGetLastError());
    return CAXSI_OK;
}
