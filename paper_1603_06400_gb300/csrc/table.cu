// Table paths: exact evaluation through the piecewise-linear structure of the
// effective spectral factor W(r, theta) (Eq. 4) in u = sin(theta/2).
//
// In energy form W(r, u) = ang(theta) * sum_k c_k f~(r, a_k u - b), with f~ the
// hat-function interpolation of the q samples (knots at every integer bin
// position).  For each energy k, f~(a_k u - b) is linear in u between the
// points u_{k,m} = (m + b)/a_k, m = -1..Q, where a q-grid node is crossed.  So
// sum_k c_k f~(...) is linear in u between consecutive elements of the sorted
// union of these points ("knots" u_1 < ... < u_B), and linear interpolation
// between its values at the knots is exact.  This turns the paper's
// scatter-angle interpolation (Sec. III-B, which samples theta uniformly and
// so approximates S) into an exact scheme:
//
//   Wtab[r][t] = sum_l f[r][l] S~[t][l],  S~[t][l] = sum_k c_k hat(a_k u_t - b - l)
//
// is a dense contraction over q (a GEMM); each (voxel, pixel) pair then finds
// the interval [u_t, u_t+1] holding its u and interpolates (forward).  The
// adjoint scatters each pair's weight onto the two knots of its interval,
// V[r][t] += (1 - alpha) w, V[r][t+1] += alpha w, and contracts
// f[r][l] = sum_t V[r][t] S~[t][l] -- the exact transpose.
//
// Knot positions are generated in FP64, rounded to FP32 (the precision of the
// per-pair u), sorted and deduplicated; S~ is evaluated in FP64 at the rounded
// knots.  Only knots inside the range of u over the open pairs, plus one
// bracketing knot on each side, are kept.  The interval search uses a uniform
// bucket grid over the knot range followed by a short scan.
//
// The per-pair stages run on the precomputed pair records (records.cu, the
// default; deterministic) or, when the detector or the knot count exceeds the
// records' 16-bit fields, on the on-the-fly kernels below, which find each
// pair's interval per call (the adjoint's shared-memory row then accumulates
// with float atomics: reproducible to rounding, not bitwise).  The
// contractions run on the tcgen05 GEMM (tc_gemm.cu) or cuBLAS.
#include <cuda_bf16.h>
#include <cuda_fp16.h>
#include <math.h>
#include <string.h>

#include <algorithm>
#include <vector>

#include "internal.cuh"
#include "pairgeo.cuh"
#include "table.cuh"

cudaError_t launch_sum_parts(const float *part, int nparts, int64_t stride, float *out,
                             int64_t n, cudaStream_t s);

namespace {

constexpr int TAB_THREADS = 1024;

// Range of u over all open pairs (plan set-up).
__global__ void k_pair_urange(PairArgs A, unsigned int *umin, unsigned int *umax) {
    const DevGeo &g = A.g;
    const int64_t npairs = (int64_t)g.R * g.M * g.N;
    float lo = 3.4e38f, hi = 0.f;
    for (int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; t < npairs;
         t += (int64_t)gridDim.x * blockDim.x) {
        const int n = (int)(t % g.N);
        const int m = (int)((t / g.N) % g.M);
        const int v = (int)(t / ((int64_t)g.N * g.M));
        const uint32_t word = A.tbits[((int64_t)v * g.M + m) * g.Nw + (n >> 5)];
        if (!((word >> (n & 31)) & 1u)) continue;
        const float4 vx = A.vox[v];
        float u, ang;
        pair_u_angular(vx.x, vx.y, vx.w, (float)n - g.cN, A.zrow[m], g.p_y, g.Xd, u, ang);
        lo = fminf(lo, u);
        hi = fmaxf(hi, u);
    }
    for (int o = 16; o > 0; o >>= 1) {
        lo = fminf(lo, __shfl_down_sync(0xffffffffu, lo, o));
        hi = fmaxf(hi, __shfl_down_sync(0xffffffffu, hi, o));
    }
    if ((threadIdx.x & 31) == 0) {
        atomicMin(umin, __float_as_uint(lo));
        atomicMax(umax, __float_as_uint(hi));
    }
}

// S~[t][l] = sum_k c_k max(0, 1 - |a_k u_t - b - l|) in FP64.
__global__ void k_build_S(int B, int Q, int K, const float2 *knots, const double *ak,
                          const double *ck, double b, float *S) {
    const int64_t idx = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (idx >= (int64_t)B * Q) return;
    const int t = (int)(idx / Q), l = (int)(idx % Q);
    const double u = (double)knots[t].x;
    double s = 0.0;
    for (int k = 0; k < K; ++k) {
        const double x = ak[k] * u - b - (double)l;
        const double h = 1.0 - fabs(x);
        if (h > 0.0) s += ck[k] * h;
    }
    S[idx] = (float)s;
}

// Forward per-pair stage: block = 1024 threads over a chunk of PPT*1024
// detector pixels and a chunk of voxels; each voxel's Wtab row is staged in
// shared memory together with the knot and bucket tables.
template <int PPT>
__global__ void __launch_bounds__(TAB_THREADS, 1)
k_fwd_table(PairArgs A, TabArgs T, const float *__restrict__ Wtab, float *__restrict__ part,
            int vc) {
    extern __shared__ __align__(16) unsigned char smem_raw[];
    const DevGeo &g = A.g;
    float2 *s_kn = reinterpret_cast<float2 *>(smem_raw);
    float *s_w = reinterpret_cast<float *>(s_kn + T.B);
    uint16_t *s_bs = reinterpret_cast<uint16_t *>(s_w + T.Bp);
    const int tid = threadIdx.x;
    for (int t = tid; t < T.B; t += TAB_THREADS) s_kn[t] = T.knots[t];
    for (int t = tid; t < T.NB; t += TAB_THREADS) s_bs[t] = T.bstart[t];

    const int64_t npix = (int64_t)g.M * g.N;
    const int64_t p0 = (int64_t)blockIdx.y * PPT * TAB_THREADS + tid;
    // pixel coordinates of this thread's first pixel, stepped by TAB_THREADS
    const int step_m = TAB_THREADS / g.N, step_n = TAB_THREADS % g.N;
    const int v0 = blockIdx.x * vc;
    const int v1 = min(v0 + vc, g.R);
    float acc[PPT];
#pragma unroll
    for (int s = 0; s < PPT; ++s) acc[s] = 0.f;
    const float u_first = T.knots[0].x, u_last = T.knots[T.B - 1].x;

    for (int v = v0; v < v1; ++v) {
        __syncthreads();
        const float *wrow = Wtab + (int64_t)v * T.Bp;
        for (int t = tid; t <= T.B; t += TAB_THREADS) s_w[t] = wrow[t];
        __syncthreads();
        const int i = v / g.J, j = v - i * g.J;
        const float4 vx = A.vox[v];
        const uint32_t *tb = A.tbits + (int64_t)v * g.M * g.Nw;
        const float *god_i = A.god + (int64_t)i * g.M * g.ND - g.d_min - g.rho_y * j;
        int m = (int)(p0 / g.N), n = (int)(p0 % g.N);
#pragma unroll
        for (int s = 0; s < PPT; ++s) {
            if (p0 + (int64_t)s * TAB_THREADS < npix) {
                const uint32_t word = tb[m * g.Nw + (n >> 5)];
                if ((word >> (n & 31)) & 1u) {
                    float u, ang;
                    pair_u_angular(vx.x, vx.y, vx.w, (float)n - g.cN, A.zrow[m], g.p_y, g.Xd, u, ang);
                    if (u >= u_first && u <= u_last) {
                        const int t = find_interval(u, s_kn, s_bs, T.B, T.NB, T.u0, T.inv_h);
                        const float2 kn = s_kn[t];
                        const float al = (u - kn.x) * kn.y;
                        const float w0 = s_w[t];
                        const float W = fmaf(al, s_w[t + 1] - w0, w0);
                        acc[s] = fmaf(vx.z * god_i[(int64_t)m * g.ND + n] * ang, W, acc[s]);
                    }
                }
            }
            m += step_m;
            n += step_n;
            if (n >= g.N) { n -= g.N; ++m; }
        }
    }
#pragma unroll
    for (int s = 0; s < PPT; ++s) {
        const int64_t p = p0 + (int64_t)s * TAB_THREADS;
        if (p < npix) part[(int64_t)blockIdx.x * npix + p] = acc[s];
    }
}

// Adjoint per-pair stage: per voxel, scatter w-weighted pair contributions onto
// the two knots of each pair's interval in a shared-memory row, then write the
// row to Vtab.
template <int PPT>
__global__ void __launch_bounds__(TAB_THREADS, 1)
k_adj_table(PairArgs A, TabArgs T, const float *__restrict__ w, float *__restrict__ Vtab, int vc) {
    extern __shared__ __align__(16) unsigned char smem_raw[];
    const DevGeo &g = A.g;
    float2 *s_kn = reinterpret_cast<float2 *>(smem_raw);
    float *s_v = reinterpret_cast<float *>(s_kn + T.B);
    uint16_t *s_bs = reinterpret_cast<uint16_t *>(s_v + T.Bp);
    const int tid = threadIdx.x;
    for (int t = tid; t < T.B; t += TAB_THREADS) s_kn[t] = T.knots[t];
    for (int t = tid; t < T.NB; t += TAB_THREADS) s_bs[t] = T.bstart[t];

    const int64_t npix = (int64_t)g.M * g.N;
    const int step_m = TAB_THREADS / g.N, step_n = TAB_THREADS % g.N;
    const int v0 = blockIdx.x * vc;
    const int v1 = min(v0 + vc, g.R);
    const float u_first = T.knots[0].x, u_last = T.knots[T.B - 1].x;

    for (int v = v0; v < v1; ++v) {
        __syncthreads();
        for (int t = tid; t < T.Bp; t += TAB_THREADS) s_v[t] = 0.f;
        __syncthreads();
        const int i = v / g.J, j = v - i * g.J;
        const float4 vx = A.vox[v];
        const uint32_t *tb = A.tbits + (int64_t)v * g.M * g.Nw;
        const float *god_i = A.god + (int64_t)i * g.M * g.ND - g.d_min - g.rho_y * j;
        for (int64_t pc = 0; pc < npix; pc += (int64_t)PPT * TAB_THREADS) {
            const int64_t p0 = pc + tid;
            int m = (int)(p0 / g.N), n = (int)(p0 % g.N);
#pragma unroll
            for (int s = 0; s < PPT; ++s) {
                const int64_t p = p0 + (int64_t)s * TAB_THREADS;
                if (p < npix) {
                    const uint32_t word = tb[m * g.Nw + (n >> 5)];
                    const float wv = w[p];
                    if (((word >> (n & 31)) & 1u) && wv != 0.f) {
                        float u, ang;
                        pair_u_angular(vx.x, vx.y, vx.w, (float)n - g.cN, A.zrow[m], g.p_y, g.Xd, u, ang);
                        if (u >= u_first && u <= u_last) {
                            const int t = find_interval(u, s_kn, s_bs, T.B, T.NB, T.u0, T.inv_h);
                            const float2 kn = s_kn[t];
                            const float al = (u - kn.x) * kn.y;
                            const float c = vx.z * god_i[(int64_t)m * g.ND + n] * ang * wv;
                            const float hi = c * al;
                            atomicAdd(&s_v[t], c - hi);
                            atomicAdd(&s_v[t + 1], hi);
                        }
                    }
                }
                m += step_m;
                n += step_n;
                if (n >= g.N) { n -= g.N; ++m; }
            }
        }
        __syncthreads();
        float *vrow = Vtab + (int64_t)v * T.Bp;
        for (int t = tid; t < T.B; t += TAB_THREADS) vrow[t] = s_v[t];
    }
}

// Deterministic adjoint per-pair stage.  The structure of k_adj_table, but each
// contribution is converted to a 64-bit fixed-point integer (x 2^e, rounded) and
// the knot row is accumulated with 64-bit integer atomics, which are exact and
// so independent of the order in which the threads add: repeated calls are
// bitwise identical.  The exponent e is chosen per call so that no row entry can
// overflow: every contribution is at most cmax * max|w| (cmax = 2 max(C G_so) max(G_od
// dtheta), computed when the table is built; the angular factor is at most 2), a
// row entry sums at most M N of them, and e = 61 - ceil(log2(M N cmax max|w|)).
// The quantum 2^-e is then below 2^-61 of the largest possible entry: far under
// the FP32 rounding of any entry that matters for f = V S~.
#define CAXSI_CUDA_TRY_E(expr)                  \
    do {                                        \
        cudaError_t _e = (expr);                \
        if (_e != cudaSuccess) return _e;       \
    } while (0)

// max over voxels of C G_so (the z component of the voxel table)
__global__ void k_vox_zmax(const float4 *__restrict__ vox, int n, unsigned *out) {
    float m = 0.f;
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x) m = fmaxf(m, fabsf(vox[i].z));
    for (int o = 16; o > 0; o >>= 1) m = fmaxf(m, __shfl_down_sync(0xffffffffu, m, o));
    if ((threadIdx.x & 31) == 0) atomicMax(out, __float_as_uint(m));
}

__global__ void k_absmax(const float *__restrict__ x, int64_t n, unsigned *out) {
    float m = 0.f;
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x)
        m = fmaxf(m, fabsf(x[i]));
    for (int o = 16; o > 0; o >>= 1) m = fmaxf(m, __shfl_down_sync(0xffffffffu, m, o));
    if ((threadIdx.x & 31) == 0) atomicMax(out, __float_as_uint(m));   // non-negative floats order as integers
}

template <int PPT>
__global__ void __launch_bounds__(TAB_THREADS, 1)
k_adj_table_fx(PairArgs A, TabArgs T, const float *__restrict__ w, float *__restrict__ Vtab, int vc, float cmax,
               const unsigned *__restrict__ wmax_bits) {
    extern __shared__ __align__(16) unsigned char smem_raw[];
    const DevGeo &g = A.g;
    float2 *s_kn = reinterpret_cast<float2 *>(smem_raw);
    unsigned long long *s_v = reinterpret_cast<unsigned long long *>(s_kn + T.B);   // [Bp] two's complement
    uint16_t *s_bs = reinterpret_cast<uint16_t *>(s_v + T.Bp);
    const int tid = threadIdx.x;
    for (int t = tid; t < T.B; t += TAB_THREADS) s_kn[t] = T.knots[t];
    for (int t = tid; t < T.NB; t += TAB_THREADS) s_bs[t] = T.bstart[t];

    const int64_t npix = (int64_t)g.M * g.N;
    const int step_m = TAB_THREADS / g.N, step_n = TAB_THREADS % g.N;
    const int v0 = blockIdx.x * vc;
    const int v1 = min(v0 + vc, g.R);
    const float u_first = T.knots[0].x, u_last = T.knots[T.B - 1].x;
    // the fixed-point scale 2^e of this call
    const double bound = (double)npix * (double)cmax * (double)__uint_as_float(*wmax_bits);
    int e = 0;
    if (bound > 0.0 && isfinite(bound)) {
        frexp(bound, &e);                     // bound < 2^e
        e = 61 - e;
    }
    const double scale = ldexp(1.0, e), inv_scale = ldexp(1.0, -e);

    for (int v = v0; v < v1; ++v) {
        __syncthreads();
        for (int t = tid; t < T.Bp; t += TAB_THREADS) s_v[t] = 0ull;
        __syncthreads();
        const int i = v / g.J, j = v - i * g.J;
        const float4 vx = A.vox[v];
        const uint32_t *tb = A.tbits + (int64_t)v * g.M * g.Nw;
        const float *god_i = A.god + (int64_t)i * g.M * g.ND - g.d_min - g.rho_y * j;
        for (int64_t pc = 0; pc < npix; pc += (int64_t)PPT * TAB_THREADS) {
            const int64_t p0 = pc + tid;
            int m = (int)(p0 / g.N), n = (int)(p0 % g.N);
#pragma unroll
            for (int s = 0; s < PPT; ++s) {
                const int64_t p = p0 + (int64_t)s * TAB_THREADS;
                if (p < npix) {
                    const uint32_t word = tb[m * g.Nw + (n >> 5)];
                    const float wv = w[p];
                    if (((word >> (n & 31)) & 1u) && wv != 0.f) {
                        float u, ang;
                        pair_u_angular(vx.x, vx.y, vx.w, (float)n - g.cN, A.zrow[m], g.p_y, g.Xd, u, ang);
                        if (u >= u_first && u <= u_last) {
                            const int t = find_interval(u, s_kn, s_bs, T.B, T.NB, T.u0, T.inv_h);
                            const float2 kn = s_kn[t];
                            const float al = (u - kn.x) * kn.y;
                            const float c = vx.z * god_i[(int64_t)m * g.ND + n] * ang * wv;
                            const float hi = c * al;
                            atomicAdd(&s_v[t], (unsigned long long)__double2ll_rn((double)(c - hi) * scale));
                            atomicAdd(&s_v[t + 1], (unsigned long long)__double2ll_rn((double)hi * scale));
                        }
                    }
                }
                m += step_m;
                n += step_n;
                if (n >= g.N) { n -= g.N; ++m; }
            }
        }
        __syncthreads();
        float *vrow = Vtab + (int64_t)v * T.Bp;
        for (int t = tid; t < T.B; t += TAB_THREADS)
            vrow[t] = (float)((double)(long long)s_v[t] * inv_scale);
    }
}

template <int PPT>
cudaError_t launch_fwd(const caxsi_plan *p, const TablePath *T, float *part, cudaStream_t s) {
    dim3 grid(T->fwd_chunks, T->pix_chunks);
    auto kfn = k_fwd_table<PPT>;
    cudaError_t e = cudaFuncSetAttribute(kfn, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)T->smem_fwd);
    if (e != cudaSuccess) return e;
    TabArgs ta = tab_args(T);
    kfn<<<grid, TAB_THREADS, T->smem_fwd, s>>>(pair_args(p), ta, T->tab, part, T->fwd_vc);
    return cudaGetLastError();
}

template <int PPT>
cudaError_t launch_adj(const caxsi_plan *p, const TablePath *T, const float *w, cudaStream_t s) {
    auto kfn = k_adj_table<PPT>;
    cudaError_t e = cudaFuncSetAttribute(kfn, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)T->smem_adj);
    if (e != cudaSuccess) return e;
    TabArgs ta = tab_args(T);
    kfn<<<T->adj_chunks, TAB_THREADS, T->smem_adj, s>>>(pair_args(p), ta, w, T->tab, T->adj_vc);
    return cudaGetLastError();
}

cudaError_t dispatch_fwd(const caxsi_plan *p, const TablePath *T, float *part, cudaStream_t s) {
    switch (T->ppt) {
        case 1: return launch_fwd<1>(p, T, part, s);
        case 2: return launch_fwd<2>(p, T, part, s);
        case 4: return launch_fwd<4>(p, T, part, s);
        case 8: return launch_fwd<8>(p, T, part, s);
        default: return launch_fwd<16>(p, T, part, s);
    }
}

cudaError_t dispatch_adj(const caxsi_plan *p, const TablePath *T, const float *w, cudaStream_t s) {
    if (T->smem_adj_fx) {
        // deterministic form: the exact fixed-point sums, scaled by max|w| of this call
        CAXSI_CUDA_TRY_E(cudaMemsetAsync(T->wmax, 0, sizeof(unsigned), s));
        const int64_t npix = (int64_t)p->dg.M * p->dg.N;
        k_absmax<<<(unsigned)std::min<int64_t>(ceil_div64(npix, 256), 4 * p->num_sms), 256, 0, s>>>(w, npix, T->wmax);
        CAXSI_CUDA_TRY_E(cudaGetLastError());
        TabArgs ta = tab_args(T);
        switch (T->ppt) {
#define CAXSI_FX(PP)                                                                                           \
    case PP: {                                                                                                 \
        CAXSI_CUDA_TRY_E(cudaFuncSetAttribute(k_adj_table_fx<PP>, cudaFuncAttributeMaxDynamicSharedMemorySize, \
                                              (int)T->smem_adj_fx));                                            \
        k_adj_table_fx<PP><<<T->adj_chunks, TAB_THREADS, T->smem_adj_fx, s>>>(pair_args(p), ta, w, T->tab,     \
                                                                             T->adj_vc, T->cmax, T->wmax);     \
        return cudaGetLastError();                                                                             \
    }
            CAXSI_FX(1)
            CAXSI_FX(2)
            CAXSI_FX(4)
            CAXSI_FX(8)
            CAXSI_FX(16)
#undef CAXSI_FX
        }
    }
    switch (T->ppt) {
        case 1: return launch_adj<1>(p, T, w, s);
        case 2: return launch_adj<2>(p, T, w, s);
        case 4: return launch_adj<4>(p, T, w, s);
        case 8: return launch_adj<8>(p, T, w, s);
        default: return launch_adj<16>(p, T, w, s);
    }
}

void free_table(TablePath *T) {
    if (T) cudaFree(T->wmax);
    if (!T) return;
    records_free(T);
    cudaFree(T->S_hi);
    cudaFree(T->S_lo);
    cudaFree(T->St_hi);
    cudaFree(T->St_lo);
    cudaFree(T->St16[0]);
    cudaFree(T->St16[1]);
    for (int k = 0; k < 2; ++k) {
        cudaFree(T->kband[k]);
        cudaFree(T->nband[k]);
    }
    cudaFree(T->f_hi);
    if (T->blas) cublasDestroy(T->blas);
    cudaFree(T->blas_ws);
    cudaFree(T->S16[0]);
    cudaFree(T->S16[1]);
    cudaFree(T->f16);
    cudaFree(T->v16);
    cudaFree(T->knots);
    cudaFree(T->bstart);
    cudaFree(T->S);
    cudaFree(T->tab);
    cudaFree(T->fwd_part);
    BatchState &bs = T->batch;
    cudaFree(bs.items);
    cudaFree(bs.rowmap);
    cudaFree(bs.obj_items);
    cudaFree(bs.tab);
    cudaFree(bs.f_hi);
    cudaFree(bs.fpk);
    cudaFree(bs.part);
    delete T;
}

caxsi_status build_table(caxsi_plan *p) {
    const caxsi_geometry &G = p->g;
    const DevGeo &d = p->dg;
    TablePath *T = new TablePath();
    caxsi_status st = CAXSI_OK;
    unsigned int *ur = nullptr;
    double *ak_d = nullptr, *ck_d = nullptr;
    do {
        // 1. range of u over the open pairs
        if (cudaMalloc(&ur, 2 * sizeof(unsigned int)) != cudaSuccess) { st = CAXSI_ERR_OOM; break; }
        unsigned int init[2] = {0x7f7fffffu, 0u};
        cudaMemcpy(ur, init, sizeof(init), cudaMemcpyHostToDevice);
        k_pair_urange<<<4 * p->num_sms, 256>>>(pair_args(p), ur, ur + 1);
        unsigned int got[2];
        if (cudaGetLastError() != cudaSuccess ||
            cudaMemcpy(got, ur, sizeof(got), cudaMemcpyDeviceToHost) != cudaSuccess) {
            st = CAXSI_ERR_CUDA;
            break;
        }
        float ulo, uhi;
        memcpy(&ulo, &got[0], 4);
        memcpy(&uhi, &got[1], 4);

        // 2. knots u_{k,m} = (m + b)/a_k in FP64, rounded to FP32, sorted, unique
        const double dE = (G.E_max - G.E_min) / G.K;
        const double dq = (G.q_max - G.q_min) / (G.Q - 1);
        const double b = G.q_min / dq;
        std::vector<double> ak(G.K), ck(G.K);
        std::vector<float> kn;
        kn.reserve((size_t)G.K * (G.Q + 2));
        for (int k = 0; k < G.K; ++k) {
            const double E = G.E_min + (k + 0.5) * dE;
            ak[k] = E / (G.hc * dq);
            for (int m = -1; m <= G.Q; ++m) {
                const double u = (m + b) / ak[k];
                if (u > 0.0) kn.push_back((float)u);
            }
        }
        // with q_min < dq every tau_k(0) = -b lies inside (-1, 0], where f~ is
        // already nonzero: W is then linear on [0, first crossing] and u = 0
        // must be a knot too
        if (b < 1.0) kn.push_back(0.f);
        std::sort(kn.begin(), kn.end());
        kn.erase(std::unique(kn.begin(), kn.end()), kn.end());
        if (kn.size() < 2) { st = CAXSI_ERR_UNSUPPORTED; break; }
        // keep [last knot <= ulo, first knot >= uhi]
        int lo = 0, hi = (int)kn.size() - 1;
        if (got[1] >= got[0]) {
            auto itl = std::upper_bound(kn.begin(), kn.end(), ulo);
            lo = itl == kn.begin() ? 0 : (int)(itl - kn.begin()) - 1;
            auto ith = std::lower_bound(kn.begin(), kn.end(), uhi);
            hi = ith == kn.end() ? (int)kn.size() - 1 : (int)(ith - kn.begin());
        }
        if (hi - lo + 1 < 2) { if (hi + 1 < (int)kn.size()) ++hi; else if (lo > 0) --lo; }
        std::vector<float> knots(kn.begin() + lo, kn.begin() + hi + 1);
        if (p->u_samples >= 2) {
            // N uniform samples over the same range instead of the exact knots: W is
            // then interpolated between samples (an approximation of A)
            const int N = p->u_samples;
            const double u_a = knots.front(), u_b = knots.back();
            knots.resize(N);
            for (int j = 0; j < N; ++j) knots[j] = (float)(u_a + (u_b - u_a) * j / (N - 1));
            knots.back() = (float)u_b;
            knots.erase(std::unique(knots.begin(), knots.end()), knots.end());
        }
        const int B = (int)knots.size();
        if (B < 2 || B > 65535) { st = CAXSI_ERR_UNSUPPORTED; break; }
        T->B = B;
        T->Bp = ((B + 1) + 7) / 8 * 8;

        // spectral weights c_k = Phi_k E_k dE / hc^2 in FP64 (energy form of Eq. 4)
        for (int k = 0; k < G.K; ++k) {
            const double E = G.E_min + (k + 0.5) * dE;
            ck[k] = p->phi[k] * E * dE / (G.hc * G.hc);
        }

        // 3. knot records and bucket grid
        std::vector<float2> krec(B);
        for (int t = 0; t < B; ++t) {
            const float ut = knots[t];
            const float inv = (t + 1 < B) ? (float)(1.0 / ((double)knots[t + 1] - (double)ut)) : 0.f;
            krec[t] = make_float2(ut, inv);
        }
        const int NB = std::min(65535, 2 * B);
        const double span = (double)knots[B - 1] - (double)knots[0];
        const double h = span / NB;
        T->NB = NB;
        T->u0 = knots[0];
        T->inv_h = (float)(1.0 / h);
        std::vector<uint16_t> bs(NB);
        {
            int t = 0;
            for (int bk = 0; bk < NB; ++bk) {
                const double start = (double)knots[0] + bk * h;
                while (t + 1 < B && (double)knots[t + 1] <= start) ++t;
                bs[bk] = (uint16_t)t;
            }
        }
        const int64_t R = d.R;
        if (cudaMalloc(&T->knots, B * sizeof(float2)) != cudaSuccess ||
            cudaMalloc(&T->bstart, NB * sizeof(uint16_t)) != cudaSuccess ||
            cudaMalloc(&T->S, (size_t)B * G.Q * sizeof(float)) != cudaSuccess ||
            cudaMalloc(&T->tab, (size_t)R * T->Bp * sizeof(float)) != cudaSuccess ||
            cudaMalloc(&ak_d, G.K * sizeof(double)) != cudaSuccess ||
            cudaMalloc(&ck_d, G.K * sizeof(double)) != cudaSuccess) {
            st = CAXSI_ERR_OOM;
            break;
        }
        cudaMemcpy(T->knots, krec.data(), B * sizeof(float2), cudaMemcpyHostToDevice);
        cudaMemcpy(T->bstart, bs.data(), NB * sizeof(uint16_t), cudaMemcpyHostToDevice);
        cudaMemcpy(ak_d, ak.data(), G.K * sizeof(double), cudaMemcpyHostToDevice);
        cudaMemcpy(ck_d, ck.data(), G.K * sizeof(double), cudaMemcpyHostToDevice);
        cudaMemset(T->tab, 0, (size_t)R * T->Bp * sizeof(float));
        k_build_S<<<(unsigned)ceil_div64((int64_t)B * G.Q, 256), 256>>>(B, G.Q, G.K, T->knots, ak_d, ck_d, b, T->S);
        if (cudaGetLastError() != cudaSuccess || cudaDeviceSynchronize() != cudaSuccess) {
            st = CAXSI_ERR_CUDA;
            break;
        }

        // 4. launch shapes
        const int64_t npix = (int64_t)G.M * G.N;
        int ppt = 1;
        while (ppt < 16 && (int64_t)ppt * TAB_THREADS < npix) ppt *= 2;
        T->ppt = ppt;
        T->pix_chunks = (int)ceil_div64(npix, (int64_t)ppt * TAB_THREADS);
        int chunks = (int)ceil_div64(2 * p->num_sms, T->pix_chunks);
        if (chunks > d.R) chunks = d.R;
        T->fwd_vc = (int)ceil_div64(d.R, chunks);
        T->fwd_chunks = (int)ceil_div64(d.R, T->fwd_vc);
        int ac = 2 * p->num_sms;
        if (ac > d.R) ac = d.R;
        T->adj_vc = (int)ceil_div64(d.R, ac);
        T->adj_chunks = (int)ceil_div64(d.R, T->adj_vc);
        T->smem_fwd = (size_t)B * sizeof(float2) + (size_t)T->Bp * sizeof(float) + (size_t)NB * sizeof(uint16_t);
        T->smem_adj = T->smem_fwd;
        int smem_max = 0;
        cudaDeviceGetAttribute(&smem_max, cudaDevAttrMaxSharedMemoryPerBlockOptin, p->device);
        // the deterministic adjoint holds its knot row as 64-bit integers: where that
        // fits (up to about 14 000 knots) it replaces the float atomics
        {
            const size_t fx = (size_t)B * sizeof(float2) + (size_t)T->Bp * sizeof(unsigned long long) +
                              (size_t)NB * sizeof(uint16_t);
            T->smem_adj_fx = fx <= (size_t)smem_max ? fx : 0;
        }
        if (T->smem_adj_fx) {
            // cmax = 2 max(C G_so) max(G_od dtheta), with a margin for rounding
            unsigned h[2] = {0u, 0u};
            if (cudaMalloc(&T->wmax, 2 * sizeof(unsigned)) != cudaSuccess ||
                cudaMemset(T->wmax, 0, 2 * sizeof(unsigned)) != cudaSuccess) {
                st = CAXSI_ERR_OOM;
                break;
            }
            const int64_t n_god = (int64_t)d.X * d.M * d.ND;
            k_vox_zmax<<<(unsigned)std::min<int64_t>(ceil_div64(d.R, 256), 4 * p->num_sms), 256>>>(p->vox, d.R, T->wmax);
            k_absmax<<<(unsigned)std::min<int64_t>(ceil_div64(n_god, 256), 4 * p->num_sms), 256>>>(p->god, n_god,
                                                                                                 T->wmax + 1);
            if (cudaGetLastError() != cudaSuccess ||
                cudaMemcpy(h, T->wmax, 2 * sizeof(unsigned), cudaMemcpyDeviceToHost) != cudaSuccess) {
                st = CAXSI_ERR_CUDA;
                break;
            }
            float zmax, gmax;
            memcpy(&zmax, &h[0], sizeof(float));
            memcpy(&gmax, &h[1], sizeof(float));
            T->cmax = 2.f * zmax * gmax * 1.001f;
        }
        if ((size_t)smem_max < T->smem_fwd) { st = CAXSI_ERR_UNSUPPORTED; break; }
        if (cudaMalloc(&T->fwd_part, (size_t)T->fwd_chunks * npix * sizeof(float)) != cudaSuccess) {
            st = CAXSI_ERR_OOM;
            break;
        }
        p->table_bytes += (int64_t)B * 8 + NB * 2 + (int64_t)B * G.Q * 4 + R * T->Bp * 4 +
                          (int64_t)T->fwd_chunks * npix * 4;
        // 5. per-pair records (precomputed intervals and weights), when they fit
        if ((st = records_build(p, T)) != CAXSI_OK) break;
        // 6. mirror-symmetric records for the forward, when the geometry allows them
        if ((st = sym_build(p, T)) != CAXSI_OK) break;
        if (T->use_records && T->rec_chunks > T->fwd_chunks) {
            cudaFree(T->fwd_part);
            T->fwd_part = nullptr;
            if (cudaMalloc(&T->fwd_part, (size_t)T->rec_chunks * npix * sizeof(float)) != cudaSuccess) {
                st = CAXSI_ERR_OOM;
                break;
            }
        }
    } while (0);
    cudaFree(ur);
    cudaFree(ak_d);
    cudaFree(ck_d);
    if (st != CAXSI_OK) {
        free_table(T);
        return st;
    }
    p->table = T;
    return CAXSI_OK;
}

}  // namespace

int64_t table_breakpoints(const caxsi_plan *p) { return p->table ? p->table->B : 0; }
int64_t table_records(const caxsi_plan *p) { return p->table ? p->table->rec.n : 0; }
int64_t table_sym_records(const caxsi_plan *p) { return p->table ? p->table->sym.adj.n : 0; }

namespace {

// Row-padded operand copies: x [rows][Q] -> y [rows][Qp] (zeros beyond Q), as
// bf16 (kind 1), fp16 (kind 2), a TF32 high/low split rounded to nearest (kind
// 0, the B operands) or truncated (kind 3, the A operands).
__global__ void k_pad_convert(const float *__restrict__ x, int64_t rows, int Q, int Qp, int kind,
                              void *__restrict__ y, float *__restrict__ ylo) {
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= rows * Qp) return;
    const int64_t r = i / Qp;
    const int l = (int)(i - r * Qp);
    const float v = l < Q ? x[r * Q + l] : 0.f;
    if (kind == 1) {
        reinterpret_cast<__nv_bfloat16 *>(y)[i] = __float2bfloat16_rn(v);
    } else if (kind == 2) {
        reinterpret_cast<__half *>(y)[i] = __float2half_rn(v);
    } else if (kind == 4) {   // the padded FP32 copy (split on chip by the contraction)
        reinterpret_cast<float *>(y)[i] = v;
    } else {
        float h, lo;
        if (kind == 3) tf32_split_trunc(v, h, lo);
        else tf32_split(v, h, lo);
        reinterpret_cast<float *>(y)[i] = h;
        ylo[i] = lo;
    }
}

cudaError_t pad_convert(const float *x, int64_t rows, int Q, int Qp, int kind, void *y, float *ylo,
                        cudaStream_t s) {
    const int64_t n = rows * Qp;
    k_pad_convert<<<(unsigned)ceil_div64(n, 256), 256, 0, s>>>(x, rows, Q, Qp, kind, y, ylo);
    return cudaGetLastError();
}

// S~^T [Q][Bp] from S~ [B][Q]: TF32 split and 16-bit copies (zero padding t >= B).
// S~ [B][Q] TF32-split for the forward contraction (B operand, 256-row n-tiles),
// stored in k-block order: element (t, l) at ((t / 256) nkq + l / 32) 256 * 32 +
// (t % 256) 32 + l % 32, nkq = ceil(Q / 32): each 256-row k-block tile is one
// contiguous 32 KB block (the rest of the buffer is zero).
__global__ void k_block_S(const float *__restrict__ S, int B, int Q, float *__restrict__ hi,
                          float *__restrict__ lo) {
    const int64_t idx = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (idx >= (int64_t)B * Q) return;
    const int t = (int)(idx / Q), l = (int)(idx % Q);
    float h, lw;
    tf32_split(S[idx], h, lw);
    const int64_t nkq = (Q + 31) / 32;
    const int64_t i = ((t / 256) * nkq + l / 32) * 8192 + (t % 256) * 32 + l % 32;
    hi[i] = h;
    lo[i] = lw;
}

// S~^T [Q][B] for the adjoint contraction, stored as the GEMM's B operand in
// k-block order: element (l, t) at ((l / 128) nkb + t / KE) 128 KE + (l % 128) KE
// + t % KE, KE = 32 (FP32 splits) or 64 (16-bit copies), nkb = ceil(B / KE), so
// that each 128-row k-block tile is one contiguous 16 KB block (the rest of the
// buffer is zero).
__global__ void k_transpose_S(const float *__restrict__ S, int B, int Q, float *__restrict__ hi,
                              float *__restrict__ lo, __nv_bfloat16 *__restrict__ bf, __half *__restrict__ hf) {
    const int64_t idx = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (idx >= (int64_t)Q * B) return;
    const int l = (int)(idx / B), t = (int)(idx % B);
    const float x = S[(int64_t)t * Q + l];
    float h, lw;
    tf32_split(x, h, lw);
    const int64_t nkb32 = (B + 31) / 32, nkb64 = (B + 63) / 64;
    const int64_t i32 = ((l / 128) * nkb32 + t / 32) * 4096 + (l % 128) * 32 + t % 32;
    const int64_t i64 = ((l / 128) * nkb64 + t / 64) * 8192 + (l % 128) * 64 + t % 64;
    hi[i32] = h;
    lo[i32] = lw;
    bf[i64] = __float2bfloat16_rn(x);
    hf[i64] = __float2half_rn(x);
}

// cuBLAS handle, workspace and 16-bit operand copies (first table call).
caxsi_status blas_setup(caxsi_plan *p, TablePath *T) {
    const DevGeo &d = p->dg;
    if (cublasCreate(&T->blas) != CUBLAS_STATUS_SUCCESS) {
        T->blas = nullptr;
        return CAXSI_ERR_CUDA;
    }
    T->blas_ws_bytes = (size_t)64 << 20;
    T->Qp = (d.Q + 7) / 8 * 8;
    const int64_t nS = (int64_t)T->B * T->Qp;
    if (cudaMalloc(&T->blas_ws, T->blas_ws_bytes) != cudaSuccess ||
        cudaMalloc(&T->S16[0], nS * 2) != cudaSuccess || cudaMalloc(&T->S16[1], nS * 2) != cudaSuccess ||
        cudaMalloc(&T->f16, (size_t)d.R * T->Qp * 2) != cudaSuccess ||
        cudaMalloc(&T->v16, (size_t)d.R * T->Bp * 2) != cudaSuccess)
        return CAXSI_ERR_OOM;
    if (cublasSetWorkspace(T->blas, T->blas_ws, T->blas_ws_bytes) != CUBLAS_STATUS_SUCCESS)
        return CAXSI_ERR_CUDA;
    if (pad_convert(T->S, T->B, d.Q, T->Qp, 1, T->S16[0], nullptr, 0) != cudaSuccess ||
        pad_convert(T->S, T->B, d.Q, T->Qp, 2, T->S16[1], nullptr, 0) != cudaSuccess ||
        cudaDeviceSynchronize() != cudaSuccess)
        return CAXSI_ERR_CUDA;
    p->table_bytes += (int64_t)T->blas_ws_bytes + 2 * nS * 2 + (int64_t)d.R * T->Qp * 2 + (int64_t)d.R * T->Bp * 2;
    // operands of the hand-written tcgen05 GEMM
    // S~^T in k-block order (k_transpose_S): whole 128-row blocks, zero padding
    const int64_t nf = (int64_t)d.R * T->Qp;
    const int64_t nrb = (d.Q + 127) / 128;
    const int64_t nSt32 = nrb * ((T->B + 31) / 32) * 4096, nSt16 = nrb * ((T->B + 63) / 64) * 8192;
    const int64_t nSb = std::max<int64_t>(nS, (int64_t)(T->B + 255) / 256 * ((d.Q + 31) / 32) * 8192);
    if (cudaMalloc(&T->S_hi, nSb * 4) != cudaSuccess || cudaMalloc(&T->S_lo, nSb * 4) != cudaSuccess ||
        cudaMalloc(&T->St_hi, nSt32 * 4) != cudaSuccess || cudaMalloc(&T->St_lo, nSt32 * 4) != cudaSuccess ||
        cudaMalloc(&T->St16[0], nSt16 * 2) != cudaSuccess || cudaMalloc(&T->St16[1], nSt16 * 2) != cudaSuccess ||
        cudaMalloc(&T->f_hi, nf * 4) != cudaSuccess)
        return CAXSI_ERR_OOM;
    if (cudaMemset(T->St_hi, 0, nSt32 * 4) != cudaSuccess || cudaMemset(T->St_lo, 0, nSt32 * 4) != cudaSuccess ||
        cudaMemset(T->St16[0], 0, nSt16 * 2) != cudaSuccess || cudaMemset(T->St16[1], 0, nSt16 * 2) != cudaSuccess)
        return CAXSI_ERR_CUDA;
    if (cudaMemset(T->S_hi, 0, nSb * 4) != cudaSuccess || cudaMemset(T->S_lo, 0, nSb * 4) != cudaSuccess)
        return CAXSI_ERR_CUDA;
    k_block_S<<<(unsigned)ceil_div64((int64_t)T->B * d.Q, 256), 256>>>(T->S, T->B, d.Q, T->S_hi, T->S_lo);
    k_transpose_S<<<(unsigned)ceil_div64((int64_t)d.Q * T->B, 256), 256>>>(
        T->S, T->B, d.Q, T->St_hi, T->St_lo, (__nv_bfloat16 *)T->St16[0], (__half *)T->St16[1]);
    if (cudaGetLastError() != cudaSuccess || cudaDeviceSynchronize() != cudaSuccess) return CAXSI_ERR_CUDA;
    p->table_bytes += 2 * nS * 4 + nSt32 * 8 + nSt16 * 4 + nf * 4;
    // the q band of each knot's row of S~ (first and last nonzero), and the GEMMs'
    // band tables from it
    std::vector<float> hS((size_t)T->B * d.Q);
    if (cudaMemcpy(hS.data(), T->S, hS.size() * 4, cudaMemcpyDeviceToHost) != cudaSuccess) return CAXSI_ERR_CUDA;
    std::vector<int2> nz(T->B);
    for (int t = 0; t < T->B; ++t) {
        int lo = d.Q, hi = -1;
        for (int l = 0; l < d.Q; ++l)
            if (hS[(size_t)t * d.Q + l] != 0.f) {
                lo = std::min(lo, l);
                hi = l;
            }
        nz[t] = make_int2(lo, hi);
    }
    for (int k = 0; k < 2; ++k) {
        const int eb = k == 0 ? 4 : 2;
        const std::vector<int2> kb = tc_kband(nz, T->B, 256, d.Q, eb);
        const std::vector<int2> nb = tc_nband(nz, d.Q, 128, T->B, eb);
        if (cudaMalloc(&T->kband[k], kb.size() * sizeof(int2)) != cudaSuccess ||
            cudaMalloc(&T->nband[k], nb.size() * sizeof(int2)) != cudaSuccess)
            return CAXSI_ERR_OOM;
        if (cudaMemcpy(T->kband[k], kb.data(), kb.size() * sizeof(int2), cudaMemcpyHostToDevice) != cudaSuccess ||
            cudaMemcpy(T->nband[k], nb.data(), nb.size() * sizeof(int2), cudaMemcpyHostToDevice) != cudaSuccess)
            return CAXSI_ERR_CUDA;
    }
    return CAXSI_OK;
}

// Row-mapped copy of the forward input: packed row r takes source row rowmap[r]
// of x (the batched operators' packing), padded to Qp (the contraction splits it
// into TF32 parts on chip).
__global__ void k_pack_rows(const float *__restrict__ x, const int64_t *__restrict__ rowmap, int64_t rows, int Q,
                             int Qp, float *__restrict__ y) {
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= rows * Qp) return;
    const int64_t r = i / Qp;
    const int l = (int)(i - r * Qp);
    y[i] = l < Q ? x[rowmap[r] * Q + l] : 0.f;
}

// Packed adjoint rows back to each object's [R][Q] block (rows outside an
// object's range were cleared before).
__global__ void k_unpack_rows(const float *__restrict__ fpk, const int64_t *__restrict__ rowmap, int64_t rows,
                              int Q, float *__restrict__ out) {
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= rows * Q) return;
    const int64_t r = i / Q;
    const int l = (int)(i - r * Q);
    out[rowmap[r] * Q + l] = fpk[i];
}

// g_b = sum of object b's partial images, in item (voxel chunk) order.
__global__ void k_sum_parts_batch(const float *__restrict__ part, const int2 *__restrict__ obj_items, int64_t npix,
                                  float *__restrict__ g) {
    const int b = blockIdx.y;
    const int64_t idx = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (idx >= npix) return;
    const int2 oi = obj_items[b];
    // the same order and grouping of loads as k_sum_parts (equal results)
    const float *pp = part + (int64_t)oi.x * npix + idx;
    float acc = 0.f;
    int c = 0;
    for (; c + 32 <= oi.y; c += 32) {
        float v[32];
#pragma unroll
        for (int k = 0; k < 32; ++k) v[k] = pp[(int64_t)(c + k) * npix];
#pragma unroll
        for (int k = 0; k < 32; ++k) acc += v[k];
    }
    for (; c < oi.y; ++c) acc += pp[(int64_t)c * npix];
    g[(int64_t)b * npix + idx] = acc;
}

template <typename X>
cudaError_t grow(X *&ptr, int64_t &cap, int64_t need, int64_t elems_per_unit) {
    if (need <= cap && ptr) return cudaSuccess;
    cudaFree(ptr);
    ptr = nullptr;
    cap = 0;
    cudaError_t e = cudaMalloc(&ptr, (size_t)(need > 0 ? need : 1) * elems_per_unit * sizeof(X));
    if (e == cudaSuccess) cap = need;
    return e;
}

// Lay out a batch: object b is voxels [ranges[2b], ranges[2b+1]); its rows are
// packed after those of objects 0..b-1; its work items are the record kernels'
// voxel chunks cut to its range (so each object's sums run in the same order as
// a single-object call).  Reuses the device arrays when the layout is unchanged.
caxsi_status batch_layout(caxsi_plan *p, TablePath *T, int nb, const int32_t *ranges, cudaStream_t s) {
    BatchState &bs = T->batch;
    const DevGeo &d = p->dg;
    if (bs.nb == nb && bs.ranges.size() == (size_t)(2 * nb) &&
        std::equal(bs.ranges.begin(), bs.ranges.end(), ranges))
        return CAXSI_OK;
    // forget the old layout first: a failure below leaves no layout to reuse
    bs.nb = 0;
    bs.ranges.clear();
    std::vector<int4> items;
    std::vector<int2> oi(nb);
    std::vector<int64_t> rowmap;
    int64_t rows = 0;
    const int vc = T->rec_vc;
    for (int b = 0; b < nb; ++b) {
        const int vb = ranges[2 * b], ve = ranges[2 * b + 1];
        oi[b] = make_int2((int)items.size(), 0);
        if (ve > vb) {
            for (int c = vb / vc; c * vc < ve; ++c) {
                const int v0 = std::max(vb, c * vc), v1 = std::min(ve, (c + 1) * vc);
                items.push_back(make_int4(b, v0, v1, (int)(rows + (v0 - vb))));
            }
            for (int v = vb; v < ve; ++v) rowmap.push_back((int64_t)b * d.R + v);
            rows += ve - vb;
        }
        oi[b].y = (int)items.size() - oi[b].x;
    }
    if (rows >= (int64_t)1 << 31) return CAXSI_ERR_INVALID;
    int64_t icap = bs.items_cap, ncap = bs.nb_cap;
    CAXSI_CUDA_TRY(grow(bs.items, icap, (int64_t)items.size(), 1));
    CAXSI_CUDA_TRY(grow(bs.obj_items, ncap, nb, 1));
    int64_t rcap = bs.rows_cap;
    if (rows > rcap || !bs.rowmap) {
        cudaFree(bs.rowmap);
        cudaFree(bs.tab);
        cudaFree(bs.f_hi);
        cudaFree(bs.fpk);
        bs.rowmap = nullptr;
        bs.tab = bs.f_hi = bs.fpk = nullptr;
        bs.rows_cap = 0;
        const size_t r = (size_t)(rows > 0 ? rows : 1);
        CAXSI_CUDA_TRY(cudaMalloc(&bs.rowmap, r * sizeof(int64_t)));
        CAXSI_CUDA_TRY(cudaMalloc(&bs.tab, r * T->Bp * sizeof(float)));
        CAXSI_CUDA_TRY(cudaMalloc(&bs.f_hi, r * T->Qp * sizeof(float)));
        CAXSI_CUDA_TRY(cudaMalloc(&bs.fpk, r * d.Q * sizeof(float)));
        bs.rows_cap = rows;
    }
    const int64_t npix = (int64_t)d.M * d.N;
    CAXSI_CUDA_TRY(grow(bs.part, bs.part_cap, (int64_t)items.size(), npix));
    bs.items_cap = (int)icap;
    bs.nb_cap = (int)ncap;
    if (!items.empty())
        CAXSI_CUDA_TRY(cudaMemcpyAsync(bs.items, items.data(), items.size() * sizeof(int4), cudaMemcpyHostToDevice, s));
    CAXSI_CUDA_TRY(cudaMemcpyAsync(bs.obj_items, oi.data(), nb * sizeof(int2), cudaMemcpyHostToDevice, s));
    if (rows > 0)
        CAXSI_CUDA_TRY(cudaMemcpyAsync(bs.rowmap, rowmap.data(), rows * sizeof(int64_t), cudaMemcpyHostToDevice, s));
    // the host vectors are pageable: the copies have been staged when they return,
    // but keep the device state consistent with the layout only once they are done
    CAXSI_CUDA_TRY(cudaStreamSynchronize(s));
    bs.ranges.assign(ranges, ranges + 2 * nb);
    bs.nb = nb;
    bs.rows = rows;
    bs.n_items = (int)items.size();
    return CAXSI_OK;
}

caxsi_status ensure_table(caxsi_plan *p, int path) {
    if (path < CAXSI_PATH_TABLE_FP32 || path > CAXSI_PATH_TABLE_FP16) return CAXSI_ERR_UNSUPPORTED;
    if (!p->table) {
        // all or nothing: a table that failed half way is dropped, and the next call
        // builds it again
        const int64_t bytes0 = p->table_bytes;
        caxsi_status st = build_table(p);
        if (st == CAXSI_OK) st = blas_setup(p, p->table);
        if (st != CAXSI_OK) {
            cudaDeviceSynchronize();
            free_table(p->table);
            p->table = nullptr;
            p->table_bytes = bytes0;
            return st;
        }
    }
    // the 16-bit paths take their adjoint rows from the record kernel
    if (path != CAXSI_PATH_TABLE_FP32 && !p->table->use_records) return CAXSI_ERR_UNSUPPORTED;
    return CAXSI_OK;
}

cudaDataType_t dtype16(int path) { return path == CAXSI_PATH_TABLE_BF16 ? CUDA_R_16BF : CUDA_R_16F; }

// The band tables of the tcgen05 contractions (k = 0: TF32 operands, 1: 16-bit),
// or null when the plan has band skipping off.
const int2 *kband_of(const caxsi_plan *p, int k) { return p->no_bands ? nullptr : p->table->kband[k]; }
const int2 *nband_of(const caxsi_plan *p, int k) { return p->no_bands ? nullptr : p->table->nband[k]; }

}  // namespace

caxsi_status table_forward(caxsi_plan *p, const float *f, float *g_out, int path, int subset, cudaStream_t s) {
    caxsi_status st = ensure_table(p, path);
    if (st != CAXSI_OK) return st;
    TablePath *T = p->table;
    if (subset >= 0) {   // the records grouped by the current partition (built on first use)
        if (!T->use_records) return CAXSI_ERR_UNSUPPORTED;
        if ((st = table_set_subsets(p)) != CAXSI_OK) return st;
        if (subset >= T->sub.P) return CAXSI_ERR_UNSUPPORTED;
        // FP32: W only at the subset's knots, per record, instead of the whole contraction
        if (path == CAXSI_PATH_TABLE_FP32 && !p->no_sparse_subsets && sub_sparse_ok(p, f, g_out, 160)) {
            bool done = false;
            CAXSI_PROF(p, "sub_fwd_sparse", s);
            CAXSI_CUDA_TRY(sub_forward_sparse(p, T, subset, f, g_out, s, done));
            if (done) return CAXSI_OK;
        }
    }
    const DevGeo &d = p->dg;
    const float one = 1.f, zero = 0.f;
    // the full forward over the mirror-symmetric records
    const bool sym_fwd = T->use_records && subset < 0 && T->sym.ok && !p->no_symmetry;
    if (cublasSetStream(T->blas, s) != CUBLAS_STATUS_SUCCESS) return CAXSI_ERR_CUDA;
    const bool raw_hi = d.Q == T->Qp && (reinterpret_cast<uintptr_t>(f) & 15) == 0;
    // a host-buffer call: the rest of f may still be on its way
    HostPipe *pipe = p->pipe;
    const bool split = pipe && p->gemm_engine == 0 && path == CAXSI_PATH_TABLE_FP32 && raw_hi && subset < 0 &&
                       pipe->rows > 0 && pipe->rows < d.R;
    if (pipe && !split) CAXSI_CUDA_TRY(cudaStreamWaitEvent(s, pipe->in_ready, 0));
    if (split) {
        // Wtab = f S~^T as below, the rows of each part in their own launch: the
        // second after the rest of f has arrived
        const int64_t r1 = pipe->rows;
        for (int h = 0; h < 2; ++h) {
            const int64_t r0 = h ? r1 : 0, nr = h ? d.R - r1 : r1;
            if (h) CAXSI_CUDA_TRY(cudaStreamWaitEvent(s, pipe->in_ready, 0));
            {
                CAXSI_PROF(p, "tc_gemm_fwd_3xtf32", s);
                CAXSI_CUDA_TRY(tc_gemm(4, 256, (int)nr, T->B, d.Q, f + r0 * d.Q, nullptr, T->Qp, T->S_hi, T->S_lo,
                                       T->Qp, T->tab + r0 * T->Bp, T->Bp, p->err_flag + 1, p->num_sms, s,
                                       kband_of(p, 0), nullptr, nullptr, 1));
            }
            CAXSI_LAUNCH_CHECK(p);
        }
    } else if (p->gemm_engine == 0 && path == CAXSI_PATH_TABLE_FP32) {
        // Wtab[r][t] = sum_l f[r][l] S~[t][l] by the tcgen05 GEMM, 3xTF32, the TF32
        // split of f made on chip (the tensor core reads FP32 as TF32 by dropping
        // the low 13 mantissa bits; converter warps write the remainder).  Rows that
        // are not 16-byte multiples or not aligned go through a padded copy first.
        if (!raw_hi) {
            {
                CAXSI_PROF(p, "pad_f", s);
                CAXSI_CUDA_TRY(pad_convert(f, d.R, d.Q, T->Qp, 4, T->f_hi, nullptr, s));
            }
            CAXSI_LAUNCH_CHECK(p);
        }
        {
            CAXSI_PROF(p, "tc_gemm_fwd_3xtf32", s);
            CAXSI_CUDA_TRY(tc_gemm(4, 256, d.R, T->B, d.Q, raw_hi ? f : T->f_hi, nullptr, T->Qp, T->S_hi, T->S_lo,
                                   T->Qp, T->tab, T->Bp, p->err_flag + 1, p->num_sms, s, kband_of(p, 0), nullptr,
                                   nullptr, 1));
        }
        CAXSI_LAUNCH_CHECK(p);
    } else if (p->gemm_engine == 0) {
        const int k = path == CAXSI_PATH_TABLE_BF16 ? 0 : 1;
        {
            CAXSI_PROF(p, "to_16bit", s);
            CAXSI_CUDA_TRY(pad_convert(f, d.R, d.Q, T->Qp, 1 + k, T->f16, nullptr, s));
        }
        CAXSI_LAUNCH_CHECK(p);
        {
            // the bf16 path keeps its knot rows in bf16 for the mirror-symmetric forward
            // (half the bytes written here and streamed there); the fp16 path keeps
            // FP32 rows (fp16's range would not hold every table value)
            CAXSI_PROF(p, k == 0 ? "tc_gemm_fwd_bf16" : "tc_gemm_fwd_fp16", s);
            uint16_t *w16 = (k == 0 && sym_fwd) ? reinterpret_cast<uint16_t *>(T->v16) : nullptr;
            CAXSI_CUDA_TRY(tc_gemm(1 + k, 256, d.R, T->B, d.Q, T->f16, nullptr, T->Qp, T->S16[k], nullptr, T->Qp,
                                   T->tab, T->Bp, p->err_flag + 1, p->num_sms, s, kband_of(p, 1), nullptr, w16));
        }
        CAXSI_LAUNCH_CHECK(p);
    } else if (path == CAXSI_PATH_TABLE_FP32) {
        // Wtab[r][t] = sum_l f[r][l] S~[t][l]  (column-major: W^T = S~ f^T), FP32-accurate
        CAXSI_PROF(p, "gemm_fwd_fp32emu", s);
        if (cublasGemmEx(T->blas, CUBLAS_OP_T, CUBLAS_OP_N, T->B, d.R, d.Q, &one, T->S, CUDA_R_32F, d.Q,
                         f, CUDA_R_32F, d.Q, &zero, T->tab, CUDA_R_32F, T->Bp,
                         CUBLAS_COMPUTE_32F_EMULATED_16BFX9, CUBLAS_GEMM_DEFAULT) != CUBLAS_STATUS_SUCCESS)
            return CAXSI_ERR_CUDA;
    } else {
        const int k = path == CAXSI_PATH_TABLE_BF16 ? 0 : 1;
        {
            CAXSI_PROF(p, "to_16bit", s);
            CAXSI_CUDA_TRY(pad_convert(f, d.R, d.Q, T->Qp, 1 + k, T->f16, nullptr, s));
        }
        CAXSI_LAUNCH_CHECK(p);
        CAXSI_PROF(p, k == 0 ? "gemm_fwd_bf16" : "gemm_fwd_fp16", s);
        if (cublasGemmEx(T->blas, CUBLAS_OP_T, CUBLAS_OP_N, T->B, d.R, d.Q, &one, T->S16[k], dtype16(path),
                         T->Qp, T->f16, dtype16(path), T->Qp, &zero, T->tab, CUDA_R_32F, T->Bp,
                         CUBLAS_COMPUTE_32F, CUBLAS_GEMM_DEFAULT) != CUBLAS_STATUS_SUCCESS)
            return CAXSI_ERR_CUDA;
    }
    int nparts = T->fwd_chunks;
    if (sym_fwd) {
        CAXSI_PROF(p, "sym_pairs_fwd", s);
        CAXSI_CUDA_TRY(sym_forward(p, T, T->fwd_part, s, path == CAXSI_PATH_TABLE_BF16 && p->gemm_engine == 0));
        nparts = T->sym.chunks;
    } else if (T->use_records) {
        CAXSI_PROF(p, "rec_pairs_fwd", s);
        CAXSI_CUDA_TRY(records_forward(p, T, subset, T->fwd_part, s));
        nparts = T->rec_chunks;
    } else {
        CAXSI_PROF(p, "tab_pairs_fwd", s);
        CAXSI_CUDA_TRY(dispatch_fwd(p, T, T->fwd_part, s));
    }
    CAXSI_LAUNCH_CHECK(p);
    const int64_t npix = (int64_t)d.M * d.N;
    {
        CAXSI_PROF(p, "sum_parts", s);
        CAXSI_CUDA_TRY(launch_sum_parts(T->fwd_part, nparts, npix, g_out, npix, s));
    }
    CAXSI_LAUNCH_CHECK(p);
    return CAXSI_OK;
}

caxsi_status table_adjoint(caxsi_plan *p, const float *w, float *f_out, int path, int subset, cudaStream_t s) {
    caxsi_status st = ensure_table(p, path);
    if (st != CAXSI_OK) return st;
    TablePath *T = p->table;
    if (subset >= 0) {   // the records grouped by the current partition (built on first use)
        if (!T->use_records) return CAXSI_ERR_UNSUPPORTED;
        if ((st = table_set_subsets(p)) != CAXSI_OK) return st;
        if (subset >= T->sub.P) return CAXSI_ERR_UNSUPPORTED;
        // FP32: V only at the subset's knots, contracted per record
        if (path == CAXSI_PATH_TABLE_FP32 && !p->no_sparse_subsets && sub_sparse_ok(p, w, f_out, 256)) {
            CAXSI_PROF(p, "sub_adj_sparse", s);
            CAXSI_CUDA_TRY(sub_adjoint_sparse(p, T, subset, w, f_out, s));
            return CAXSI_OK;
        }
    }
    const DevGeo &d = p->dg;
    const int out_kind = path == CAXSI_PATH_TABLE_FP32 ? 0 : (path == CAXSI_PATH_TABLE_BF16 ? 1 : 2);
    const bool tc = p->gemm_engine == 0 && T->use_records;
    if (T->use_records && subset < 0 && T->sym.adj.P > 0 && !p->no_symmetry) {
        CAXSI_PROF(p, "sym_pairs_adj", s);
        CAXSI_CUDA_TRY(sym_adjoint(p, T, w, out_kind, s));
    } else if (T->use_records) {
        CAXSI_PROF(p, "rec_pairs_adj", s);
        CAXSI_CUDA_TRY(records_adjoint(p, T, subset, w, out_kind, s));
    } else {
        CAXSI_PROF(p, "tab_pairs_adj", s);
        CAXSI_CUDA_TRY(dispatch_adj(p, T, w, s));
    }
    CAXSI_LAUNCH_CHECK(p);
    const float one = 1.f, zero = 0.f;
    HostPipe *pipe = p->pipe;
    // a host-buffer call with more than one wave of 128-row tiles: the first wave's
    // rows in their own launch, copied to the host while the rest are contracted
    const int64_t r1 = (int64_t)p->num_sms * 128;
    if (tc && out_kind == 0 && subset < 0 && pipe && r1 < d.R) {
        for (int h = 0; h < 2; ++h) {
            const int64_t r0 = h ? r1 : 0, nr = h ? d.R - r1 : r1;
            {
                CAXSI_PROF(p, "tc_gemm_adj_3xtf32", s);
                CAXSI_CUDA_TRY(tc_gemm(3, 128, (int)nr, d.Q, T->B, T->tab + r0 * T->Bp, nullptr, T->Bp, T->St_hi,
                                       T->St_lo, T->Bp, f_out + r0 * d.Q, d.Q, p->err_flag + 1, p->num_sms, s,
                                       nullptr, nband_of(p, 0), nullptr, 1));
            }
            CAXSI_LAUNCH_CHECK(p);
            if (h == 0) {
                CAXSI_CUDA_TRY(cudaEventRecord(pipe->out_half, s));
                CAXSI_CUDA_TRY(cudaStreamWaitEvent(pipe->cs, pipe->out_half, 0));
                CAXSI_CUDA_TRY(cudaMemcpyAsync(pipe->out_host, f_out, r1 * d.Q * sizeof(float),
                                               cudaMemcpyDeviceToHost, pipe->cs));
                pipe->out_from = r1;
            }
        }
        return CAXSI_OK;
    }
    if (tc) {
        // f[r][l] = sum_t V[r][t] S~^T[l][t] by the tcgen05 GEMM
        const int k = out_kind;
        CAXSI_PROF(p, k == 0 ? "tc_gemm_adj_3xtf32" : (k == 1 ? "tc_gemm_adj_bf16" : "tc_gemm_adj_fp16"), s);
        if (k == 0)
            CAXSI_CUDA_TRY(tc_gemm(3, 128, d.R, d.Q, T->B, T->tab, nullptr, T->Bp, T->St_hi, T->St_lo, T->Bp,
                                   f_out, d.Q, p->err_flag + 1, p->num_sms, s, nullptr, nband_of(p, 0), nullptr,
                                   1));
        else
            CAXSI_CUDA_TRY(tc_gemm(k, 128, d.R, d.Q, T->B, T->v16, nullptr, T->Bp, T->St16[k - 1], nullptr,
                                   T->Bp, f_out, d.Q, p->err_flag + 1, p->num_sms, s, nullptr, nband_of(p, 1),
                                   nullptr, 1));
        return CAXSI_OK;
    }
    if (cublasSetStream(T->blas, s) != CUBLAS_STATUS_SUCCESS) return CAXSI_ERR_CUDA;
    // f[r][l] = sum_t V[r][t] S~[t][l]  (column-major: f^T = S~^T V^T)
    if (out_kind == 0) {
        CAXSI_PROF(p, "gemm_adj_fp32emu", s);
        if (cublasGemmEx(T->blas, CUBLAS_OP_N, CUBLAS_OP_N, d.Q, d.R, T->B, &one, T->S, CUDA_R_32F, d.Q,
                         T->tab, CUDA_R_32F, T->Bp, &zero, f_out, CUDA_R_32F, d.Q,
                         CUBLAS_COMPUTE_32F_EMULATED_16BFX9, CUBLAS_GEMM_DEFAULT) != CUBLAS_STATUS_SUCCESS)
            return CAXSI_ERR_CUDA;
    } else {
        const int k = out_kind - 1;
        CAXSI_PROF(p, k == 0 ? "gemm_adj_bf16" : "gemm_adj_fp16", s);
        if (cublasGemmEx(T->blas, CUBLAS_OP_N, CUBLAS_OP_N, d.Q, d.R, T->B, &one, T->S16[k], dtype16(path),
                         T->Qp, T->v16, dtype16(path), T->Bp, &zero, f_out, CUDA_R_32F, d.Q,
                         CUBLAS_COMPUTE_32F, CUBLAS_GEMM_DEFAULT) != CUBLAS_STATUS_SUCCESS)
            return CAXSI_ERR_CUDA;
    }
    return CAXSI_OK;
}

caxsi_status table_forward_batch(caxsi_plan *p, int nb, const int32_t *ranges, const float *f, float *g_out,
                                 int path, cudaStream_t s) {
    if (path != CAXSI_PATH_TABLE_FP32 || p->gemm_engine != 0) return CAXSI_ERR_UNSUPPORTED;
    caxsi_status st = ensure_table(p, path);
    if (st != CAXSI_OK) return st;
    TablePath *T = p->table;
    if (!T->use_records) return CAXSI_ERR_UNSUPPORTED;
    if ((st = batch_layout(p, T, nb, ranges, s)) != CAXSI_OK) return st;
    BatchState &bs = T->batch;
    const DevGeo &d = p->dg;
    const int64_t npix = (int64_t)d.M * d.N;
    if (bs.rows > 0) {
        {
            CAXSI_PROF(p, "pack_rows", s);
            k_pack_rows<<<(unsigned)ceil_div64(bs.rows * T->Qp, 256), 256, 0, s>>>(f, bs.rowmap, bs.rows, d.Q,
                                                                                 T->Qp, bs.f_hi);
        }
        CAXSI_LAUNCH_CHECK(p);
        {
            CAXSI_PROF(p, "tc_gemm_fwd_3xtf32", s);
            CAXSI_CUDA_TRY(tc_gemm(4, 256, bs.rows, T->B, d.Q, bs.f_hi, nullptr, T->Qp, T->S_hi, T->S_lo, T->Qp,
                                   bs.tab, T->Bp, p->err_flag + 1, p->num_sms, s, kband_of(p, 0), nullptr, nullptr,
                                   1));
        }
        CAXSI_LAUNCH_CHECK(p);
        {
            CAXSI_PROF(p, "rec_pairs_fwd", s);
            CAXSI_CUDA_TRY(records_forward_items(p, T, bs.items, bs.n_items, bs.tab, bs.part, s));
        }
        CAXSI_LAUNCH_CHECK(p);
    }
    {
        CAXSI_PROF(p, "sum_parts", s);
        k_sum_parts_batch<<<dim3((unsigned)ceil_div64(npix, 256), (unsigned)nb), 256, 0, s>>>(bs.part, bs.obj_items,
                                                                                          npix, g_out);
    }
    CAXSI_LAUNCH_CHECK(p);
    return CAXSI_OK;
}

caxsi_status table_adjoint_batch(caxsi_plan *p, int nb, const int32_t *ranges, const float *w, float *f_out,
                                 int path, cudaStream_t s) {
    if (path != CAXSI_PATH_TABLE_FP32 || p->gemm_engine != 0) return CAXSI_ERR_UNSUPPORTED;
    caxsi_status st = ensure_table(p, path);
    if (st != CAXSI_OK) return st;
    TablePath *T = p->table;
    if (!T->use_records) return CAXSI_ERR_UNSUPPORTED;
    if ((st = batch_layout(p, T, nb, ranges, s)) != CAXSI_OK) return st;
    BatchState &bs = T->batch;
    const DevGeo &d = p->dg;
    const int64_t nf = (int64_t)d.R * d.Q;
    CAXSI_CUDA_TRY(cudaMemsetAsync(f_out, 0, (size_t)nb * nf * sizeof(float), s));
    if (bs.rows == 0) return CAXSI_OK;
    {
        CAXSI_PROF(p, "rec_pairs_adj", s);
        CAXSI_CUDA_TRY(records_adjoint_items(p, T, bs.items, bs.n_items, w, (int64_t)d.M * d.N, bs.tab, s));
    }
    CAXSI_LAUNCH_CHECK(p);
    {
        CAXSI_PROF(p, "tc_gemm_adj_3xtf32", s);
        CAXSI_CUDA_TRY(tc_gemm(3, 128, bs.rows, d.Q, T->B, bs.tab, nullptr, T->Bp, T->St_hi, T->St_lo, T->Bp,
                               bs.fpk, d.Q, p->err_flag + 1, p->num_sms, s, nullptr, nband_of(p, 0), nullptr, 1));
    }
    CAXSI_LAUNCH_CHECK(p);
    {
        CAXSI_PROF(p, "unpack_rows", s);
        k_unpack_rows<<<(unsigned)ceil_div64(bs.rows * d.Q, 256), 256, 0, s>>>(bs.fpk, bs.rowmap, bs.rows, d.Q,
                                                                            f_out);
    }
    CAXSI_LAUNCH_CHECK(p);
    return CAXSI_OK;
}

caxsi_status table_set_subsets(caxsi_plan *p) {
    caxsi_status st = ensure_table(p, CAXSI_PATH_TABLE_FP32);
    if (st != CAXSI_OK) return st;
    if (p->table->sub_gen == p->sub_gen) return CAXSI_OK;
    st = records_build_subsets(p, p->table, p->n_subsets, p->sub_host.data());
    if (st == CAXSI_OK) {
        CAXSI_CUDA_TRY(cudaDeviceSynchronize());
        p->table->sub_gen = p->sub_gen;
    }
    return st;
}

void table_destroy(caxsi_plan *p) {
    free_table(p->table);
    p->table = nullptr;
}
