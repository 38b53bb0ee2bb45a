// Per-pair work of the direct (matrix-free, FP32) forward and adjoint, shared
// by the single-plan kernels (direct.cu) and the persistent multi-object kernels
// (multi.cu), so that both evaluate every object with the same arithmetic in
// the same order.  See direct.cu for the structure of the two operators.
#pragma once

#include "internal.cuh"
#include "pairgeo.cuh"

namespace direct_impl {

constexpr int FWD_WARPS = 8;
constexpr int FWD_THREADS = FWD_WARPS * 32;
constexpr int FWD_VS = 32;  // voxels staged per shared-memory round
constexpr int ADJ_WARPS = 4;

// The energies whose term can be nonzero for a pair with u = sin(theta/2):
// tau_k = a_k u - b rises with k (a_k = a0 + k da), and a term is an exact zero
// unless -1 < tau_k < Q (outside, the interpolation reads the zero padding of the
// staged q row, or the adjoint scatters into its discarded padding rows).  The
// range [k0, k1) is widened by two energies at each end against rounding; a
// u of 0 or a non-finite bound gives the whole range or none, as the terms do.
__device__ __forceinline__ void energy_range(const DevGeo &g, float u, int &k0, int &k1) {
    const float lo = ((g.b - 1.f) / u - g.a0) / g.da, hi = ((g.Qf + g.b) / u - g.a0) / g.da;
    k0 = lo > 2.f ? (lo < (float)g.K ? (int)lo - 2 : g.K) : 0;
    k1 = hi < (float)g.K - 3.f ? max(0, (int)fmaxf(hi, -8.f) + 3) : g.K;
}

struct Tables {
    DevGeo g;
    const float4 *vox;
    const float *zrow;
    const float *god;
    const uint32_t *tbits;
    const float2 *energy;
};


// One block's work of the forward: detector tile bx (or listed pixels bx * 256 ..)
// and voxel chunk by, written to partial image by.  Shared by the single-plan
// kernel (bx, by = the block index) and the persistent multi-object kernel.
//
// Lane l of a warp owns one pixel; the block stages FWD_VS voxels (their q rows
// and positions) at a time.  A warp queues the open pairs of its 32 pixels with
// the staged voxels, voxel by voxel, in a ring of 64 slots and takes them 32 at a
// time, one per lane, so that no lane idles on a closed pair (about half are
// closed by the mask).  A pair's contribution goes to its pixel's accumulator in
// shared memory; the pairs of one pixel within a batch are applied in rounds by
// their rank in the queue, so that every pixel adds its open voxels' terms in
// ascending voxel order, one fma each: the result is that of a plain loop over
// the voxels.
template <bool LIST>
__device__ __forceinline__ void fwd_direct_body(const Tables &T, const float *__restrict__ f,
                                                float *__restrict__ part, int vc, int tiles_n,
                                                const int *__restrict__ list, int np, int bx, int by,
                                                unsigned char *smem_raw) {
    const DevGeo &g = T.g;
    const int QP = g.Q + 2;
    float2 *s_en = reinterpret_cast<float2 *>(smem_raw);
    float4 *s_vox = reinterpret_cast<float4 *>(s_en + ((g.K + 1) & ~1));
    float2 *s_f = reinterpret_cast<float2 *>(s_vox + FWD_VS);
    float *s_acc = reinterpret_cast<float *>(s_f + (size_t)FWD_VS * QP);   // [FWD_WARPS][32] per pixel
    int *s_q = reinterpret_cast<int *>(s_acc + FWD_THREADS);              // [FWD_WARPS][64] ring

    const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
    int m, n, e = 0;
    bool valid;
    if (LIST) {   // listed pixel e
        e = bx * FWD_THREADS + tid;
        valid = e < np;
        const int p = valid ? list[e] : 0;
        m = p / g.N;
        n = p - m * g.N;
    } else {      // 8 x 32 tile of the detector
        const int tm = bx / tiles_n, tn = bx % tiles_n;
        m = tm * FWD_WARPS + warp;
        n = tn * 32 + lane;
        valid = (m < g.M) && (n < g.N);
    }
    const int v0 = by * vc;
    const int v1 = min(v0 + vc, g.R);

    for (int k = tid; k < g.K; k += FWD_THREADS) s_en[k] = T.energy[k];
    const float Npix = (float)n - g.cN;
    const float sz = valid ? T.zrow[m] : 0.f;
    const int wsel = n >> 5, bsel = n & 31;
    float *acc = s_acc + warp * 32;
    int *q = s_q + warp * 64;
    acc[lane] = 0.f;
    const unsigned lt = (1u << lane) - 1u;

    for (int vb = v0; vb < v1; vb += FWD_VS) {
        const int nv = min(FWD_VS, v1 - vb);
        __syncthreads();
        for (int idx = tid; idx < nv * QP; idx += FWD_THREADS) {
            const int vv = idx / QP, lp = idx - vv * QP;
            const float *row = f + (int64_t)(vb + vv) * g.Q;
            const float F0 = (lp >= 1 && lp <= g.Q) ? row[lp - 1] : 0.f;
            const float F1 = (lp + 1 <= g.Q) ? row[lp] : 0.f;
            s_f[idx] = make_float2(F0, F1 - F0);
        }
        if (tid < nv) s_vox[tid] = T.vox[vb + tid];
        __syncthreads();
        // pair (staged voxel vv, pixel of lane pl), or none (entry < 0): its term,
        // added to the pixel's accumulator; a pixel's pairs in one batch are applied
        // in rounds by their order in the queue (ascending voxel)
        auto take = [&](int entry) {
            const int pl = entry >= 0 ? (entry & 31) : lane;
            const int pm = __shfl_sync(0xffffffffu, m, pl), pn = __shfl_sync(0xffffffffu, n, pl);
            const float pN = __shfl_sync(0xffffffffu, Npix, pl), pz = __shfl_sync(0xffffffffu, sz, pl);
            float c = 0.f, e_acc = 0.f;
            if (entry >= 0) {
                const int vv = entry >> 5, v = vb + vv;
                const int i = v / g.J, j = v - i * g.J;
                const float4 vx = s_vox[vv];
                float u, ang;
                pair_u_angular(vx.x, vx.y, vx.w, pN, pz, g.p_y, g.Xd, u, ang);
                const float gd = T.god[((int64_t)i * g.M + pm) * g.ND + (pn - g.rho_y * j - g.d_min)];
                const float2 *fr = s_f + vv * QP;
                int k0, k1;
                energy_range(g, u, k0, k1);
#pragma unroll 8
                for (int k = k0; k < k1; ++k) {
                    const float2 ak = s_en[k];
                    float tau = fmaf(ak.x, u, -g.b);
                    tau = fminf(fmaxf(tau, -1.f), g.Qf);
                    const float fl = floorf(tau);
                    const float al = tau - fl;
                    const float2 F = fr[(int)fl + 1];
                    e_acc = fmaf(ak.y, fmaf(al, F.y, F.x), e_acc);
                }
                c = vx.z * gd * ang;
            }
            const unsigned same = __match_any_sync(0xffffffffu, entry >= 0 ? pl : 32 + lane);
            const int rank = __popc(same & lt);
            const int rounds = (int)__reduce_max_sync(0xffffffffu, entry >= 0 ? (unsigned)rank + 1u : 0u);
            for (int r = 0; r < rounds; ++r) {   // warp-uniform
                if (entry >= 0 && rank == r) acc[pl] = fmaf(c, e_acc, acc[pl]);
                __syncwarp();
            }
        };
        // the open pairs of the warp's pixels, voxel by voxel (lanes in pixel order)
        int head = 0, cnt = 0;
        for (int vv = 0; vv < nv; ++vv) {
            bool ok = false;
            if (valid) {
                const uint32_t word = T.tbits[((int64_t)(vb + vv) * g.M + m) * g.Nw + wsel];
                ok = ((word >> bsel) & 1u) != 0u;
            }
            const unsigned bal = __ballot_sync(0xffffffffu, ok);
            if (ok) q[(head + cnt + __popc(bal & lt)) & 63] = (vv << 5) | lane;
            cnt += __popc(bal);
            __syncwarp();
            if (cnt >= 32) {   // warp-uniform
                const int entry = q[(head + lane) & 63];
                head = (head + 32) & 63;
                cnt -= 32;
                __syncwarp();   // the batch is read before later voxels refill its slots
                take(entry);
            }
        }
        if (cnt > 0) {   // the rest, before the next stage replaces the staged voxels
            const int entry = lane < cnt ? q[(head + lane) & 63] : -1;
            __syncwarp();
            take(entry);
        }
    }
    __syncwarp();
    if (valid) {
        const float total = acc[lane];
        if (LIST) part[(int64_t)by * np + e] = total;
        else part[(int64_t)by * g.M * g.N + (int64_t)m * g.N + n] = total;
    }
}

// One warp's work of the adjoint: voxel v, detector rows of split part sp (or the
// listed pixels), into the warp's lane-private rows acc ([Q+3][32], zeroed by the
// caller), written to out + (sp R + v) Q.  Shared by the single-plan kernel and
// the persistent multi-object kernel.
template <bool LIST>
__device__ __forceinline__ void adj_direct_body(const Tables &T, const float *__restrict__ w,
                                                float *__restrict__ out, int rows_per_split,
                                                const int *__restrict__ list, int np, int v, int sp,
                                                const float2 *s_en, float *acc, int lane) {
    const DevGeo &g = T.g;
    const int i = v / g.J, j = v - i * g.J;
    const float4 vx = T.vox[v];
    float *my = acc + lane;
    // one open pair (pixel (m, n), weight wv != 0) scattered into the lane's q row
    auto pair_open = [&](int m, int n, float wv) {
        float u, ang;
        pair_u_angular(vx.x, vx.y, vx.w, (float)n - g.cN, T.zrow[m], g.p_y, g.Xd, u, ang);
        const float base = vx.z * T.god[((int64_t)i * g.M + m) * g.ND + (n - g.rho_y * j - g.d_min)] * ang * wv;
        int k0, k1;
        energy_range(g, u, k0, k1);
#pragma unroll 4
        for (int k = k0; k < k1; ++k) {
            const float2 ak = s_en[k];
            float tau = fmaf(ak.x, u, -g.b);
            tau = fminf(fmaxf(tau, -1.f), g.Qf);
            const float fl = floorf(tau);
            const float al = tau - fl;
            const int lp = (int)fl + 1;
            const float cb = ak.y * base;
            const float hi = cb * al;
            my[lp * 32] += cb - hi;
            my[(lp + 1) * 32] += hi;
        }
    };
    auto is_open = [&](int m, int n) {
        const uint32_t word = T.tbits[((int64_t)v * g.M + m) * g.Nw + (n >> 5)];
        return ((word >> (n & 31)) & 1u) != 0u;
    };
    if (LIST) {
        for (int e = lane; e < np; e += 32) {
            const int p = list[e];
            const int m = p / g.N, n = p - m * g.N;
            const float wv = w[p];
            if (is_open(m, n) && wv != 0.f) pair_open(m, n, wv);
        }
    } else {
        // The open pairs with a nonzero weight are queued in pixel order in a ring of
        // 64 slots after the warp's q rows and taken 32 at a time, one per lane, so
        // the lanes of a batch all do work (about half the pairs are closed by the
        // mask).  The assignment of pairs to lanes is fixed by the pixel order.
        int *q = reinterpret_cast<int *>(acc + (g.Q + 3) * 32);
        const unsigned lt = (1u << lane) - 1u;
        int head = 0, cnt = 0;
        auto take = [&](int p) {
            const int m = p / g.N;
            pair_open(m, p - m * g.N, w[p]);
        };
        const int m0 = sp * rows_per_split, m1 = min(g.M, m0 + rows_per_split);
        for (int m = m0; m < m1; ++m)
            for (int nb = 0; nb < g.N; nb += 32) {
                const int n = nb + lane;
                const bool ok = n < g.N && is_open(m, n) && w[(int64_t)m * g.N + n] != 0.f;
                const unsigned bal = __ballot_sync(0xffffffffu, ok);
                if (ok) q[(head + cnt + __popc(bal & lt)) & 63] = m * g.N + n;
                cnt += __popc(bal);
                __syncwarp();
                if (cnt >= 32) {   // warp-uniform
                    const int p = q[(head + lane) & 63];
                    head = (head + 32) & 63;
                    cnt -= 32;
                    __syncwarp();   // the batch is read before later groups refill its slots
                    take(p);
                }
            }
        if (cnt > 0) {
            const int p = lane < cnt ? q[(head + lane) & 63] : -1;
            __syncwarp();
            if (p >= 0) take(p);
        }
    }
    __syncwarp();
    float *dst = out + ((int64_t)sp * g.R + v) * g.Q;
    for (int lp = 1 + lane; lp <= g.Q; lp += 32) {
        const float *rowp = acc + lp * 32;
        float s = 0.f;
        for (int c = 0; c < 32; ++c) s += rowp[(lane + c) & 31];
        dst[lp - 1] = s;
    }
}

inline Tables tables_of(const caxsi_plan *p) {
    Tables T;
    T.g = p->dg;
    T.vox = p->vox;
    T.zrow = p->zrow;
    T.god = p->god;
    T.tbits = p->tbits;
    T.energy = p->energy;
    return T;
}

// energies, staged voxels and q rows, per-pixel accumulators, per-warp rings of 64 pairs
inline size_t fwd_smem(const DevGeo &g) {
    return ((g.K + 1) & ~1) * sizeof(float2) + FWD_VS * sizeof(float4) +
           (size_t)FWD_VS * (g.Q + 2) * sizeof(float2) + FWD_THREADS * sizeof(float) + FWD_WARPS * 64 * sizeof(int);
}
// per warp: q rows [(Q + 3) x 32] floats and a ring of 64 queued pixels
__host__ __device__ inline size_t adj_warp_floats(int Q) { return (size_t)(Q + 3) * 32 + 64; }
inline size_t adj_smem(const DevGeo &g) {
    return ((g.K + 1) & ~1) * sizeof(float2) + (size_t)ADJ_WARPS * adj_warp_floats(g.Q) * sizeof(float);
}

}  // namespace direct_impl
