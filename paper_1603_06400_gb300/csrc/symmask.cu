// Direct forward and adjoint for a mirror-symmetric secondary mask, with the mask
// factor computed online (Sec. III-A mirror symmetries, Sec. III-C online/offline
// trade-off, Algorithm 2's four-quadrant structure).
//
// When the mask is symmetric about the central ray in y and in z (and J, M, N are
// even), the pair (v, m, n), its up-down image (v, M-1-m, n), its left-right image
// (v', m, N-1-n) with v' = (i, J-1-j), and the image under both share the scatter
// angle, G_so, G_od, dtheta AND the mask factor T; only the left-right images read
// another object column (f at v' instead of v).  So:
//   forward: per voxel pair (v, v') (v in the left half, j < J/2) and upper-half
//     pixel (m < M/2, any n): the geometry and T once, the energy sum W for f[v]
//     and for f[v'] (the paper's W_L, W_R); c W_v goes to (m, n) and (M-1-m, n),
//     c W_v' to (m, N-1-n) and (M-1-m, N-1-n) -- a quarter of the geometry and
//     half of the energy sums of the plain kernel;
//   adjoint: per voxel and upper-half pixel (m, n): the geometry and T once, one
//     energy scatter of c (w[m][n] + w[M-1-m][n]) -- half of the plain kernel's.
// T is not read from the precomputed per-pair bits: each block (warp) computes the
// mask cells its rays cross for its staged voxels and its detector rows and
// columns -- in FP32, and with the plan builder's FP64 formula where the FP32
// estimate lies next to a cell edge (maskgeo.cuh), so the decision is the plan's
// -- and looks the cell up in the mask array (rows x cols bytes, L1-resident).  The
// per-pair bit table is then not needed by these kernels.
#include <algorithm>

#include "direct_body.cuh"
#include "maskgeo.cuh"

namespace {

using namespace direct_impl;

constexpr int SVS = 16;   // voxel pairs staged per shared-memory round (forward)

struct SymTables {
    Tables T;
    PlanGeo64 g64;
    MaskGeo32 g32;
    const uint8_t *mask;   // [rows][cols], 0 / 1
};

// Block: 8 warps over 8 upper-half rows (m < M/2) and 16 mirrored column pairs:
// lane l < 16 takes column n = 16 tn + l, lane l + 16 its mirror N-1-n; voxel
// pairs [by pc, (by + 1) pc) of the X * J/2 pairs p = i (J/2) + j, v = i J + j,
// v' = i J + J-1-j.  Lane l accumulates c W_v (its own column, from v) and c W_v'
// (the mirror column, from v'); a pixel's sum is its lane's first plus its mirror
// lane's second.  Writes each pixel and its up-down image in partial image by.
__global__ void __launch_bounds__(FWD_THREADS)
k_fwd_direct_symmask(SymTables S, const float *__restrict__ f, float *__restrict__ part, int pc, int tiles_n) {
    extern __shared__ __align__(16) unsigned char smem_raw[];
    const Tables &T = S.T;
    const DevGeo &g = T.g;
    const int QP = g.Q + 2;
    const int Mh = g.M / 2, Nh = g.N / 2, Jh = g.J / 2;
    float2 *s_en = reinterpret_cast<float2 *>(smem_raw);
    float4 *s_vox = reinterpret_cast<float4 *>(s_en + ((g.K + 1) & ~1));
    float2 *s_f = reinterpret_cast<float2 *>(s_vox + SVS);            // [2 SVS][QP]
    int *s_row = reinterpret_cast<int *>(s_f + 2 * SVS * QP);         // [SVS][FWD_WARPS]
    int *s_col = s_row + SVS * FWD_WARPS;                             // [SVS][32]
    float *s_acc = reinterpret_cast<float *>(s_col + SVS * 32);       // [FWD_WARPS][2][32]
    int *s_q = reinterpret_cast<int *>(s_acc + FWD_WARPS * 64);       // [FWD_WARPS][64] ring

    const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
    const int tm = blockIdx.x / tiles_n, tn = blockIdx.x % tiles_n;
    const int c16 = tn * 16 + (lane & 15);          // left-half column of the lane's pair
    const int m = tm * FWD_WARPS + warp, n = lane < 16 ? c16 : g.N - 1 - c16;
    const bool valid = m < Mh && c16 < Nh;
    const int R2 = g.X * Jh;
    const int p0 = blockIdx.y * pc, p1 = min(p0 + pc, R2);

    for (int k = tid; k < g.K; k += FWD_THREADS) s_en[k] = T.energy[k];
    const float Npix = (float)n - g.cN;
    const float sz = valid ? T.zrow[m] : 0.f;
    // per lane: the sums for its own column (from v) and for its mirror column (from v')
    float *accL = s_acc + warp * 64, *accR = accL + 32;
    int *q = s_q + warp * 64;
    accL[lane] = 0.f;
    accR[lane] = 0.f;
    const unsigned lt = (1u << lane) - 1u;

    for (int pb = p0; pb < p1; pb += SVS) {
        const int nv = min(SVS, p1 - pb);
        __syncthreads();
        for (int idx = tid; idx < 2 * nv * QP; idx += FWD_THREADS) {
            const int r = idx / QP, lp = idx - r * QP;
            const int pp = pb + (r >> 1), i = pp / Jh, j = pp - i * Jh;
            const int v = i * g.J + ((r & 1) ? g.J - 1 - j : j);
            const float *row = f + (int64_t)v * g.Q;
            const float F0 = (lp >= 1 && lp <= g.Q) ? row[lp - 1] : 0.f;
            const float F1 = (lp + 1 <= g.Q) ? row[lp] : 0.f;
            s_f[idx] = make_float2(F0, F1 - F0);
        }
        for (int idx = tid; idx < nv * (FWD_WARPS + 32); idx += FWD_THREADS) {
            const int vv = idx / (FWD_WARPS + 32), k = idx - vv * (FWD_WARPS + 32);
            const int pp = pb + vv, i = pp / Jh, j = pp - i * Jh;
            if (k < FWD_WARPS) {
                const int mm = tm * FWD_WARPS + k;
                s_row[vv * FWD_WARPS + k] = mm < Mh ? mask_row_fast(S.g64, S.g32, i, mm) : -1;
            } else {
                const int l = k - FWD_WARPS, cc = tn * 16 + (l & 15);
                s_col[vv * 32 + l] = cc < Nh ? mask_col_fast(S.g64, S.g32, i, j, l < 16 ? cc : g.N - 1 - cc) : -1;
            }
        }
        if (tid < nv) {
            const int pp = pb + tid, i = pp / Jh, j = pp - i * Jh;
            s_vox[tid] = T.vox[i * g.J + j];
        }
        __syncthreads();
        // pair (staged voxel pair vv, pixel of lane pl), or none (entry < 0): the two
        // energy sums, added to lane pl's accumulators; a lane's pairs within one
        // batch are applied in rounds by their order in the queue (ascending vv)
        auto take = [&](int entry) {
            const int pl = entry >= 0 ? (entry & 31) : lane;
            const int pn = __shfl_sync(0xffffffffu, n, pl);
            const float pN = __shfl_sync(0xffffffffu, Npix, pl), pz = __shfl_sync(0xffffffffu, sz, pl);
            float c = 0.f, wl = 0.f, wr = 0.f;
            if (entry >= 0) {
                const int vv = entry >> 5;
                const int pp = pb + vv, i = pp / Jh, j = pp - i * Jh;
                const float4 vx = s_vox[vv];
                float u, ang;
                pair_u_angular(vx.x, vx.y, vx.w, pN, pz, g.p_y, g.Xd, u, ang);
                const float gd = T.god[((int64_t)i * g.M + m) * g.ND + (pn - g.rho_y * j - g.d_min)];
                const float2 *fl = s_f + (2 * vv) * QP, *fr = fl + QP;
                int k0, k1;
                energy_range(g, u, k0, k1);
#pragma unroll 4
                for (int k = k0; k < k1; ++k) {
                    const float2 ak = s_en[k];
                    float tau = fmaf(ak.x, u, -g.b);
                    tau = fminf(fmaxf(tau, -1.f), g.Qf);
                    const float flo = floorf(tau);
                    const float al = tau - flo;
                    const int b = (int)flo + 1;
                    const float2 A = fl[b], B = fr[b];
                    wl = fmaf(ak.y, fmaf(al, A.y, A.x), wl);
                    wr = fmaf(ak.y, fmaf(al, B.y, B.x), wr);
                }
                c = vx.z * gd * ang;
            }
            const unsigned same = __match_any_sync(0xffffffffu, entry >= 0 ? pl : 32 + lane);
            const int rank = __popc(same & lt);
            const int rounds = (int)__reduce_max_sync(0xffffffffu, entry >= 0 ? (unsigned)rank + 1u : 0u);
            for (int r = 0; r < rounds; ++r) {   // warp-uniform
                if (entry >= 0 && rank == r) {
                    accL[pl] = fmaf(c, wl, accL[pl]);
                    accR[pl] = fmaf(c, wr, accR[pl]);
                }
                __syncwarp();
            }
        };
        // the open pairs of the warp's lanes, voxel pair by voxel pair (the mask cell
        // of each from the staged rows and columns)
        int head = 0, cnt = 0;
        for (int vv = 0; vv < nv; ++vv) {
            bool ok = false;
            if (valid) {
                const int row = s_row[vv * FWD_WARPS + warp], col = s_col[vv * 32 + lane];
                ok = row >= 0 && col >= 0 && S.mask[row * S.g64.cols + col];
            }
            const unsigned bal = __ballot_sync(0xffffffffu, ok);
            if (ok) q[(head + cnt + __popc(bal & lt)) & 63] = (vv << 5) | lane;
            cnt += __popc(bal);
            __syncwarp();
            if (cnt >= 32) {   // warp-uniform
                const int entry = q[(head + lane) & 63];
                head = (head + 32) & 63;
                cnt -= 32;
                __syncwarp();   // the batch is read before later pairs refill its slots
                take(entry);
            }
        }
        if (cnt > 0) {   // the rest, before the next stage replaces the staged pairs
            const int entry = lane < cnt ? q[(head + lane) & 63] : -1;
            __syncwarp();
            take(entry);
        }
    }
    __syncwarp();
    const float myL = accL[lane], myR = accR[lane];
    // the mirror column's contributions from the right-half voxels are the mirror lane's
    const float sum = myL + __shfl_xor_sync(0xffffffffu, myR, 16);
    if (valid) {
        float *dst = part + (int64_t)blockIdx.y * g.M * g.N;
        dst[(int64_t)m * g.N + n] = sum;
        dst[(int64_t)(g.M - 1 - m) * g.N + n] = sum;
    }
}

// Warp per (voxel, range of upper-half rows); lane-private q rows as in the plain
// adjoint, the voxel's mask columns for every detector column cached in the
// warp's shared-memory slice, the open pairs queued and taken 32 at a time as in
// the plain adjoint.  Shared memory per warp: [(Q+3) x 32] floats, then [N] ints,
// then a ring of 64 ints.
__global__ void __launch_bounds__(ADJ_WARPS * 32)
k_adj_direct_symmask(SymTables S, const float *__restrict__ w, float *__restrict__ out, int split,
                     int rows_per_split) {
    extern __shared__ __align__(16) unsigned char smem_raw[];
    const Tables &T = S.T;
    const DevGeo &g = T.g;
    const int QB = g.Q + 3;
    const int Mh = g.M / 2;
    float2 *s_en = reinterpret_cast<float2 *>(smem_raw);
    float *s_warp = reinterpret_cast<float *>(s_en + ((g.K + 1) & ~1));
    const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
    float *acc = s_warp + (int64_t)warp * (QB * 32 + g.N + 64);
    int *colc = reinterpret_cast<int *>(acc + QB * 32);
    int *ring = colc + g.N;   // [64] queued open pairs (m N + n)
    const int item = blockIdx.x * ADJ_WARPS + warp;
    const int v = item / split, sp = item - (item / split) * split;
    for (int k = tid; k < g.K; k += blockDim.x) s_en[k] = T.energy[k];
    for (int b = lane; b < QB * 32; b += 32) acc[b] = 0.f;
    __syncthreads();
    if (v >= g.R) return;
    const int i = v / g.J, j = v - i * g.J;
    for (int nn = lane; nn < g.N; nn += 32) colc[nn] = mask_col_fast(S.g64, S.g32, i, j, nn);
    __syncwarp();
    const float4 vx = T.vox[v];
    float *my = acc + lane;
    const int m0 = sp * rows_per_split, m1 = min(Mh, m0 + rows_per_split);
    // one open pair (upper-half pixel m, n; the up-down pair's weights added)
    auto take = [&](int p) {
        const int m = p / g.N, n = p - m * g.N;
        const float wv = w[p] + w[(int64_t)(g.M - 1 - m) * g.N + n];
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
    // the open pairs with a nonzero weight queued in pixel order, taken 32 at a time
    const unsigned lt = (1u << lane) - 1u;
    int head = 0, cnt = 0;
    for (int m = m0; m < m1; ++m) {
        const int row = mask_row_fast(S.g64, S.g32, i, m);
        if (row < 0) continue;   // warp-uniform
        const uint8_t *mrow = S.mask + row * S.g64.cols;
        const float *wa = w + (int64_t)m * g.N, *wb = w + (int64_t)(g.M - 1 - m) * g.N;
        for (int nb = 0; nb < g.N; nb += 32) {
            const int n = nb + lane;
            bool ok = false;
            if (n < g.N) {
                const int col = colc[n];
                ok = col >= 0 && mrow[col] && wa[n] + wb[n] != 0.f;
            }
            const unsigned bal = __ballot_sync(0xffffffffu, ok);
            if (ok) ring[(head + cnt + __popc(bal & lt)) & 63] = m * g.N + n;
            cnt += __popc(bal);
            __syncwarp();
            if (cnt >= 32) {
                const int p = ring[(head + lane) & 63];
                head = (head + 32) & 63;
                cnt -= 32;
                __syncwarp();
                take(p);
            }
        }
    }
    if (cnt > 0) {
        const int p = lane < cnt ? ring[(head + lane) & 63] : -1;
        __syncwarp();
        if (p >= 0) take(p);
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

SymTables sym_tables(const caxsi_plan *p) {
    SymTables S;
    S.T = tables_of(p);
    S.g64 = plan_geo64(p);
    S.g32 = mask_geo32(S.g64);
    S.mask = p->mask01;
    return S;
}

}  // namespace

cudaError_t launch_sum_parts(const float *part, int nparts, int64_t stride, float *out, int64_t n, cudaStream_t s);

size_t symmask_fwd_smem(const DevGeo &g) {
    return ((g.K + 1) & ~1) * sizeof(float2) + SVS * sizeof(float4) + (size_t)2 * SVS * (g.Q + 2) * sizeof(float2) +
           (size_t)SVS * (FWD_WARPS + 32) * sizeof(int) + (size_t)FWD_WARPS * 64 * sizeof(float) +
           (size_t)FWD_WARPS * 64 * sizeof(int);
}
size_t symmask_adj_smem(const DevGeo &g) {
    return ((g.K + 1) & ~1) * sizeof(float2) + (size_t)ADJ_WARPS * ((g.Q + 3) * 32 + g.N + 64) * sizeof(float);
}

caxsi_status symmask_forward(caxsi_plan *p, const float *f, float *g_out, cudaStream_t s) {
    const DevGeo &g = p->dg;
    const int Mh = g.M / 2, Nh = g.N / 2, R2 = g.X * (g.J / 2);
    const int tiles_n = (int)ceil_div64(Nh, 16);
    const int tiles = (int)ceil_div64(Mh, FWD_WARPS) * tiles_n;
    // chunks of voxel pairs: about 16 blocks per SM, at most the plan's partial images
    int chunks = (int)std::min<int64_t>(ceil_div64(16 * p->num_sms, tiles), p->fwd_chunks);
    if (chunks > R2) chunks = R2;
    int pc = (int)ceil_div64(R2, chunks);
    if (pc < 8) pc = 8;
    chunks = (int)ceil_div64(R2, pc);
    const size_t sm = symmask_fwd_smem(g);
    CAXSI_CUDA_TRY(cudaFuncSetAttribute(k_fwd_direct_symmask, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm));
    {
        CAXSI_PROF(p, "fwd_direct_symmask", s);
        k_fwd_direct_symmask<<<dim3(tiles, chunks), FWD_THREADS, sm, s>>>(sym_tables(p), f, p->fwd_part, pc, tiles_n);
    }
    CAXSI_LAUNCH_CHECK(p);
    const int64_t npix = (int64_t)g.M * g.N;
    {
        CAXSI_PROF(p, "sum_parts", s);
        CAXSI_CUDA_TRY(launch_sum_parts(p->fwd_part, chunks, npix, g_out, npix, s));
    }
    CAXSI_LAUNCH_CHECK(p);
    return CAXSI_OK;
}

caxsi_status symmask_adjoint(caxsi_plan *p, const float *w, float *f_out, cudaStream_t s) {
    const DevGeo &g = p->dg;
    const int Mh = g.M / 2;
    // the upper-half rows split like the plain adjoint's rows, into at most its partials
    int split = std::min(p->adj_split, Mh);
    const int rps = (int)ceil_div64(Mh, split);
    split = (int)ceil_div64(Mh, rps);
    const size_t sm = symmask_adj_smem(g);
    CAXSI_CUDA_TRY(cudaFuncSetAttribute(k_adj_direct_symmask, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm));
    const int64_t items = (int64_t)g.R * split;
    float *dst = split > 1 ? p->adj_part : f_out;
    {
        CAXSI_PROF(p, "adj_direct_symmask", s);
        k_adj_direct_symmask<<<(unsigned)ceil_div64(items, ADJ_WARPS), ADJ_WARPS * 32, sm, s>>>(sym_tables(p), w, dst,
                                                                                                 split, rps);
    }
    CAXSI_LAUNCH_CHECK(p);
    if (split > 1) {
        const int64_t nf = (int64_t)g.R * g.Q;
        {
            CAXSI_PROF(p, "sum_parts", s);
            CAXSI_CUDA_TRY(launch_sum_parts(p->adj_part, split, nf, f_out, nf, s));
        }
        CAXSI_LAUNCH_CHECK(p);
    }
    return CAXSI_OK;
}
