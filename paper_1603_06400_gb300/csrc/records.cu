// Pair records for the table paths.
//
// The per-pair part of the table paths depends only on the geometry: for every
// open (voxel, pixel) pair, the knot interval t of its u = sin(theta/2), and
// the weights w0 = c (1 - alpha), w1 = c alpha with c = C G_so G_od T dtheta
// (1 + cos^2 theta) cos(theta/2) and alpha the interpolation position in the
// interval.  They are computed once per plan (the paper's online/offline
// trade-off, Sec. III-C, with HBM-resident storage) and streamed by every
// forward and adjoint:
//
//   forward:  g[pix] += w0 Wtab[v][t] + w1 Wtab[v][t+1]
//   adjoint:  V[v][t] += w0 w[pix],  V[v][t+1] += w1 w[pix]
//
// Records are voxel-major and sorted by (t, pixel) inside each voxel (a stable
// counting sort, one warp per voxel, deterministic); each voxel's list is
// padded to whole 16-byte quads with zero-weight copies of its last record.  A
// second set groups each voxel's records by detector subset first (ordered
// subsets, Sec. VI).  The forward accumulates one voxel at a time into a
// shared-memory detector image, one quad per thread (a pixel occurs once per
// voxel, and its pad copies are in the same quad).  The adjoint gives each
// thread an equal part of the voxel's list and the runs of equal t that start
// in it; runs that cross parts are combined through per-thread slots in a fixed
// order.  Neither kernel uses atomics; both are deterministic.
//
// Record layout (structure of arrays, 12 bytes per record):
//   key = pixel | (t << 16) (uint32), w0 (float), w1 (float).
//
// Mirror-symmetric records (Sec. III-A, when J, M and N are even) serve a pair
// and its left-right / up-down mirror images, which share the interval and the
// weights: the full forward streams one 21-byte record per voxel pair and
// quadrant pixel (8 pairs, k_fwd_sym), the full adjoint t-sorted lists per voxel
// pair of 12-byte records that stand for 4 pairs each (k_adj_sym: one warp per
// voxel pair and knot segment, runs of equal t joined across lanes by a warp
// scan).  The subset and batched operators stream the one-pair records.
#include <cuda_bf16.h>
#include <cuda_fp16.h>

#include <algorithm>
#include <cstring>
#include <vector>

#include "internal.cuh"
#include "pairgeo.cuh"
#include "table.cuh"

namespace {

constexpr int RT = 1024;                 // threads of the streaming kernels
constexpr uint32_t SENT = 0xffffffffu;   // "no run" marker
constexpr uint32_t WAIT_LIMIT = 1u << 24;

struct RecArgs {
    int R, npix, Bp, B;
    int ostride, osel;    // voxel v's records: [off[v * ostride + osel], off[v * ostride + osel + 1])
    const int64_t *off;
    const uint32_t *key;
    const float *w0, *w1;
    // Work items {obj, v0, v1, row0}: voxels [v0, v1) of object obj, whose table
    // row (Wtab / Vtab) is row0 + v - v0; the forward's partial image of item k
    // goes to slot k.  Blocks take items k = blockIdx.x, + gridDim.x, ...
    const int4 *items;    // null: item k is voxel chunk k, {0, k vc, min(R, (k+1) vc), k vc}
    int n_items, vc;
    int64_t w_stride;     // adjoint input image of object obj: w + obj * w_stride
    // Test hooks of the forward record kernel (plan options; 0 in normal use):
    // the polls of its copy waits (0 = WAIT_LIMIT), and whether it withholds the
    // first row copy of each block so that the wait for it runs out.
    uint32_t wait_limit;
    int withhold;
};

// subset < 0: every record of each voxel; else the records of that subset.
RecArgs rec_args(const caxsi_plan *p, const TablePath *T, int subset) {
    const RecSet &r = subset < 0 ? T->rec : T->sub;
    RecArgs a;
    a.R = p->dg.R;
    a.npix = p->dg.M * p->dg.N;
    a.Bp = T->Bp;
    a.B = T->B;
    a.ostride = r.P;
    a.osel = subset < 0 ? 0 : subset;
    a.off = r.off;
    a.key = r.key;
    a.w0 = r.w0;
    a.w1 = r.w1;
    a.items = nullptr;
    a.n_items = T->rec_chunks;
    a.vc = T->rec_vc;
    a.w_stride = 0;
    a.wait_limit = p->test_wait_limit ? p->test_wait_limit : WAIT_LIMIT;
    a.withhold = p->test_withhold;
    return a;
}

template <bool ITEMS>
__device__ __forceinline__ int4 item_at(const RecArgs &A, int k) {
    if (ITEMS) return A.items[k];
    const int v0 = k * A.vc;
    return make_int4(0, v0, min(A.R, v0 + A.vc), v0);
}

__device__ __forceinline__ int64_t rec_begin(const RecArgs &A, int v) {
    return A.off[(int64_t)v * A.ostride + A.osel];
}
__device__ __forceinline__ int64_t rec_end(const RecArgs &A, int v) {
    return A.off[(int64_t)v * A.ostride + A.osel + 1];
}

// ---- one pair, as the on-the-fly table kernels evaluate it --------------------
struct PairRec {
    bool ok;
    int t;
    float w0, w1;
};

__device__ __forceinline__ bool pair_open(const PairArgs &A, int v, int m, int n) {
    const DevGeo &g = A.g;
    const uint32_t word = A.tbits[((int64_t)v * g.M + m) * g.Nw + (n >> 5)];
    return (word >> (n & 31)) & 1u;
}

// The interval and weights of pair (voxel v = (i, j), pixel (m, n)), mask factor
// aside (ok = false when u lies outside the knot range).
__device__ __forceinline__ PairRec pair_geometry(const PairArgs &A, const TabArgs &T, float u_first,
                                                 float u_last, int i, int j, float4 vx, int m, int n) {
    const DevGeo &g = A.g;
    PairRec r;
    r.ok = false;
    float u, ang;
    pair_u_angular(vx.x, vx.y, vx.w, (float)n - g.cN, A.zrow[m], g.p_y, g.Xd, u, ang);
    if (!(u >= u_first && u <= u_last)) return r;
    const int t = find_interval(u, T.knots, T.bstart, T.B, T.NB, T.u0, T.inv_h);
    const float2 kn = T.knots[t];
    const float al = (u - kn.x) * kn.y;
    const float c = vx.z * A.god[((int64_t)i * g.M + m) * g.ND + (n - g.rho_y * j - g.d_min)] * ang;
    r.ok = true;
    r.t = t;
    r.w1 = c * al;
    r.w0 = c - r.w1;
    return r;
}

__device__ __forceinline__ PairRec pair_record(const PairArgs &A, const TabArgs &T, float u_first,
                                               float u_last, int v, int i, int j, float4 vx, int m,
                                               int n) {
    const DevGeo &g = A.g;
    PairRec r;
    r.ok = false;
    const uint32_t word = A.tbits[((int64_t)v * g.M + m) * g.Nw + (n >> 5)];
    if (!((word >> (n & 31)) & 1u)) return r;
    float u, ang;
    pair_u_angular(vx.x, vx.y, vx.w, (float)n - g.cN, A.zrow[m], g.p_y, g.Xd, u, ang);
    if (!(u >= u_first && u <= u_last)) return r;
    const int t = find_interval(u, T.knots, T.bstart, T.B, T.NB, T.u0, T.inv_h);
    const float2 kn = T.knots[t];
    const float al = (u - kn.x) * kn.y;
    const float c = vx.z * A.god[((int64_t)i * g.M + m) * g.ND + (n - g.rho_y * j - g.d_min)] * ang;
    r.ok = true;
    r.t = t;
    r.w1 = c * al;
    r.w0 = c - r.w1;
    return r;
}

// Count the records of each (voxel, group): one warp per voxel, P counters per
// warp in shared memory; the group of a pixel is sub[pixel] (group 0 without sub).
__global__ void k_rec_count(PairArgs A, TabArgs T, const int *sub, int P, int64_t *cnt) {
    extern __shared__ int cnt_s[];
    const DevGeo &g = A.g;
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int v = (blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    if (v >= g.R) return;   // warp-uniform
    int *c = cnt_s + warp * P;
    for (int k = lane; k < P; k += 32) c[k] = 0;
    __syncwarp();
    const float u_first = T.knots[0].x, u_last = T.knots[T.B - 1].x;
    const int i = v / g.J, j = v - i * g.J;
    const float4 vx = A.vox[v];
    const int npix = g.M * g.N;
    for (int p = lane; p < npix; p += 32) {
        const int m = p / g.N, n = p - m * g.N;
        if (pair_record(A, T, u_first, u_last, v, i, j, vx, m, n).ok) atomicAdd(&c[sub ? sub[p] : 0], 1);
    }
    __syncwarp();
    for (int k = lane; k < P; k += 32) cnt[(int64_t)v * P + k] = c[k];
}
// Fill the records of each (voxel, group), sorted by (t, pixel) within the group:
// one warp per voxel, a counting sort over t in a per-warp histogram.  Group s
// holds the pixels sp_pix[sp_off[s] .. sp_off[s+1]) (all pixels when sp_off is
// null, P = 1).  Each group's list is padded to whole 16-byte quads with
// zero-weight copies of its last record (same pixel and interval, so the order
// by t is kept).
__global__ void k_rec_fill(PairArgs A, TabArgs T, int wpb, int P, const int *sp_off, const int *sp_pix,
                           const int64_t *off, uint32_t *key, float *w0, float *w1) {
    extern __shared__ __align__(16) int rec_smem[];
    const DevGeo &g = A.g;
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int v = blockIdx.x * wpb + warp;
    if (warp >= wpb || v >= g.R) return;
    int *hist = rec_smem + warp * (T.B + 1);
    const float u_first = T.knots[0].x, u_last = T.knots[T.B - 1].x;
    const int i = v / g.J, j = v - i * g.J;
    const float4 vx = A.vox[v];
    const unsigned lt = (1u << lane) - 1u;
    for (int s = 0; s < P; ++s) {
        const int64_t base = off[(int64_t)v * P + s], gend = off[(int64_t)v * P + s + 1];
        if (gend == base) continue;   // warp-uniform: no records in this group
        const int np = sp_off ? sp_off[s + 1] - sp_off[s] : g.M * g.N;
        const int *list = sp_off ? sp_pix + sp_off[s] : nullptr;
        for (int t = lane; t <= T.B; t += 32) hist[t] = 0;
        __syncwarp();
        for (int k = lane; k < np; k += 32) {
            const int p = list ? list[k] : k;
            const int m = p / g.N, n = p - m * g.N;
            const PairRec r = pair_record(A, T, u_first, u_last, v, i, j, vx, m, n);
            if (r.ok) atomicAdd(&hist[r.t], 1);
        }
        __syncwarp();
        // exclusive scan of hist[0..B) by the warp: contiguous chunks per lane
        const int chunk = (T.B + 31) / 32;
        const int t0 = min(T.B, lane * chunk), t1 = min(T.B, t0 + chunk);
        int local = 0;
        for (int t = t0; t < t1; ++t) local += hist[t];
        int incl = local;
        for (int o = 1; o < 32; o <<= 1) {
            const int y = __shfl_up_sync(0xffffffffu, incl, o);
            if (lane >= o) incl += y;
        }
        int run = incl - local;
        for (int t = t0; t < t1; ++t) {
            const int h = hist[t];
            hist[t] = run;
            run += h;
        }
        __syncwarp();
        for (int kb = 0; kb < np; kb += 32) {
            const int k = kb + lane;
            PairRec r;
            r.ok = false;
            int p = 0;
            if (k < np) {
                p = list ? list[k] : k;
                const int m = p / g.N, n = p - m * g.N;
                r = pair_record(A, T, u_first, u_last, v, i, j, vx, m, n);
            }
            const unsigned act = __ballot_sync(0xffffffffu, r.ok);
            unsigned grp = 0;
            int pos = 0;
            if (r.ok) {
                grp = __match_any_sync(act, r.t);
                pos = hist[r.t] + __popc(grp & lt);
            }
            __syncwarp();
            if (r.ok) {
                if ((grp & lt) == 0) hist[r.t] += __popc(grp);
                const int64_t q = base + pos;
                key[q] = (uint32_t)p | ((uint32_t)r.t << 16);
                w0[q] = r.w0;
                w1[q] = r.w1;
            }
            __syncwarp();
        }
        const int creal = __shfl_sync(0xffffffffu, incl, 31);
        const int npadv = (int)(gend - base) - creal;
        if (lane < npadv) {
            const int64_t q = base + creal + lane;
            key[q] = key[base + creal - 1];
            w0[q] = 0.f;
            w1[q] = 0.f;
        }
        __syncwarp();
    }
}

// ---- TMA bulk copy + mbarrier helpers -----------------------------------------
__device__ __forceinline__ uint32_t smem_u32(const void *p) {
    return (uint32_t)__cvta_generic_to_shared(p);
}
__device__ __forceinline__ void mbar_init(uint64_t *bar, uint32_t count) {
    asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_u32(bar)), "r"(count) : "memory");
}
__device__ __forceinline__ void mbar_expect_tx(uint64_t *bar, uint32_t bytes) {
    asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(smem_u32(bar)), "r"(bytes)
                 : "memory");
}
__device__ __forceinline__ void bulk_g2s(void *dst, const void *src, uint32_t bytes, uint64_t *bar) {
    asm volatile(
        "cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];" ::"r"(
            smem_u32(dst)),
        "l"(src), "r"(bytes), "r"(smem_u32(bar))
        : "memory");
}
__device__ __forceinline__ bool mbar_try_wait(uint64_t *bar, uint32_t parity) {
    uint32_t ok;
    asm volatile(
        "{\n .reg .pred p;\n mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n selp.u32 %0, 1, 0, p;\n}\n"
        : "=r"(ok)
        : "r"(smem_u32(bar)), "r"(parity)
        : "memory");
    return ok != 0;
}
// Bulk prefetch of [src, src + bytes) into L2, trimmed inwards to whole 16-byte
// units (the copy's alignment rule); the trimmed edges are left to the loads.
__device__ __forceinline__ void bulk_prefetch_l2(const void *src, size_t bytes) {
    const uintptr_t a = reinterpret_cast<uintptr_t>(src);
    const uintptr_t b = (a + 15) & ~(uintptr_t)15, e = (a + bytes) & ~(uintptr_t)15;
    if (e > b)
        asm volatile("cp.async.bulk.prefetch.L2.global [%0], %1;" ::"l"(b), "r"((uint32_t)(e - b)) : "memory");
}
// Bounded wait: false if the phase did not complete within `limit` polls.
__device__ __forceinline__ bool mbar_wait(uint64_t *bar, uint32_t parity, uint32_t limit = WAIT_LIMIT) {
    for (uint32_t k = 0; k < limit; ++k)
        if (mbar_try_wait(bar, parity)) return true;
    return false;
}

// Forward streaming kernel.  Block = 1024 threads, work items of voxels (one
// chunk of an object's voxels each; a single-object call has one item per
// block); the detector image accumulates in shared memory and is written out per
// item; each voxel's Wtab row arrives by a TMA bulk copy, double-buffered one
// voxel ahead, and the next voxel's records are prefetched into L2 meanwhile.
constexpr int FWD_U = 2;   // quads a thread loads before it uses the first
template <bool ITEMS>
__global__ void __launch_bounds__(RT, 1)
k_fwd_rec(RecArgs A, const float *__restrict__ Wtab, float *__restrict__ part, int *err) {
    extern __shared__ __align__(128) unsigned char smem_raw[];
    const int npix_al = (A.npix + 3) & ~3;
    float *g_s = reinterpret_cast<float *>(smem_raw);
    float *wbuf0 = g_s + npix_al;
    float *wbuf1 = wbuf0 + A.Bp;
    uint64_t *bar = reinterpret_cast<uint64_t *>(wbuf1 + A.Bp);
    const int tid = threadIdx.x;
    if (blockIdx.x >= (unsigned)A.n_items) return;   // block-uniform
    const uint32_t row_bytes = (uint32_t)A.Bp * 4u;
    if (tid == 0) {
        mbar_init(&bar[0], 1);
        mbar_init(&bar[1], 1);
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    }
    bool ok = true;
    uint32_t ph0 = 0u, ph1 = 0u;   // mbarrier phase parity of each buffer
    bool pend0 = false, pend1 = false;   // thread 0: a copy it issued on that buffer has not been awaited
    for (int k = blockIdx.x; k < A.n_items && ok; k += gridDim.x) {
        const int4 it = item_at<ITEMS>(A, k);
        const int v0 = it.y, v1 = it.z;
        const int64_t r0 = (int64_t)it.w - v0;   // table row of voxel v: r0 + v
        for (int p = tid; p < A.npix; p += RT) g_s[p] = 0.f;
        if (tid == 0 && !A.withhold) {
            // buffer 0 was last read before the barrier that ended the previous item
            asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
            mbar_expect_tx(&bar[0], row_bytes);
            bulk_g2s(wbuf0, Wtab + (r0 + v0) * A.Bp, row_bytes, &bar[0]);
            pend0 = true;
        }
        __syncthreads();
        for (int v = v0; v < v1; ++v) {
            const int buf = (v - v0) & 1;
            float *w_s = buf ? wbuf1 : wbuf0;
            if (tid == 0 && v + 1 < v1) {
                // the other buffer was last read by voxel v - 1, finished at the barrier below
                asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
                mbar_expect_tx(&bar[buf ^ 1], row_bytes);
                bulk_g2s(buf ? wbuf0 : wbuf1, Wtab + (r0 + v + 1) * A.Bp, row_bytes, &bar[buf ^ 1]);
                if (buf) pend0 = true; else pend1 = true;
            }
            if (tid == 32 && v + 1 < v1) {
                const int64_t nb = rec_begin(A, v + 1), nbytes = 4 * (rec_end(A, v + 1) - nb);
                bulk_prefetch_l2(A.key + nb, (size_t)nbytes);
                bulk_prefetch_l2(A.w0 + nb, (size_t)nbytes);
                bulk_prefetch_l2(A.w1 + nb, (size_t)nbytes);
            }
            const int late = mbar_wait(&bar[buf], buf ? ph1 : ph0, A.wait_limit) ? 0 : 1;
            if (__syncthreads_or(late)) {   // block-uniform decision
                ok = false;
                break;
            }
            if (buf) { ph1 ^= 1u; pend1 = false; } else { ph0 ^= 1u; pend0 = false; }
            // Whole 16-byte quads per thread: a pixel occurs once per voxel, except the
            // zero-weight pad records, which share the last record's pixel and sit in
            // its quad, so they are accumulated by the same thread, in order.
            const int64_t b = rec_begin(A, v);
            const int nq = (int)((rec_end(A, v) - b) >> 2);
            const uint4 *K4 = reinterpret_cast<const uint4 *>(A.key + b);
            const float4 *A4 = reinterpret_cast<const float4 *>(A.w0 + b);
            const float4 *C4 = reinterpret_cast<const float4 *>(A.w1 + b);
            auto one = [&](uint32_t key, float a0, float a1) {
                const int t = (int)(key >> 16);
                g_s[key & 0xffffu] += fmaf(a0, w_s[t], a1 * w_s[t + 1]);
            };
            for (int q0 = tid; q0 < nq; q0 += FWD_U * RT) {
                uint4 k4[FWD_U];
                float4 a4[FWD_U], c4[FWD_U];
#pragma unroll
                for (int u = 0; u < FWD_U; ++u) {
                    const int q = q0 + u * RT;
                    if (q < nq) {
                        k4[u] = K4[q];
                        a4[u] = A4[q];
                        c4[u] = C4[q];
                    }
                }
#pragma unroll
                for (int u = 0; u < FWD_U; ++u) {
                    if (q0 + u * RT >= nq) break;
                    one(k4[u].x, a4[u].x, c4[u].x);
                    one(k4[u].y, a4[u].y, c4[u].y);
                    one(k4[u].z, a4[u].z, c4[u].z);
                    one(k4[u].w, a4[u].w, c4[u].w);
                }
            }
            __syncthreads();
        }
        if (!ok) break;
        float *dst = part + (int64_t)k * A.npix;
        for (int p = tid; p < A.npix; p += RT) dst[p] = g_s[p];
        __syncthreads();
    }
    if (!ok && tid == 0) {
        // a copy did not land in time: report, drain the copies this block issued, stop
        atomicExch(err, 1);
        if (pend0) mbar_wait(&bar[0], ph0);
        if (pend1) mbar_wait(&bar[1], ph1);
    }
}

__device__ __forceinline__ void store_v4(float *p, float4 x) { *reinterpret_cast<float4 *>(p) = x; }
__device__ __forceinline__ void store_v4(__nv_bfloat16 *p, float4 x) {
    __nv_bfloat162 lo = __floats2bfloat162_rn(x.x, x.y), hi = __floats2bfloat162_rn(x.z, x.w);
    uint2 u;
    u.x = *reinterpret_cast<uint32_t *>(&lo);
    u.y = *reinterpret_cast<uint32_t *>(&hi);
    *reinterpret_cast<uint2 *>(p) = u;
}
__device__ __forceinline__ void store_v2(float *p, float a, float b) { *reinterpret_cast<float2 *>(p) = make_float2(a, b); }
__device__ __forceinline__ void store_v2(__nv_bfloat16 *p, float a, float b) {
    *reinterpret_cast<__nv_bfloat162 *>(p) = __floats2bfloat162_rn(a, b);
}
__device__ __forceinline__ void store_v2(__half *p, float a, float b) {
    *reinterpret_cast<__half2 *>(p) = __floats2half2_rn(a, b);
}
__device__ __forceinline__ void store_v4(__half *p, float4 x) {
    __half2 lo = __floats2half2_rn(x.x, x.y), hi = __floats2half2_rn(x.z, x.w);
    uint2 u;
    u.x = *reinterpret_cast<uint32_t *>(&lo);
    u.y = *reinterpret_cast<uint32_t *>(&hi);
    *reinterpret_cast<uint2 *>(p) = u;
}

// Adjoint streaming kernel: V[t] = sum over records of interval t of w0 * w[pixel]
// plus sum over records of interval t - 1 of w1 * w[pixel] (the two knots of each
// record's interval).  One block of ADJ_T threads per SM, a chunk of voxels; the
// input image w is staged once in shared memory and V is built in shared memory.
//
// Every voxel's list is whole 16-byte quads.  Per voxel, thread i takes the i-th of
// ADJ_T equal parts (in quads) of the t-sorted list and sums each run of equal t in
// registers.  A run that starts in the part is the thread's ("head" run); a run that
// began in a lower part leaves its partial sums in the thread's slot.  Complete head
// runs are written at once: V[t] = LO(t) + HI(t-1) when the same thread owns run
// t-1, V[t'+1] = HI(t') at a gap.  After a barrier each thread adds the slots of the
// following threads that continue its last run, in thread order, and writes that
// run's V entry; after a second barrier it adds the run's HI to the next knot.  Every
// V entry thus has one writer per phase and a fixed order of additions: no atomics,
// deterministic results.
//
// Each warp's segment of the next voxel (its first ADJ_SQ quads of keys, w0 and w1,
// and the quad before the segment) is brought into shared memory by TMA bulk copies
// on the warp's mbarrier while the current voxel is processed.  Waits are bounded: a
// copy that does not land sets *err, and the block drains its copies and stops.
constexpr int ADJ_T = 1024;
constexpr int ADJ_W = ADJ_T / 32;
constexpr int ADJ_SQ = 64;

template <typename OutT, bool ITEMS>
__global__ void __launch_bounds__(ADJ_T, 1)
k_adj_rec(RecArgs A, const float *__restrict__ w, OutT *__restrict__ Vtab, int *err) {
    extern __shared__ __align__(128) unsigned char smem_raw[];
    const int npix_al = (A.npix + 3) & ~3;
    float *w_s = reinterpret_cast<float *>(smem_raw);
    float *V = w_s + npix_al;
    uint4 *stg_k = reinterpret_cast<uint4 *>(V + A.Bp);           // [ADJ_W][ADJ_SQ]
    float4 *stg_a = reinterpret_cast<float4 *>(stg_k + ADJ_W * ADJ_SQ);
    float4 *stg_c = stg_a + ADJ_W * ADJ_SQ;
    uint4 *stg_p = reinterpret_cast<uint4 *>(stg_c + ADJ_W * ADJ_SQ);   // [ADJ_W]
    uint32_t *slot_t = reinterpret_cast<uint32_t *>(stg_p + ADJ_W);
    float *slot_lo = reinterpret_cast<float *>(slot_t + ADJ_T);
    float *slot_hi = slot_lo + ADJ_T;
    uint64_t *bar = reinterpret_cast<uint64_t *>(slot_hi + ADJ_T);    // [ADJ_W]
    const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
    if (blockIdx.x >= (unsigned)A.n_items) return;   // block-uniform

    // The warp's quads [ws, we) of the voxel with list [ob, oe): thread parts of perq
    // quads, ADJ_T parts.
    auto segment = [&](int64_t ob, int64_t oe, int &ws, int &we, int &perq) {
        const int nq = (int)((oe - ob) >> 2);
        perq = (nq + ADJ_T - 1) / ADJ_T;
        ws = min(nq, warp * 32 * perq);
        we = min(nq, ws + 32 * perq);
    };
    // The whole warp: stage the warp's segment of the voxel [ob, oe), one copy per
    // lane 0-3 after lane 0 has set the expected bytes (the stage was last read
    // through the generic proxy, hence the proxy fences).
    auto issue = [&](int64_t ob, int64_t oe) {
        int ws, we, perq;
        segment(ob, oe, ws, we, perq);
        const int ns = min(we, ws + ADJ_SQ) - ws;
        const bool kp = ws > 0 && ws < we;
        if (lane == 0) mbar_expect_tx(&bar[warp], 48u * (uint32_t)ns + (kp ? 16u : 0u));
        __syncwarp();
        if (lane < 4) asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
        const int64_t r = ob + 4 * (int64_t)ws;
        if (lane == 0 && ns > 0) bulk_g2s(stg_k + warp * ADJ_SQ, A.key + r, 16u * ns, &bar[warp]);
        if (lane == 1 && ns > 0) bulk_g2s(stg_a + warp * ADJ_SQ, A.w0 + r, 16u * ns, &bar[warp]);
        if (lane == 2 && ns > 0) bulk_g2s(stg_c + warp * ADJ_SQ, A.w1 + r, 16u * ns, &bar[warp]);
        if (lane == 3 && kp) bulk_g2s(stg_p + warp, A.key + ob + 4 * (int64_t)(ws - 1), 16u, &bar[warp]);
    };

    if (tid == 0) {
        for (int k = 0; k < ADJ_W; ++k) mbar_init(&bar[k], 1);
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    }
    for (int t = tid; t < A.Bp; t += ADJ_T) V[t] = 0.f;
    uint32_t par = 0u;       // parity of the warp's outstanding phase
    bool pending = false;    // the warp has staged copies in flight
    bool ok = true;
    int staged = -1;         // the object whose w is in w_s
    for (int k = blockIdx.x; k < A.n_items && ok; k += gridDim.x) {
    const int4 item = item_at<ITEMS>(A, k);
    const int v0 = item.y, v1 = item.z;
    const int64_t r0 = (int64_t)item.w - v0;   // table row of voxel v: r0 + v
    if (item.x != staged) {
        // (the previous voxel ended with a barrier: no thread reads w_s any more)
        const float *wo = w + (int64_t)item.x * A.w_stride;
        for (int p = tid; p < A.npix; p += ADJ_T) w_s[p] = wo[p];
        staged = item.x;
    }
    __syncthreads();
    int64_t ob = rec_begin(A, v0), oe = rec_end(A, v0);
    issue(ob, oe);
    pending = true;
    const int vn = min(v0 + 1, v1 - 1);
    int64_t on0 = rec_begin(A, vn), on1 = rec_end(A, vn);   // the next voxel's list
    for (int v = v0; v < v1; ++v) {
        const int late = __any_sync(0xffffffffu, !mbar_wait(&bar[warp], par)) ? 1 : 0;
        int ws, we, perq;
        segment(ob, oe, ws, we, perq);
        const int q0 = min(we, ws + lane * perq), q1 = min(we, q0 + perq);
        const int i0 = q0 - ws, sb = warp * ADJ_SQ;
        const uint4 *K4 = reinterpret_cast<const uint4 *>(A.key + ob);
        const float4 *A4 = reinterpret_cast<const float4 *>(A.w0 + ob);
        const float4 *C4 = reinterpret_cast<const float4 *>(A.w1 + ob);
        uint4 k0 = make_uint4(0u, 0u, 0u, 0u), k1 = k0;
        float4 a0 = make_float4(0.f, 0.f, 0.f, 0.f), a1 = a0, c0 = a0, c1 = a0;
        uint32_t kprev = 0u;
        if (!late) {
            if (q0 < q1) {
                if (i0 < ADJ_SQ) { k0 = stg_k[sb + i0]; a0 = stg_a[sb + i0]; c0 = stg_c[sb + i0]; }
                else { k0 = K4[q0]; a0 = A4[q0]; c0 = C4[q0]; }
                if (q0 > 0) {
                    if (lane == 0) kprev = stg_p[warp].w;
                    else if (i0 - 1 < ADJ_SQ) kprev = stg_k[sb + i0 - 1].w;
                    else kprev = A.key[ob + 4 * (int64_t)q0 - 1];
                }
            }
            if (q0 + 1 < q1) {
                if (i0 + 1 < ADJ_SQ) { k1 = stg_k[sb + i0 + 1]; a1 = stg_a[sb + i0 + 1]; c1 = stg_c[sb + i0 + 1]; }
                else { k1 = K4[q0 + 1]; a1 = A4[q0 + 1]; c1 = C4[q0 + 1]; }
            }
            // `dep` is 0 but depends on every register read from the stage, so the
            // warp barrier below is passed only once those reads have completed.
            unsigned dep = k0.x ^ k0.y ^ k0.z ^ k0.w ^ k1.x ^ k1.y ^ k1.z ^ k1.w ^ kprev ^
                           __float_as_uint(a0.x) ^ __float_as_uint(a0.y) ^ __float_as_uint(a0.z) ^
                           __float_as_uint(a0.w) ^ __float_as_uint(a1.x) ^ __float_as_uint(a1.y) ^
                           __float_as_uint(a1.z) ^ __float_as_uint(a1.w) ^ __float_as_uint(c0.x) ^
                           __float_as_uint(c0.y) ^ __float_as_uint(c0.z) ^ __float_as_uint(c0.w) ^
                           __float_as_uint(c1.x) ^ __float_as_uint(c1.y) ^ __float_as_uint(c1.z) ^
                           __float_as_uint(c1.w);
            asm volatile("and.b32 %0, %0, 0;" : "+r"(dep));
            kprev += dep;
        }
        __syncwarp();
        if (!late) {   // warp-uniform
            par ^= 1u;
            pending = false;
            if (v + 1 < v1) {
                issue(on0, on1);
                pending = true;
            }
        }
        // the current voxel's list is no longer needed past this point (pointers
        // taken above); load the one after the next
        ob = on0;
        oe = on1;
        {
            const int vn2 = min(v + 2, v1 - 1);
            on0 = rec_begin(A, vn2);
            on1 = rec_end(A, vn2);
        }

        // A part that does not start the voxel begins inside the run of the record
        // before it, with zero partial sums (a zero slot if that run ends there).
        uint32_t ct = SENT, pt = SENT, st = SENT;
        bool cont = false;
        float clo = 0.f, chi = 0.f, ph = 0.f, slo = 0.f, shi = 0.f;
        if (!late && q0 < q1) {
            cont = q0 > 0;
            ct = (cont ? kprev : k0.x) >> 16;
            auto take = [&](uint32_t k, float wa, float wb) {
                const uint32_t t = k >> 16;
                const float x = w_s[k & 0xffffu];
                if (t != ct) {
                    if (cont) {   // the continued run ends inside the part
                        st = ct;
                        slo = clo;
                        shi = chi;
                        cont = false;
                    } else {      // a complete head run
                        const float lo = clo + (pt + 1 == ct ? ph : 0.f);
                        if (pt != SENT && pt + 1 != ct) V[pt + 1] = ph;
                        V[ct] = lo;
                        pt = ct;
                        ph = chi;
                    }
                    ct = t;
                    clo = 0.f;
                    chi = 0.f;
                }
                clo = fmaf(wa, x, clo);
                chi = fmaf(wb, x, chi);
            };
            auto take4 = [&](const uint4 &k, const float4 &a, const float4 &c) {
                take(k.x, a.x, c.x);
                take(k.y, a.y, c.y);
                take(k.z, a.z, c.z);
                take(k.w, a.w, c.w);
            };
            take4(k0, a0, c0);
            if (q0 + 1 < q1) take4(k1, a1, c1);
            for (int q = q0 + 2; q < q1; ++q) take4(K4[q], A4[q], C4[q]);
            if (cont) {      // the whole part continues one run
                st = ct;
                slo = clo;
                shi = chi;
                ct = SENT;
            }
        }
        slot_t[tid] = st;
        slot_lo[tid] = slo;
        slot_hi[tid] = shi;
        if (__syncthreads_or(late)) {   // block-uniform decision
            ok = false;
            break;
        }
        if (ct != SENT) {    // the last head run: add its continuations, in order
            for (int k = tid + 1; k < ADJ_T && slot_t[k] == ct; ++k) {
                clo += slot_lo[k];
                chi += slot_hi[k];
            }
            float lo = clo;
            if (pt != SENT) {
                if (pt + 1 == ct) lo += ph;
                else V[pt + 1] = ph;
            }
            V[ct] = lo;
        }
        __syncthreads();
        if (ct != SENT) V[ct + 1] += chi;
        __syncthreads();
        // write the row (all Bp entries, whole quads) and clear V for the next voxel
        OutT *vrow = Vtab + (r0 + v) * A.Bp;
        float4 *V4 = reinterpret_cast<float4 *>(V);
        const float4 zero4 = make_float4(0.f, 0.f, 0.f, 0.f);
        for (int t4 = tid; t4 < (A.Bp >> 2); t4 += ADJ_T) {
            store_v4(vrow + 4 * t4, V4[t4]);
            V4[t4] = zero4;
        }
        __syncthreads();
    }
    }
    if (!ok && lane == 0) {
        // a copy did not land in time: report, drain this warp's copy in flight, stop
        atomicExch(err, 1);
        if (pending) mbar_wait(&bar[warp], par);
    }
}

// ---- mirror-symmetric records (forward) ------------------------------------------
struct SymArgs {
    int R2, J2, J, M, N, NH, npix, Bp, nrec, vc;
    const uint32_t *tt;
    const uint8_t *tb;
    const float4 *w;
};

SymArgs sym_args(const caxsi_plan *p, const TablePath *T) {
    SymArgs a;
    a.R2 = T->sym.R2;
    a.J = p->dg.J;
    a.J2 = p->dg.J / 2;
    a.M = p->dg.M;
    a.N = p->dg.N;
    a.NH = p->dg.N / 2;
    a.npix = p->dg.M * p->dg.N;
    a.Bp = T->Bp;
    a.nrec = T->sym.nrec;
    a.vc = T->sym.vc;
    a.tt = T->sym.tt;
    a.tb = T->sym.tb;
    a.w = T->sym.w;
    return a;
}

// Record (s, r): voxel pair s = (i, jq), v = (i, jq), v' = (i, J-1-jq); quadrant
// pixel r = (m, n), m < M/2, n < N/2.  Mask bits: 0 (v, m, n), 1 (v, M-1-m, n),
// 2 (v', m, N-1-n), 3 (v', M-1-m, N-1-n) [class A]; 4 (v, m, N-1-n),
// 5 (v, M-1-m, N-1-n), 6 (v', m, n), 7 (v', M-1-m, n) [class B].
__global__ void k_sym_build(PairArgs A, TabArgs T, int R2, int nrec, uint32_t *__restrict__ tt,
                            uint8_t *__restrict__ tb, float4 *__restrict__ w) {
    const DevGeo &g = A.g;
    const int64_t idx = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (idx >= (int64_t)R2 * nrec) return;
    const int s = (int)(idx / nrec), r = (int)(idx - (int64_t)s * nrec);
    const int J2 = g.J / 2, NH = g.N / 2;
    const int i = s / J2, jq = s - i * J2;
    const int v = i * g.J + jq, vp = i * g.J + (g.J - 1 - jq);
    const int m = r / NH, n = r - m * NH;
    const int mm = g.M - 1 - m, nn = g.N - 1 - n;
    const float u_first = T.knots[0].x, u_last = T.knots[T.B - 1].x;
    const float4 vx = A.vox[v];
    const PairRec a = pair_geometry(A, T, u_first, u_last, i, jq, vx, m, n);
    const PairRec b = pair_geometry(A, T, u_first, u_last, i, jq, vx, m, nn);
    uint32_t bits = 0;
    bits |= pair_open(A, v, m, n) ? 1u : 0u;
    bits |= pair_open(A, v, mm, n) ? 2u : 0u;
    bits |= pair_open(A, vp, m, nn) ? 4u : 0u;
    bits |= pair_open(A, vp, mm, nn) ? 8u : 0u;
    bits |= pair_open(A, v, m, nn) ? 16u : 0u;
    bits |= pair_open(A, v, mm, nn) ? 32u : 0u;
    bits |= pair_open(A, vp, m, n) ? 64u : 0u;
    bits |= pair_open(A, vp, mm, n) ? 128u : 0u;
    if (!a.ok) bits &= ~15u;
    if (!b.ok) bits &= ~240u;
    tt[idx] = (uint32_t)(a.ok ? a.t : 0) | ((uint32_t)(b.ok ? b.t : 0) << 16);
    tb[idx] = (uint8_t)bits;
    w[idx] = make_float4(a.ok ? a.w0 : 0.f, a.ok ? a.w1 : 0.f, b.ok ? b.w0 : 0.f, b.ok ? b.w1 : 0.f);
}

// Forward over the symmetric records: a block takes a chunk of voxel pairs;
// the two W rows of each pair arrive by TMA bulk copies into a ring of NB
// buffers, and the next pair's records are prefetched into L2; each record adds
// its 8 pairs' contributions to its 4 pixels.  A thread takes the same record
// slots r of every pair, so it alone updates their pixels: the warps need no
// block barrier between pairs and drift apart by up to NB - 1 pairs.  A warp
// that is done with a pair counts itself on the pair's buffer; the last one
// issues the copy of pair s + NB into it, the first one prefetches the records
// of pair s + 2.  A thread loads SYM_U records before it uses the first, so that
// their loads overlap.
// WT: the element type of the knot rows (float, or bf16 for the bf16 path).
constexpr int SYM_U = 4;
// Four bf16 record weights, widened exactly to FP32.
__device__ __forceinline__ float4 bf16x4_to_f4(uint2 u) {
    return make_float4(__uint_as_float(u.x << 16), __uint_as_float(u.x & 0xffff0000u), __uint_as_float(u.y << 16),
                       __uint_as_float(u.y & 0xffff0000u));
}

__device__ __forceinline__ float wval(const float *w, int t) { return w[t]; }
__device__ __forceinline__ float wval(const __nv_bfloat16 *w, int t) { return __bfloat162float(w[t]); }

// W row buffers of k_fwd_sym: 2 for FP32 rows, 4 for bf16 rows (the same bytes).
template <typename WT> struct FwdSymRing { static constexpr int NB = sizeof(WT) == 4 ? 2 : 4; };

template <typename WT>
__global__ void __launch_bounds__(RT, 1)
k_fwd_sym(SymArgs S, const WT *__restrict__ Wtab, float *__restrict__ part, int *err) {
    constexpr int NB = FwdSymRing<WT>::NB;
    constexpr int NW = RT / 32;
    extern __shared__ __align__(128) unsigned char smem_raw[];
    const int npix_al = (S.npix + 3) & ~3;
    float *g_s = reinterpret_cast<float *>(smem_raw);
    WT *wb = reinterpret_cast<WT *>(g_s + npix_al);             // [NB buffers][2 rows][Bp]
    uint64_t *bar = reinterpret_cast<uint64_t *>(wb + 2 * NB * S.Bp);   // [NB] rows landed
    int *done = reinterpret_cast<int *>(bar + NB);                       // [NB] warps done with the buffer
    int *issued = done + NB;                                             // [NB] last pair copied into it
    __shared__ int failed;
    const int tid = threadIdx.x, lane = tid & 31;
    const int s0 = blockIdx.x * S.vc, s1 = min(s0 + S.vc, S.R2);
    if (s0 >= s1) return;   // block-uniform
    const uint32_t row_bytes = (uint32_t)S.Bp * (uint32_t)sizeof(WT);
    auto issue = [&](int s, int buf) {
        const int i = s / S.J2, jq = s - i * S.J2;
        const int64_t v = (int64_t)i * S.J + jq, vp = (int64_t)i * S.J + (S.J - 1 - jq);
        issued[buf] = s;
        asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
        mbar_expect_tx(&bar[buf], 2u * row_bytes);
        bulk_g2s(wb + (2 * buf) * S.Bp, Wtab + v * S.Bp, row_bytes, &bar[buf]);
        bulk_g2s(wb + (2 * buf + 1) * S.Bp, Wtab + vp * S.Bp, row_bytes, &bar[buf]);
    };
    auto prefetch = [&](int s) {
        const int64_t b = (int64_t)s * S.nrec;
        bulk_prefetch_l2(S.tt + b, (size_t)S.nrec * 4);
        bulk_prefetch_l2(S.tb + b, (size_t)S.nrec);
        bulk_prefetch_l2(S.w + b, (size_t)S.nrec * 16);
    };
    for (int p = tid; p < S.npix; p += RT) g_s[p] = 0.f;
    if (tid == 0) {
        failed = 0;
        for (int b = 0; b < NB; ++b) {
            mbar_init(&bar[b], 1);
            done[b] = 0;
            issued[b] = -1;
        }
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
        for (int k = 0; k < NB && s0 + k < s1; ++k) issue(s0 + k, k);
    }
    if (tid == 32 && s0 + 1 < s1) prefetch(s0 + 1);
    __syncthreads();
    for (int s = s0; s < s1; ++s) {
        const int k = s - s0, buf = k % NB;
        // warp-uniform: a warp goes on only if every lane saw the rows land
        if (!__all_sync(0xffffffffu, mbar_wait(&bar[buf], (uint32_t)(k / NB) & 1u))) {
            failed = 1;
            break;
        }
        const WT *Wv = wb + (2 * buf) * S.Bp, *Wp = Wv + S.Bp;
        const int64_t base = (int64_t)s * S.nrec;
        for (int r0 = tid; r0 < S.nrec; r0 += SYM_U * RT) {
            uint32_t t2[SYM_U], bits[SYM_U];
            float4 ww[SYM_U];
#pragma unroll
            for (int u = 0; u < SYM_U; ++u) {
                const int r = r0 + u * RT;
                t2[u] = 0u;
                bits[u] = 0u;
                ww[u] = make_float4(0.f, 0.f, 0.f, 0.f);
                if (r < S.nrec) {
                    t2[u] = S.tt[base + r];
                    bits[u] = S.tb[base + r];
                    ww[u] = S.w[base + r];
                }
            }
#pragma unroll
            for (int u = 0; u < SYM_U; ++u) {
                const int r = r0 + u * RT;
                if (r >= S.nrec) break;
                const int ta = (int)(t2[u] & 0xffffu), tbb = (int)(t2[u] >> 16);
                const float xav = fmaf(ww[u].x, wval(Wv, ta), ww[u].y * wval(Wv, ta + 1));
                const float xap = fmaf(ww[u].x, wval(Wp, ta), ww[u].y * wval(Wp, ta + 1));
                const float xbv = fmaf(ww[u].z, wval(Wv, tbb), ww[u].w * wval(Wv, tbb + 1));
                const float xbp = fmaf(ww[u].z, wval(Wp, tbb), ww[u].w * wval(Wp, tbb + 1));
                const uint32_t bt = bits[u];
                const int m = r / S.NH, n = r - m * S.NH;
                const int mm = S.M - 1 - m, nn = S.N - 1 - n;
                g_s[m * S.N + n] += ((bt & 1u) ? xav : 0.f) + ((bt & 64u) ? xbp : 0.f);
                g_s[mm * S.N + n] += ((bt & 2u) ? xav : 0.f) + ((bt & 128u) ? xbp : 0.f);
                g_s[m * S.N + nn] += ((bt & 4u) ? xap : 0.f) + ((bt & 16u) ? xbv : 0.f);
                g_s[mm * S.N + nn] += ((bt & 8u) ? xap : 0.f) + ((bt & 32u) ? xbv : 0.f);
            }
        }
        // this warp is done with the buffer (its reads of the rows are complete)
        __syncwarp();
        if (lane == 0) {
            __threadfence_block();
            const int old = atomicAdd(&done[buf], 1);
            if (old == 0 && s + 2 < s1) prefetch(s + 2);
            if (old == NW - 1) {   // the last warp: the buffer is free for pair s + NB
                __threadfence_block();
                done[buf] = 0;
                if (s + NB < s1) issue(s + NB, buf);
            }
        }
    }
    __syncthreads();
    if (failed) {
        // a copy that did not land in time: record it, and wait (bounded) for every
        // copy still in flight before the block's shared memory goes away
        if (tid == 0) {
            atomicExch(err, 1);
            for (int b = 0; b < NB; ++b)
                if (issued[b] >= 0) mbar_wait(&bar[b], (uint32_t)((issued[b] - s0) / NB) & 1u);
        }
        return;
    }
    float *dst = part + (int64_t)blockIdx.x * S.npix;
    for (int p = tid; p < S.npix; p += RT) dst[p] = g_s[p];
}

// ---- mirror-symmetric records (adjoint) -------------------------------------------
// Candidate k of voxel pair (i, jq) (v = (i, jq), v' = (i, J-1-jq)): class c = k /
// ((M/2)(N/2)), quadrant pixel r = k mod (M/2)(N/2) = (m, n0); its column is n = n0
// for class 0 and N-1-n0 for class 1.  The record stands for the four pairs (v, m, n),
// (v, M-1-m, n), (v', m, N-1-n), (v', M-1-m, N-1-n), which share the interval and the
// weights of (v, m, n); ok is false when all four are closed or u is out of range.
// The mask bits are in the order of the quadrant's pixels (m, n0), (M-1-m, n0),
// (m, N-1-n0), (M-1-m, N-1-n0): for class 0 the first two pairs are v's, for class 1
// the last two.
struct SymRec {
    bool ok;
    int t, r, c;
    uint32_t bits;
    float w0, w1;
};

__device__ __forceinline__ SymRec sym_adj_record(const PairArgs &A, const TabArgs &T, float u_first,
                                                 float u_last, int i, int jq, float4 vx, int k) {
    const DevGeo &g = A.g;
    const int NH = g.N / 2, nq = (g.M / 2) * NH;
    const int c = k >= nq ? 1 : 0, r = k - c * nq;
    const int m = r / NH, n0 = r - m * NH;
    const int n = c ? g.N - 1 - n0 : n0;
    const int mm = g.M - 1 - m, nn = g.N - 1 - n;
    const int v = i * g.J + jq, vp = i * g.J + (g.J - 1 - jq);
    SymRec s;
    s.ok = false;
    s.r = r;
    s.c = c;
    const uint32_t b = (pair_open(A, v, m, n) ? 1u : 0u) | (pair_open(A, v, mm, n) ? 2u : 0u) |
                       (pair_open(A, vp, m, nn) ? 4u : 0u) | (pair_open(A, vp, mm, nn) ? 8u : 0u);
    s.bits = c ? ((b & 3u) << 2) | (b >> 2) : b;
    if (!s.bits) return s;
    const PairRec pr = pair_geometry(A, T, u_first, u_last, i, jq, vx, m, n);
    if (!pr.ok) return s;
    s.ok = true;
    s.t = pr.t;
    s.w0 = pr.w0;
    s.w1 = pr.w1;
    return s;
}

// Count the records of each voxel pair: one warp per pair.
__global__ void k_sadj_count(PairArgs A, TabArgs T, int R2, int64_t *cnt) {
    const DevGeo &g = A.g;
    const int lane = threadIdx.x & 31;
    const int s = (blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    if (s >= R2) return;   // warp-uniform
    const int J2 = g.J / 2, i = s / J2, jq = s - i * J2;
    const float4 vx = A.vox[i * g.J + jq];
    const float u_first = T.knots[0].x, u_last = T.knots[T.B - 1].x;
    const int nk = (g.M / 2) * g.N;
    int c = 0;
    for (int k = lane; k < nk; k += 32) c += sym_adj_record(A, T, u_first, u_last, i, jq, vx, k).ok ? 1 : 0;
    for (int o = 16; o > 0; o >>= 1) c += __shfl_xor_sync(0xffffffffu, c, o);
    if (lane == 0) cnt[s] = c;
}

// Fill each voxel pair's list sorted by (t, candidate index): one warp per pair, a
// counting sort over t in a per-warp histogram; the list is padded to whole quads
// with zero-weight copies of its last record.  Key: mask bits | class << 4 | quadrant
// pixel << 5 | t << 18.
__global__ void k_sadj_fill(PairArgs A, TabArgs T, int R2, int wpb, const int64_t *off, uint32_t *key,
                            float *w0, float *w1) {
    extern __shared__ __align__(16) int rec_smem[];
    const DevGeo &g = A.g;
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int s = blockIdx.x * wpb + warp;
    if (warp >= wpb || s >= R2) return;   // warp-uniform
    int *hist = rec_smem + warp * (T.B + 1);
    const int J2 = g.J / 2, i = s / J2, jq = s - i * J2;
    const float4 vx = A.vox[i * g.J + jq];
    const float u_first = T.knots[0].x, u_last = T.knots[T.B - 1].x;
    const unsigned lt = (1u << lane) - 1u;
    const int nk = (g.M / 2) * g.N;
    const int64_t base = off[s], lend = off[s + 1];
    if (lend == base) return;
    for (int t = lane; t <= T.B; t += 32) hist[t] = 0;
    __syncwarp();
    for (int k = lane; k < nk; k += 32) {
        const SymRec r = sym_adj_record(A, T, u_first, u_last, i, jq, vx, k);
        if (r.ok) atomicAdd(&hist[r.t], 1);
    }
    __syncwarp();
    const int chunk = (T.B + 31) / 32;
    const int t0 = min(T.B, lane * chunk), t1 = min(T.B, t0 + chunk);
    int local = 0;
    for (int t = t0; t < t1; ++t) local += hist[t];
    int incl = local;
    for (int o = 1; o < 32; o <<= 1) {
        const int y = __shfl_up_sync(0xffffffffu, incl, o);
        if (lane >= o) incl += y;
    }
    int run = incl - local;
    for (int t = t0; t < t1; ++t) {
        const int h = hist[t];
        hist[t] = run;
        run += h;
    }
    __syncwarp();
    for (int kb = 0; kb < nk; kb += 32) {
        const int k = kb + lane;
        SymRec r;
        r.ok = false;
        if (k < nk) r = sym_adj_record(A, T, u_first, u_last, i, jq, vx, k);
        const unsigned act = __ballot_sync(0xffffffffu, r.ok);
        unsigned grp = 0;
        int pos = 0;
        if (r.ok) {
            grp = __match_any_sync(act, r.t);
            pos = hist[r.t] + __popc(grp & lt);
        }
        __syncwarp();
        if (r.ok) {
            if ((grp & lt) == 0) hist[r.t] += __popc(grp);
            const int64_t q = base + pos;
            key[q] = r.bits | ((uint32_t)r.c << 4) | ((uint32_t)r.r << 5) | ((uint32_t)r.t << 18);
            w0[q] = r.w0;
            w1[q] = r.w1;
        }
        __syncwarp();
    }
    const int creal = __shfl_sync(0xffffffffu, incl, 31);
    const int npadv = (int)(lend - base) - creal;
    if (lane < npadv) {
        const int64_t q = base + creal + lane;
        key[q] = key[base + creal - 1];
        w0[q] = 0.f;
        w1[q] = 0.f;
    }
}

// Adjoint over the symmetric lists.  A record adds w0 x and w1 x to knots t and
// t + 1 of two V rows (voxels v and v' of the pair), x = w[m, n] b0 + w[M-1-m, n] b1
// for v and w[m, N-1-n] b2 + w[M-1-m, N-1-n] b3 for v' (b the mask bits).  The
// input image is held in shared memory per quadrant pixel (m, n0) as float4
// {w[m, n0], w[M-1-m, n0], w[m, N-1-n0], w[M-1-m, N-1-n0]}, so a record reads one of
// them and its class says which half is v's.
//
// Work item = (voxel pair s, knot segment [t_lo, t_lo + L)), one warp each; a warp
// takes the block's next item from a shared-memory counter when it comes free, and
// nothing else synchronises the warps once the image is loaded.  The warp reads the
// quads of the pair's t-sorted list that can reach the segment (records with t in
// [t_lo - 1, t_lo + L), from a per-plan table), 32 quads per row, lane l taking
// quad l of the row (coalesced).  Within its quad a lane sums each run of equal t;
// a run that continues across lanes is carried by a segmented scan over the lanes
// of the lanes' last runs (as many doubling steps as the longest chain of lanes
// needs), and a run that continues past the row by a warp-uniform carry.  Every run
// is completed exactly once, by the lane holding its last record, and added into
// the warp's segment buffer V[t + 1 - t_lo] (HI sums, stored) and, after a warp
// barrier, V[t - t_lo] (LO sums, added); each entry gets at most one HI and one LO
// sum, the HI sum first, so the result does not depend on the order of the runs.
// Runs outside the segment are dropped at that point.  The buffer is then written
// to the two V rows (consecutive lanes, consecutive 8 bytes) and cleared.  Every sum has a fixed order, set by the plan:
// repeated calls are bitwise equal.
constexpr int SEG_T = 1024;
constexpr int SEG_W = SEG_T / 32;
constexpr int T_NONE = -2;            // "no carried run"
constexpr int T_PAST = 1 << 30;       // t of the records past the item's last quad

struct SymAdjArgs {
    int R2, J, J2, M, N, Bp, nseg, L;
    const int64_t *off;
    const uint32_t *seg;    // [R2 * nseg] first quad | end quad << 16, relative to the pair's list
    const uint32_t *key;
    const float *w0, *w1;
    const uint16_t *w0_16, *w1_16;   // the same weights as bf16 (the bf16 path), or null
};

// Two-lane FP32 arithmetic in one packed instruction (each lane rounded as fmaf / +).
__device__ __forceinline__ float2 f2fma(float a, float2 x, float2 y) { return __ffma2_rn(make_float2(a, a), x, y); }
__device__ __forceinline__ float2 f2add(float2 a, float2 b) { return __fadd2_rn(a, b); }
__device__ __forceinline__ float2 shfl_up2(float2 v, int o) {
    return make_float2(__shfl_up_sync(0xffffffffu, v.x, o), __shfl_up_sync(0xffffffffu, v.y, o));
}
__device__ __forceinline__ float2 shfl2(float2 v, int l) {
    return make_float2(__shfl_sync(0xffffffffu, v.x, l), __shfl_sync(0xffffffffu, v.y, l));
}
__device__ __forceinline__ uint4 ld_stream_u4(const uint4 *p) {
    uint4 r;
    asm volatile("ld.global.nc.L1::no_allocate.v4.u32 {%0, %1, %2, %3}, [%4];"
                 : "=r"(r.x), "=r"(r.y), "=r"(r.z), "=r"(r.w) : "l"(p));
    return r;
}
__device__ __forceinline__ float4 ld_stream_f4(const float4 *p) {
    float4 r;
    asm volatile("ld.global.nc.L1::no_allocate.v4.f32 {%0, %1, %2, %3}, [%4];"
                 : "=f"(r.x), "=f"(r.y), "=f"(r.z), "=f"(r.w) : "l"(p));
    return r;
}
__device__ __forceinline__ uint2 ld_stream_u2(const uint2 *p) {
    uint2 r;
    asm volatile("ld.global.nc.L1::no_allocate.v2.u32 {%0, %1}, [%2];" : "=r"(r.x), "=r"(r.y) : "l"(p));
    return r;
}
// A quad's weights (four records) from FP32 or bf16 storage.
template <bool W16>
__device__ __forceinline__ float4 quad_w(const float *w, const uint16_t *w16, int64_t ob, int q) {
    if (W16) return bf16x4_to_f4(ld_stream_u2(reinterpret_cast<const uint2 *>(w16 + ob) + q));
    return ld_stream_f4(reinterpret_cast<const float4 *>(w + ob) + q);
}

template <typename OutT, bool W16>
__global__ void __launch_bounds__(SEG_T, 1)
k_adj_sym(SymAdjArgs A, const float *__restrict__ w, OutT *__restrict__ Vtab) {
    extern __shared__ __align__(128) unsigned char smem_raw[];
    __shared__ int next_item;
    const int NH = A.N / 2, nq = (A.M / 2) * NH;
    float4 *w4 = reinterpret_cast<float4 *>(smem_raw);                                  // [nq]
    const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
    float2 *V = reinterpret_cast<float2 *>(smem_raw + 16 * (size_t)nq) + (size_t)warp * A.L;   // [L]
    float4 *V4 = reinterpret_cast<float4 *>(V);
    const float2 zero2 = make_float2(0.f, 0.f);
    const float4 zero4 = make_float4(0.f, 0.f, 0.f, 0.f);
    if (tid == 0) next_item = 0;
    for (int e = tid; e < nq; e += SEG_T) {
        const int m = e / NH, n0 = e - m * NH;
        const float *ra = w + (int64_t)m * A.N, *rb = w + (int64_t)(A.M - 1 - m) * A.N;
        w4[e] = make_float4(ra[n0], rb[n0], ra[A.N - 1 - n0], rb[A.N - 1 - n0]);
    }
    for (int e = lane; e < (A.L >> 1); e += 32) V4[e] = zero4;
    __syncthreads();

    const int nitems = A.R2 * A.nseg;
    for (;;) {
        // the block's items are blockIdx.x + j gridDim.x, in segment-major order (all
        // pairs' segment 0, then segment 1, ...), so that every block gets a like mix
        // of dense and sparse segments
        int j = 0;
        if (lane == 0) j = atomicAdd(&next_item, 1);
        j = __shfl_sync(0xffffffffu, j, 0);
        // (32-bit: nitems + gridDim.x < 2^32)
        const unsigned k = blockIdx.x + (unsigned)j * gridDim.x;
        if (k >= (unsigned)nitems) break;
        const int sg = (int)(k / (unsigned)A.R2), s = (int)(k - (unsigned)sg * (unsigned)A.R2);
        const uint32_t qr = A.seg[(int64_t)s * A.nseg + sg];
        const int qa = (int)(qr & 0xffffu), qe = (int)(qr >> 16);
        const int tlo = sg * A.L;
        const unsigned L = (unsigned)min(A.L, A.Bp - tlo);   // the segment's knots
        const int64_t ob = A.off[s];
        const uint4 *K4 = reinterpret_cast<const uint4 *>(A.key + ob);
        int ct = T_NONE;                 // the run carried from the previous row
        float2 clo = zero2, chi = zero2;
        // the next row's quad is loaded while a row is summed
        uint4 nk = make_uint4(0u, 0u, 0u, 0u);
        float4 na = make_float4(0.f, 0.f, 0.f, 0.f), nc = na;
        if (qa + lane < qe) {
            nk = ld_stream_u4(K4 + qa + lane);
            na = quad_w<W16>(A.w0, A.w0_16, ob, qa + lane);
            nc = quad_w<W16>(A.w1, A.w1_16, ob, qa + lane);
        }
        for (int qb = qa; qb < qe; qb += 32) {
            const int q = qb + lane;
            const uint4 kq = nk;
            const float4 a = na, c = nc;
            if (q + 32 < qe) {
                nk = ld_stream_u4(K4 + q + 32);
                na = quad_w<W16>(A.w0, A.w0_16, ob, q + 32);
                nc = quad_w<W16>(A.w1, A.w1_16, ob, q + 32);
            }
            int t[4];
            float2 lo[4], hi[4];
            if (q < qe) {
                const uint32_t kk[4] = {kq.x, kq.y, kq.z, kq.w};
                const float aa[4] = {a.x, a.y, a.z, a.w}, cc[4] = {c.x, c.y, c.z, c.w};
#pragma unroll
                for (int r = 0; r < 4; ++r) {
                    const uint32_t kr = kk[r];
                    t[r] = (int)(kr >> 18);
                    const float4 im = w4[(kr >> 5) & 0x1fffu];
                    // {image pixels 0 + 1, pixels 2 + 3} of the open pairs; the class
                    // says which of the two is voxel v's
                    const float2 sp = __fadd2_rn(make_float2((kr & 1u) ? im.x : 0.f, (kr & 4u) ? im.z : 0.f),
                                                 make_float2((kr & 2u) ? im.y : 0.f, (kr & 8u) ? im.w : 0.f));
                    const bool cls = (kr & 16u) != 0u;
                    const float2 x = make_float2(cls ? sp.y : sp.x, cls ? sp.x : sp.y);
                    lo[r] = f2fma(aa[r], x, zero2);
                    hi[r] = f2fma(cc[r], x, zero2);
                }
            } else {
#pragma unroll
                for (int r = 0; r < 4; ++r) {
                    t[r] = T_PAST;
                    lo[r] = zero2;
                    hi[r] = zero2;
                }
            }
            // runs within the quad, summed from zero; lo[r] / hi[r] become the sums of
            // the runs that end at record r (r < 3), and the last run's sum goes to
            // (alo, ahi)
            float2 alo = lo[0], ahi = hi[0];
#pragma unroll
            for (int r = 1; r < 4; ++r) {
                if (t[r] != t[r - 1]) {
                    lo[r - 1] = alo;
                    hi[r - 1] = ahi;
                    alo = lo[r];
                    ahi = hi[r];
                } else {
                    alo = f2add(alo, lo[r]);
                    ahi = f2add(ahi, hi[r]);
                }
            }
            const int t0 = t[0], t3 = t[3];
            // the last run continued from the lane before (lane 0: from the row before)
            const int tprev = __shfl_up_sync(0xffffffffu, t3, 1);
            const bool cont = lane == 0 ? t0 == ct : t0 == tprev;
            const bool link = cont && t0 == t3;   // the whole quad continues that run
            // segmented inclusive scan over the lanes of the last runs' sums: a segment
            // starts at every lane that does not continue its predecessor's run; the
            // doubling stops once it spans the longest segment
            float2 Olo = alo, Ohi = ahi;
            if (lane == 0 && link) {
                Olo = f2add(Olo, clo);
                Ohi = f2add(Ohi, chi);
            }
            const unsigned starts = __ballot_sync(0xffffffffu, lane == 0 || !link);
            const int sst = 31 - __clz(starts & (0xffffffffu >> (31 - lane)));
            const unsigned span = __reduce_max_sync(0xffffffffu, (unsigned)(lane - sst));
            for (int o = 1; (unsigned)o <= span; o <<= 1) {   // warp-uniform
                const float2 ylo = shfl_up2(Olo, o), yhi = shfl_up2(Ohi, o);
                if (lane - o >= sst) {
                    Olo = f2add(Olo, ylo);
                    Ohi = f2add(Ohi, yhi);
                }
            }
            // the carry into this lane's first run
            const float2 plo = shfl_up2(Olo, 1), phi = shfl_up2(Ohi, 1);
            float2 Clo = zero2, Chi = zero2;
            if (cont) {
                Clo = lane == 0 ? clo : plo;
                Chi = lane == 0 ? chi : phi;
            }
            // the carried run of the row before ends there if lane 0 does not continue it
            const bool flush = __shfl_sync(0xffffffffu, !cont, 0) && ct != T_NONE;
            const int tnext = __shfl_down_sync(0xffffffffu, t0, 1);
            const bool fin3 = lane < 31 && t3 != tnext;   // the last run ends in this lane
            lo[3] = alo;
            hi[3] = ahi;
            // HI sums of the completed runs, then (after a warp barrier) the LO sums.
            // The HI sum of run t is the first value knot t + 1 receives: run t + 1,
            // whose LO sum goes there too, completes after run t (in this row's LO
            // phase or a later row), so the HI sums are plain stores into the
            // cleared buffer and only the LO sums read back.
#pragma unroll
            for (int r = 0; r < 4; ++r) {
                const bool end = r < 3 ? t[r] != t[r + 1] : fin3;
                if (end) {
                    if (t[r] == t0) {
                        lo[r] = f2add(Clo, lo[r]);
                        hi[r] = f2add(Chi, hi[r]);
                    }
                    const unsigned d = (unsigned)(t[r] + 1 - tlo);
                    if (d < L) V[d] = hi[r];
                }
            }
            if (flush && lane == 0) {
                const unsigned d = (unsigned)(ct + 1 - tlo);
                if (d < L) V[d] = chi;
            }
            __syncwarp();
#pragma unroll
            for (int r = 0; r < 4; ++r) {
                const bool end = r < 3 ? t[r] != t[r + 1] : fin3;
                if (end) {
                    const unsigned d = (unsigned)(t[r] - tlo);
                    if (d < L) V[d] = f2add(V[d], lo[r]);
                }
            }
            if (flush && lane == 0) {
                const unsigned d = (unsigned)(ct - tlo);
                if (d < L) V[d] = f2add(V[d], clo);
            }
            __syncwarp();
            // lane 31's last run goes on into the next row
            ct = __shfl_sync(0xffffffffu, t3, 31);
            clo = shfl2(Olo, 31);
            chi = shfl2(Ohi, 31);
        }
        if (ct != T_NONE && lane == 0) {   // the last carried run ends with the item
            const unsigned d = (unsigned)(ct - tlo);
            if (d < L) V[d] = f2add(V[d], clo);
            const unsigned d1 = (unsigned)(ct + 1 - tlo);
            if (d1 < L) V[d1] = f2add(V[d1], chi);
        }
        __syncwarp();
        // rows v and v' over the segment; clear the buffer for the next item
        const int i = s / A.J2, jq = s - i * A.J2;
        OutT *rv = Vtab + ((int64_t)i * A.J + jq) * A.Bp + tlo;
        OutT *rp = Vtab + ((int64_t)i * A.J + (A.J - 1 - jq)) * A.Bp + tlo;
        const int nL = (int)L;
        for (int e = lane; 2 * e < nL; e += 32) {
            const float4 x = V4[e];
            V4[e] = zero4;
            store_v2(rv + 2 * e, x.x, x.z);
            store_v2(rp + 2 * e, x.y, x.w);
        }
        __syncwarp();
    }
}

// Shared memory of k_adj_sym: the quadrant image and one segment buffer per warp.
size_t adj_sym_smem(int nq, int L) { return 16 * (size_t)nq + (size_t)SEG_W * L * sizeof(float2); }

// The quad range of each (voxel pair, knot segment) item: the quads that hold the
// records with t in [sg L - 1, (sg + 1) L), by binary search in the t-sorted list.
__global__ void k_sadj_segs(const int64_t *__restrict__ off, const uint32_t *__restrict__ key, int R2, int nseg,
                            int L, uint32_t *__restrict__ seg) {
    const int64_t it = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (it >= (int64_t)R2 * nseg) return;
    const int s = (int)(it / nseg), sg = (int)(it - (int64_t)s * nseg);
    const int64_t b = off[s];
    const int n = (int)(off[s + 1] - b);
    auto first_at_least = [&](int tv) {
        int lo = 0, hi = n;
        while (lo < hi) {
            const int mid = (lo + hi) >> 1;
            if ((int)(key[b + mid] >> 18) < tv) lo = mid + 1;
            else hi = mid;
        }
        return lo;
    };
    const int a = first_at_least(sg * L - 1), e = first_at_least((sg + 1) * L);
    seg[it] = (uint32_t)(a >> 2) | ((uint32_t)((e + 3) >> 2) << 16);
}

// ---- sparse subset operators (ordered subsets) -----------------------------------
// A subset operator needs W = f S~^T (and V) only at the knots of its own pairs:
// about 1/P of each voxel's records.  These kernels contract record by record on
// the CUDA cores against the rows of S~ ([B][Q] FP32, L2-resident) instead of
// running the whole-object contractions: one warp per voxel, lane l holding the
// q bins 4l .. 4l + 3 (Q <= 128, Q % 4 == 0).  The pad records (zero weights)
// are skipped.  Both are deterministic (fixed orders, no atomics).
struct SubArgs {
    int R, Q, P, subset, np;
    const int64_t *off;        // records of (voxel v, subset s): [off[v P + s], off[v P + s + 1])
    const uint32_t *key;       // pixel | t << 16
    const float *w0, *w1;
    const float *S;            // [B][Q]
    const int *pos;            // [M*N] position of a pixel in its subset's list
};

__device__ __forceinline__ float warp_sum(float x) {
    for (int o = 16; o > 0; o >>= 1) x += __shfl_xor_sync(0xffffffffu, x, o);
    return x;
}

// Forward: W at a record's two knots as dot products of the voxel's f row with
// two rows of S~, once per run of equal t; the runs of a batch of 32 records are
// found with a ballot and taken four at a time, their eight rows loaded before
// any is reduced (the loads, not the arithmetic, set the pace).  Each warp adds
// w0 W_t + w1 W_t+1 of its records into its own compact image (np floats, by
// list position), and the block sums its warps' images in warp order into its
// partial image part[blockIdx.x][np].
__global__ void k_fwd_sub(SubArgs A, const float *__restrict__ f, float *__restrict__ part) {
    extern __shared__ __align__(16) float img[];   // [warps][np]
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31, nw = blockDim.x >> 5;
    float *mine = img + (size_t)warp * A.np;
    for (int e = lane; e < A.np; e += 32) mine[e] = 0.f;
    __syncwarp();
    const bool ql = 4 * lane < A.Q;
    for (int v = blockIdx.x * nw + warp; v < A.R; v += gridDim.x * nw) {
        const int64_t b = A.off[(int64_t)v * A.P + A.subset], e = A.off[(int64_t)v * A.P + A.subset + 1];
        if (b == e) continue;   // warp-uniform
        const float4 fq = ql ? *reinterpret_cast<const float4 *>(f + (int64_t)v * A.Q + 4 * lane)
                             : make_float4(0.f, 0.f, 0.f, 0.f);
        auto row = [&](int t) {
            return ql ? *reinterpret_cast<const float4 *>(A.S + (int64_t)t * A.Q + 4 * lane)
                      : make_float4(0.f, 0.f, 0.f, 0.f);
        };
        auto dot = [&](float4 s) { return warp_sum(fmaf(fq.x, s.x, fmaf(fq.y, s.y, fmaf(fq.z, s.z, fq.w * s.w)))); };
        int ct = -2;                // the run in progress at the end of the previous batch
        float wt = 0.f, wt1 = 0.f;  // its W at t and t + 1
        for (int64_t r0 = b; r0 < e; r0 += 32) {
            const int n = (int)min((int64_t)32, e - r0);
            uint32_t k = 0u;
            float a = 0.f, c = 0.f;
            if (lane < n) {
                k = A.key[r0 + lane];
                a = A.w0[r0 + lane];
                c = A.w1[r0 + lane];
            }
            // the batch's runs of equal t: a lane's run starts at the last run start at or
            // before it (none: the run continued from the previous batch)
            const int tl = (int)(k >> 16);
            const int tprev = __shfl_up_sync(0xffffffffu, tl, 1);
            unsigned starts = __ballot_sync(0xffffffffu, lane < n && (lane == 0 ? tl != ct : tl != tprev));
            const unsigned upto = starts & (lane == 31 ? 0xffffffffu : ((2u << lane) - 1u));
            const int my_start = upto ? 31 - __clz(upto) : -1;
            float val = fmaf(a, wt, c * wt1);   // for a run continued from the previous batch
            // the runs four at a time: their eight rows of S~ are loaded before any is reduced
            while (starts) {
                int js[4], ts[4], cnt = 0;
                for (; cnt < 4 && starts; ++cnt) {
                    js[cnt] = __ffs(starts) - 1;
                    starts &= starts - 1u;
                    ts[cnt] = __shfl_sync(0xffffffffu, tl, js[cnt]);
                }
                float4 s0[4], s1[4];
#pragma unroll
                for (int q = 0; q < 4; ++q)
                    if (q < cnt) {
                        s0[q] = row(ts[q]);
                        s1[q] = row(ts[q] + 1);
                    }
#pragma unroll
                for (int q = 0; q < 4; ++q)
                    if (q < cnt) {
                        wt = dot(s0[q]);
                        wt1 = dot(s1[q]);
                        ct = ts[q];
                        if (my_start == js[q]) val = fmaf(a, wt, c * wt1);
                    }
            }
            if (lane < n && a != 0.f) mine[A.pos[k & 0xffffu]] += val;   // distinct pixels within a voxel
            __syncwarp();
        }
    }
    __syncthreads();
    for (int e = threadIdx.x; e < A.np; e += blockDim.x) {
        float s = 0.f;
        for (int w = 0; w < nw; ++w) s += img[(size_t)w * A.np + e];
        part[(int64_t)blockIdx.x * A.np + e] = s;
    }
}

// Adjoint: per voxel, the records' coefficients w[pixel] w0 and w[pixel] w1 are
// summed over each run of equal t; a run adds its lower sum times S~[t] and
// leaves its upper sum pending for knot t + 1 (merged with the next run's lower
// sum when that run is t + 1).  out[v][4l .. 4l + 3] = the lane's sums.
__global__ void k_adj_sub(SubArgs A, const float *__restrict__ w, float *__restrict__ out) {
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31, nw = blockDim.x >> 5;
    const int v = blockIdx.x * nw + warp;
    if (v >= A.R) return;   // warp-uniform
    const bool ql = 4 * lane < A.Q;
    float4 acc = make_float4(0.f, 0.f, 0.f, 0.f);
    auto add_row = [&](int t, float c) {
        if (ql && t >= 0 && c != 0.f) {
            const float4 s = *reinterpret_cast<const float4 *>(A.S + (int64_t)t * A.Q + 4 * lane);
            acc.x = fmaf(c, s.x, acc.x);
            acc.y = fmaf(c, s.y, acc.y);
            acc.z = fmaf(c, s.z, acc.z);
            acc.w = fmaf(c, s.w, acc.w);
        }
    };
    int pt = -1, ct = -1;
    float pc = 0.f, c0 = 0.f, c1 = 0.f;
    auto end_run = [&]() {   // run ct with sums (c0, c1)
        if (ct < 0) return;
        float lo = c0;
        if (pt == ct) lo += pc;
        else add_row(pt, pc);
        add_row(ct, lo);
        pt = ct + 1;
        pc = c1;
    };
    const int64_t b = A.off[(int64_t)v * A.P + A.subset], e = A.off[(int64_t)v * A.P + A.subset + 1];
    for (int64_t r0 = b; r0 < e; r0 += 32) {
        const int n = (int)min((int64_t)32, e - r0);
        uint32_t k = 0u;
        float a = 0.f, c = 0.f;
        if (lane < n) {
            k = A.key[r0 + lane];
            const float wv = w[k & 0xffffu];
            a = wv * A.w0[r0 + lane];
            c = wv * A.w1[r0 + lane];
        }
        for (int j = 0; j < n; ++j) {
            const int t = (int)(__shfl_sync(0xffffffffu, k, j) >> 16);
            const float aj = __shfl_sync(0xffffffffu, a, j), cj = __shfl_sync(0xffffffffu, c, j);
            if (t != ct) {   // warp-uniform
                end_run();
                ct = t;
                c0 = 0.f;
                c1 = 0.f;
            }
            c0 += aj;
            c1 += cj;
        }
    }
    end_run();
    add_row(pt, pc);
    if (ql) *reinterpret_cast<float4 *>(out + (int64_t)v * A.Q + 4 * lane) = acc;
}

// the partial image, 4 rows of FP32 (2 buffers) or 8 of bf16 (4 buffers), the
// buffers' barriers and counters
size_t fwd_sym_smem(int npix, int Bp) { return (size_t)((npix + 3) & ~3) * 4 + 4 * (size_t)Bp * 4 + 64; }

size_t fwd_rec_smem(int npix, int Bp) {
    return (size_t)((npix + 3) & ~3) * 4 + 2 * (size_t)Bp * 4 + 16;
}
size_t adj_rec_smem(int npix, int Bp) {
    return (size_t)((npix + 3) & ~3) * 4 + (size_t)Bp * 4 + (size_t)ADJ_W * ADJ_SQ * 48 + ADJ_W * 16 +
           3 * (size_t)ADJ_T * 4 + ADJ_W * 8;
}

}  // namespace

namespace {

void free_set(RecSet &r) {
    cudaFree(r.off);
    cudaFree(r.key);
    cudaFree(r.w0);
    cudaFree(r.w1);
    r = RecSet();
}

// Count, allocate and fill one record set with P groups per voxel (group of a
// pixel: sub_dev[pixel], with the pixel lists sp_off_dev / sp_pix_dev; all
// pixels in one group when sub_dev is null).  Returns OK with r.P = 0 when the
// device memory is not available.
caxsi_status build_set(caxsi_plan *p, TablePath *T, RecSet &r, int P, const int *sub_dev,
                       const int *sp_off_dev, const int *sp_pix_dev, int wpb) {
    const DevGeo &g = p->dg;
    const int64_t ng = (int64_t)g.R * P;
    int64_t *cnt = nullptr;
    if (cudaMalloc(&cnt, (size_t)ng * sizeof(int64_t)) != cudaSuccess) {
        cudaGetLastError();
        return CAXSI_OK;
    }
    const PairArgs pa = pair_args(p);
    const TabArgs ta = tab_args(T);
    k_rec_count<<<(unsigned)ceil_div64((int64_t)g.R * 32, 256), 256, 8 * P * sizeof(int)>>>(pa, ta, sub_dev, P,
                                                                                          cnt);
    std::vector<int64_t> h(ng + 1);
    if (cudaGetLastError() != cudaSuccess ||
        cudaMemcpy(h.data() + 1, cnt, (size_t)ng * sizeof(int64_t), cudaMemcpyDeviceToHost) != cudaSuccess) {
        cudaFree(cnt);
        return CAXSI_ERR_CUDA;
    }
    cudaFree(cnt);
    // every group's list is padded to a multiple of 4 records (whole 16-byte quads)
    int64_t n_real = 0;
    h[0] = 0;
    for (int64_t k = 0; k < ng; ++k) {
        n_real += h[k + 1];
        h[k + 1] = h[k] + ((h[k + 1] + 3) & ~int64_t(3));
    }
    const int64_t n = h[ng];
    const int64_t nalloc = n > 0 ? n : 4;
    if (cudaMalloc(&r.off, (size_t)(ng + 1) * sizeof(int64_t)) != cudaSuccess ||
        cudaMalloc(&r.key, (size_t)nalloc * sizeof(uint32_t)) != cudaSuccess ||
        cudaMalloc(&r.w0, (size_t)nalloc * sizeof(float)) != cudaSuccess ||
        cudaMalloc(&r.w1, (size_t)nalloc * sizeof(float)) != cudaSuccess) {
        cudaGetLastError();
        free_set(r);
        return CAXSI_OK;
    }
    if (cudaMemcpy(r.off, h.data(), (size_t)(ng + 1) * sizeof(int64_t), cudaMemcpyHostToDevice) != cudaSuccess) {
        free_set(r);
        return CAXSI_ERR_CUDA;
    }
    const size_t smem = (size_t)wpb * (T->B + 1) * sizeof(int);
    if (cudaFuncSetAttribute(k_rec_fill, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem) != cudaSuccess) {
        free_set(r);
        return CAXSI_ERR_CUDA;
    }
    k_rec_fill<<<(unsigned)ceil_div64(g.R, wpb), wpb * 32, smem>>>(pa, ta, wpb, P, sp_off_dev, sp_pix_dev, r.off,
                                                                 r.key, r.w0, r.w1);
    if (cudaGetLastError() != cudaSuccess || cudaDeviceSynchronize() != cudaSuccess) {
        free_set(r);
        return CAXSI_ERR_CUDA;
    }
    r.P = P;
    r.n = n_real;
    p->table_bytes += n * 12 + (ng + 1) * 8;
    return CAXSI_OK;
}

// Warps per block of the fill kernel (its histogram of B + 1 ints per warp must
// fit shared memory), or 0 when records cannot be used: the sizes do not fit the
// 16-bit key fields or the streaming kernels' shared memory.
int fill_warps(const caxsi_plan *p, const TablePath *T) {
    const DevGeo &g = p->dg;
    const int npix = g.M * g.N;
    if (npix > 65536 || T->B > 65535) return 0;
    int smem_max = 0;
    cudaDeviceGetAttribute(&smem_max, cudaDevAttrMaxSharedMemoryPerBlockOptin, p->device);
    const size_t need = fwd_rec_smem(npix, T->Bp) > adj_rec_smem(npix, T->Bp)
                            ? fwd_rec_smem(npix, T->Bp) : adj_rec_smem(npix, T->Bp);
    int wpb = (int)((smem_max - 1024) / ((size_t)(T->B + 1) * 4));
    if (wpb > 8) wpb = 8;
    if ((size_t)smem_max < need || wpb < 1) return 0;
    return wpb;
}

}  // namespace

void records_free(TablePath *T) {
    free_set(T->rec);
    free_set(T->sub);
    cudaFree(T->sym.tt);
    cudaFree(T->sym.tb);
    cudaFree(T->sym.w);
    cudaFree(T->sym.adj_w0_16);
    cudaFree(T->sym.adj_w1_16);
    free_set(T->sym.adj);
    cudaFree(T->sym.adj_seg);
    T->sym = SymSet();
    T->use_records = false;
}

// Build the records of the full operator.  Returns OK without records
// (use_records stays false) when the sizes do not fit the 16-bit key fields or
// shared memory, or when the device memory is not available; the on-the-fly
// table kernels are used then.
caxsi_status records_build(caxsi_plan *p, TablePath *T) {
    const int wpb = fill_warps(p, T);
    if (wpb < 1) return CAXSI_OK;
    caxsi_status st = build_set(p, T, T->rec, 1, nullptr, nullptr, nullptr, wpb);
    if (st != CAXSI_OK || T->rec.P == 0) return st;
    T->use_records = true;
    const DevGeo &g = p->dg;
    int chunks = 2 * p->num_sms;
    if (chunks > g.R) chunks = g.R;
    T->rec_vc = (int)ceil_div64(g.R, chunks);
    T->rec_chunks = (int)ceil_div64(g.R, T->rec_vc);
    return CAXSI_OK;
}

// Build the records grouped by detector subset (sub_host[pixel] in [0, P)),
// replacing an earlier grouping.  Needs the full records (use_records).
caxsi_status records_build_subsets(caxsi_plan *p, TablePath *T, int P, const int32_t *sub_host) {
    if (!T->use_records) return CAXSI_ERR_UNSUPPORTED;
    const DevGeo &g = p->dg;
    const int npix = g.M * g.N;
    free_set(T->sub);
    T->sub_gen = 0;
    // pixel lists of the subsets (counting sort of the pixels by subset)
    std::vector<int> sp_off(P + 1, 0), sp_pix(npix);
    for (int k = 0; k < npix; ++k) sp_off[sub_host[k] + 1]++;
    for (int s = 0; s < P; ++s) sp_off[s + 1] += sp_off[s];
    {
        std::vector<int> fill(sp_off.begin(), sp_off.end() - 1);
        for (int k = 0; k < npix; ++k) sp_pix[fill[sub_host[k]]++] = k;
    }
    int *d_sub = nullptr, *d_off = nullptr, *d_pix = nullptr;
    if (cudaMalloc(&d_sub, npix * sizeof(int)) != cudaSuccess ||
        cudaMalloc(&d_off, (P + 1) * sizeof(int)) != cudaSuccess ||
        cudaMalloc(&d_pix, npix * sizeof(int)) != cudaSuccess) {
        cudaGetLastError();
        cudaFree(d_sub);
        cudaFree(d_off);
        cudaFree(d_pix);
        return CAXSI_ERR_OOM;
    }
    caxsi_status st = CAXSI_OK;
    if (cudaMemcpy(d_sub, sub_host, npix * sizeof(int), cudaMemcpyHostToDevice) != cudaSuccess ||
        cudaMemcpy(d_off, sp_off.data(), (P + 1) * sizeof(int), cudaMemcpyHostToDevice) != cudaSuccess ||
        cudaMemcpy(d_pix, sp_pix.data(), npix * sizeof(int), cudaMemcpyHostToDevice) != cudaSuccess)
        st = CAXSI_ERR_CUDA;
    if (st == CAXSI_OK) st = build_set(p, T, T->sub, P, d_sub, d_off, d_pix, fill_warps(p, T));
    cudaFree(d_off);
    cudaFree(d_pix);
    cudaFree(d_sub);
    if (st == CAXSI_OK && T->sub.P == 0) st = CAXSI_ERR_OOM;
    return st;
}

// bf16 copies of the record weights for the bf16 path (round to nearest even).
__global__ void k_w_to_bf16(const float *__restrict__ x, int64_t n, uint16_t *__restrict__ y) {
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x)
        y[i] = __bfloat16_as_ushort(__float2bfloat16_rn(x[i]));
}

// Allocate and fill a bf16 copy of n FP32 weights; leaves *out null (the bf16 path
// then streams the FP32 weights) when the memory is not there.
caxsi_status bf16_copy(caxsi_plan *p, const float *x, int64_t n, uint16_t **out) {
    *out = nullptr;
    if (n <= 0) return CAXSI_OK;
    if (cudaMalloc(out, (size_t)n * sizeof(uint16_t)) != cudaSuccess) {
        cudaGetLastError();
        *out = nullptr;
        return CAXSI_OK;
    }
    k_w_to_bf16<<<(unsigned)std::min<int64_t>(ceil_div64(n, 256), 8 * (int64_t)p->num_sms), 256>>>(x, n, *out);
    if (cudaGetLastError() != cudaSuccess) {
        cudaFree(*out);
        *out = nullptr;
        return CAXSI_ERR_CUDA;
    }
    p->table_bytes += n * 2;
    return CAXSI_OK;
}

// The adjoint's symmetric lists (SymSet::adj): count, pad to quads, fill sorted by
// t, and find each (pair, knot segment) item's quad range.  Leaves adj.P = 0 (the
// adjoint then streams the ordinary records) when the sizes do not fit the key or
// shared memory, or the device memory is not there.
caxsi_status sym_adj_build(caxsi_plan *p, TablePath *T) {
    const DevGeo &g = p->dg;
    SymSet &y = T->sym;
    const int nq = (g.M / 2) * (g.N / 2);
    if (nq > 8192 || T->B > 16383) return CAXSI_OK;
    // knot segments: about 16 per pair (at least 64 knots each), as long as one
    // segment per warp fits beside the image
    int smem_max = 0;
    cudaDeviceGetAttribute(&smem_max, cudaDevAttrMaxSharedMemoryPerBlockOptin, p->device);
    const int64_t lmax = (((int64_t)smem_max - 512 - 16 * (int64_t)nq) / ((int64_t)SEG_W * 8)) & ~int64_t(7);
    if (lmax < 8) return CAXSI_OK;
    int nseg = std::max((int)ceil_div64(T->Bp, lmax), std::min(16, (int)ceil_div64(T->Bp, 64)));
    const int L = (int)((ceil_div64(T->Bp, nseg) + 7) & ~int64_t(7));
    nseg = (int)ceil_div64(T->Bp, L);
    if (L > lmax || (int64_t)y.R2 * nseg > INT32_MAX) return CAXSI_OK;
    const int wpb = fill_warps(p, T);
    if (wpb < 1) return CAXSI_OK;
    const PairArgs pa = pair_args(p);
    const TabArgs ta = tab_args(T);
    const int64_t ng = y.R2;
    int64_t *cnt = nullptr;
    if (cudaMalloc(&cnt, (size_t)ng * sizeof(int64_t)) != cudaSuccess) {
        cudaGetLastError();
        return CAXSI_OK;
    }
    k_sadj_count<<<(unsigned)ceil_div64(ng * 32, 256), 256>>>(pa, ta, y.R2, cnt);
    std::vector<int64_t> h(ng + 1);
    if (cudaGetLastError() != cudaSuccess ||
        cudaMemcpy(h.data() + 1, cnt, (size_t)ng * sizeof(int64_t), cudaMemcpyDeviceToHost) != cudaSuccess) {
        cudaFree(cnt);
        return CAXSI_ERR_CUDA;
    }
    cudaFree(cnt);
    int64_t n_real = 0;
    h[0] = 0;
    for (int64_t k = 0; k < ng; ++k) {
        n_real += h[k + 1];
        h[k + 1] = h[k] + ((h[k + 1] + 3) & ~int64_t(3));
    }
    const int64_t n = h[ng];
    const int64_t nalloc = n > 0 ? n : 4;
    const int64_t nitems = ng * nseg;
    RecSet &r = y.adj;
    if (cudaMalloc(&r.off, (size_t)(ng + 1) * sizeof(int64_t)) != cudaSuccess ||
        cudaMalloc(&r.key, (size_t)nalloc * sizeof(uint32_t)) != cudaSuccess ||
        cudaMalloc(&r.w0, (size_t)nalloc * sizeof(float)) != cudaSuccess ||
        cudaMalloc(&r.w1, (size_t)nalloc * sizeof(float)) != cudaSuccess ||
        cudaMalloc(&y.adj_seg, (size_t)nitems * sizeof(uint32_t)) != cudaSuccess) {
        cudaGetLastError();
        free_set(r);
        cudaFree(y.adj_seg);
        y.adj_seg = nullptr;
        return CAXSI_OK;
    }
    auto fail = [&]() {
        cudaGetLastError();
        free_set(r);
        cudaFree(y.adj_seg);
        y.adj_seg = nullptr;
        return CAXSI_ERR_CUDA;
    };
    if (cudaMemcpy(r.off, h.data(), (size_t)(ng + 1) * sizeof(int64_t), cudaMemcpyHostToDevice) != cudaSuccess)
        return fail();
    const size_t smem = (size_t)wpb * (T->B + 1) * sizeof(int);
    if (cudaFuncSetAttribute(k_sadj_fill, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem) != cudaSuccess)
        return fail();
    k_sadj_fill<<<(unsigned)ceil_div64(ng, wpb), wpb * 32, smem>>>(pa, ta, y.R2, wpb, r.off, r.key, r.w0, r.w1);
    if (cudaGetLastError() != cudaSuccess) return fail();
    k_sadj_segs<<<(unsigned)ceil_div64(nitems, 256), 256>>>(r.off, r.key, y.R2, nseg, L, y.adj_seg);
    if (cudaGetLastError() != cudaSuccess || cudaDeviceSynchronize() != cudaSuccess) return fail();
    r.P = 1;
    r.n = n_real;
    p->table_bytes += n * 12 + (ng + 1) * 8 + nitems * 4;
    y.adj_L = L;
    y.adj_nseg = nseg;
    caxsi_status st = bf16_copy(p, r.w0, n, &y.adj_w0_16);
    if (st == CAXSI_OK) st = bf16_copy(p, r.w1, n, &y.adj_w1_16);
    if (st == CAXSI_OK && (!y.adj_w0_16 || !y.adj_w1_16)) {   // both or neither
        cudaFree(y.adj_w0_16);
        cudaFree(y.adj_w1_16);
        y.adj_w0_16 = y.adj_w1_16 = nullptr;
    }
    return st;
}

// Build the mirror-symmetric records when the geometry allows them (J, M, N
// even, knots within 16 bits, shared memory for the forward); otherwise leave
// sym.ok false (the forward then streams the ordinary records).
caxsi_status sym_build(caxsi_plan *p, TablePath *T) {
    const DevGeo &g = p->dg;
    if (!T->use_records || g.J % 2 || g.M % 2 || g.N % 2 || T->B > 65535) return CAXSI_OK;
    int smem_max = 0;
    cudaDeviceGetAttribute(&smem_max, cudaDevAttrMaxSharedMemoryPerBlockOptin, p->device);
    if ((size_t)smem_max < fwd_sym_smem(g.M * g.N, T->Bp)) return CAXSI_OK;
    SymSet &y = T->sym;
    y.R2 = g.X * (g.J / 2);
    y.nrec = (g.M / 2) * (g.N / 2);
    const int64_t n = (int64_t)y.R2 * y.nrec;
    if (cudaMalloc(&y.tt, n * sizeof(uint32_t)) != cudaSuccess || cudaMalloc(&y.tb, n) != cudaSuccess ||
        cudaMalloc(&y.w, n * sizeof(float4)) != cudaSuccess) {
        cudaGetLastError();
        cudaFree(y.tt);
        cudaFree(y.tb);
        cudaFree(y.w);
        y = SymSet();
        return CAXSI_OK;
    }
    k_sym_build<<<(unsigned)ceil_div64(n, 256), 256>>>(pair_args(p), tab_args(T), y.R2, y.nrec, y.tt, y.tb, y.w);
    if (cudaGetLastError() != cudaSuccess || cudaDeviceSynchronize() != cudaSuccess) {
        cudaFree(y.tt);
        cudaFree(y.tb);
        cudaFree(y.w);
        y = SymSet();
        return CAXSI_ERR_CUDA;
    }
    // one block per SM (the kernel's shared memory allows one); the partial
    // images fit the forward's buffer, which holds rec_chunks of them
    int chunks = p->num_sms < T->rec_chunks ? p->num_sms : T->rec_chunks;
    if (chunks > y.R2) chunks = y.R2;
    y.vc = (int)ceil_div64(y.R2, chunks);
    y.chunks = (int)ceil_div64(y.R2, y.vc);
    y.ok = true;
    p->table_bytes += n * 21;
    return sym_adj_build(p, T);
}

cudaError_t sym_forward(const caxsi_plan *p, const TablePath *T, float *part, cudaStream_t s, bool w16) {
    const int npix = p->dg.M * p->dg.N;
    const size_t smem = fwd_sym_smem(npix, T->Bp);
    if (w16) {   // the bf16 path: bf16 knot rows (the records keep FP32 weights: bf16 ones measured slower)
        cudaError_t e = cudaFuncSetAttribute(k_fwd_sym<__nv_bfloat16>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                             (int)smem);
        if (e != cudaSuccess) return e;
        k_fwd_sym<__nv_bfloat16><<<T->sym.chunks, RT, smem, s>>>(
            sym_args(p, T), reinterpret_cast<const __nv_bfloat16 *>(T->v16), part, p->err_flag + 1);
        return cudaGetLastError();
    }
    cudaError_t e = cudaFuncSetAttribute(k_fwd_sym<float>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return e;
    k_fwd_sym<float><<<T->sym.chunks, RT, smem, s>>>(sym_args(p, T), T->tab, part, p->err_flag + 1);
    return cudaGetLastError();
}

template <typename OutT, bool W16>
cudaError_t launch_adj_sym(const caxsi_plan *p, const TablePath *T, const float *w, OutT *out, cudaStream_t s) {
    const DevGeo &g = p->dg;
    const SymSet &y = T->sym;
    const size_t smem = adj_sym_smem((g.M / 2) * (g.N / 2), y.adj_L);
    cudaError_t e =
        cudaFuncSetAttribute(k_adj_sym<OutT, W16>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return e;
    SymAdjArgs a;
    a.R2 = y.R2;
    a.J = g.J;
    a.J2 = g.J / 2;
    a.M = g.M;
    a.N = g.N;
    a.Bp = T->Bp;
    a.nseg = y.adj_nseg;
    a.L = y.adj_L;
    a.off = y.adj.off;
    a.seg = y.adj_seg;
    a.key = y.adj.key;
    a.w0 = y.adj.w0;
    a.w1 = y.adj.w1;
    a.w0_16 = y.adj_w0_16;
    a.w1_16 = y.adj_w1_16;
    const int64_t warps = (int64_t)y.R2 * y.adj_nseg;
    const int grid = (int)std::min<int64_t>(p->num_sms, ceil_div64(warps, SEG_W));
    k_adj_sym<OutT, W16><<<grid, SEG_T, smem, s>>>(a, w, out);
    return cudaGetLastError();
}

// out_kind 1 (the bf16 path): bf16 V rows, and bf16 record weights when the plan
// has them; 2 (fp16): fp16 V rows; 0: FP32.
cudaError_t sym_adjoint(const caxsi_plan *p, const TablePath *T, const float *w, int out_kind, cudaStream_t s) {
    if (out_kind == 1) {
        __nv_bfloat16 *out = reinterpret_cast<__nv_bfloat16 *>(T->v16);
        if (T->sym.adj_w0_16) return launch_adj_sym<__nv_bfloat16, true>(p, T, w, out, s);
        return launch_adj_sym<__nv_bfloat16, false>(p, T, w, out, s);
    }
    if (out_kind == 2) return launch_adj_sym<__half, false>(p, T, w, reinterpret_cast<__half *>(T->v16), s);
    return launch_adj_sym<float, false>(p, T, w, T->tab, s);
}

cudaError_t records_forward(const caxsi_plan *p, const TablePath *T, int subset, float *part, cudaStream_t s) {
    const int npix = p->dg.M * p->dg.N;
    const size_t smem = fwd_rec_smem(npix, T->Bp);
    cudaError_t e = cudaFuncSetAttribute(k_fwd_rec<false>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return e;
    k_fwd_rec<false><<<T->rec_chunks, RT, smem, s>>>(rec_args(p, T, subset), T->tab, part, p->err_flag + 1);
    return cudaGetLastError();
}

template <typename OutT>
cudaError_t launch_adj_rec(const caxsi_plan *p, const TablePath *T, int subset, const float *w, OutT *out,
                           cudaStream_t s) {
    const int npix = p->dg.M * p->dg.N;
    const size_t smem = adj_rec_smem(npix, T->Bp);
    cudaError_t e = cudaFuncSetAttribute(k_adj_rec<OutT, false>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                         (int)smem);
    if (e != cudaSuccess) return e;
    k_adj_rec<OutT, false><<<T->rec_chunks, ADJ_T, smem, s>>>(rec_args(p, T, subset), w, out, p->err_flag + 1);
    return cudaGetLastError();
}

// Batched forms: explicit work items (objects' voxel chunks) and table rows.
cudaError_t records_forward_items(const caxsi_plan *p, const TablePath *T, const int4 *items, int n_items,
                                  const float *Wtab, float *part, cudaStream_t s) {
    const int npix = p->dg.M * p->dg.N;
    const size_t smem = fwd_rec_smem(npix, T->Bp);
    cudaError_t e = cudaFuncSetAttribute(k_fwd_rec<true>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return e;
    RecArgs a = rec_args(p, T, -1);
    a.items = items;
    a.n_items = n_items;
    k_fwd_rec<true><<<std::min(n_items, T->rec_chunks), RT, smem, s>>>(a, Wtab, part, p->err_flag + 1);
    return cudaGetLastError();
}

cudaError_t records_adjoint_items(const caxsi_plan *p, const TablePath *T, const int4 *items, int n_items,
                                  const float *w, int64_t w_stride, float *Vtab, cudaStream_t s) {
    const int npix = p->dg.M * p->dg.N;
    const size_t smem = adj_rec_smem(npix, T->Bp);
    cudaError_t e = cudaFuncSetAttribute(k_adj_rec<float, true>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                         (int)smem);
    if (e != cudaSuccess) return e;
    RecArgs a = rec_args(p, T, -1);
    a.items = items;
    a.n_items = n_items;
    a.w_stride = w_stride;
    k_adj_rec<float, true><<<std::min(n_items, T->rec_chunks), ADJ_T, smem, s>>>(a, w, Vtab,
                                                                                p->err_flag + 1);
    return cudaGetLastError();
}

cudaError_t records_adjoint(const caxsi_plan *p, const TablePath *T, int subset, const float *w, int out_kind,
                            cudaStream_t s) {
    if (out_kind == 1)
        return launch_adj_rec(p, T, subset, w, reinterpret_cast<__nv_bfloat16 *>(T->v16), s);
    if (out_kind == 2)
        return launch_adj_rec(p, T, subset, w, reinterpret_cast<__half *>(T->v16), s);
    return launch_adj_rec(p, T, subset, w, T->tab, s);
}

// The sparse subset operators (k_fwd_sub / k_adj_sub) and when they pay: their
// runs of equal t each wait for rows of S~ from L2, so they win only while a
// subset has few records per voxel (measured at paper scale, 64 subsets, 125
// records per voxel and subset: adjoint 0.24 ms, forward 0.29 ms, against about
// 0.55 ms each with the contractions; 8 subsets, 1 000 records: several times
// slower than the contractions).  max_per_voxel: the average records per voxel
// and subset up to which the sparse form is used.  False also when they do not apply (q rows
// over 128 or not whole float4s, unaligned arrays), and the caller contracts.
bool sub_sparse_ok(const caxsi_plan *p, const void *a, const void *b, int max_per_voxel) {
    const int Q = p->dg.Q;
    const TablePath *T = p->table;
    if (!(Q <= 128 && Q % 4 == 0 && T && T->sub.P > 0)) return false;
    if (T->sub.n > (int64_t)max_per_voxel * p->dg.R * T->sub.P) return false;
    return ((reinterpret_cast<uintptr_t>(a) | reinterpret_cast<uintptr_t>(b)) & 15) == 0;
}

static SubArgs sub_args(const caxsi_plan *p, const TablePath *T, int subset) {
    SubArgs a;
    a.R = p->dg.R;
    a.Q = p->dg.Q;
    a.P = T->sub.P;
    a.subset = subset;
    a.np = p->sub_off[subset + 1] - p->sub_off[subset];
    a.off = T->sub.off;
    a.key = T->sub.key;
    a.w0 = T->sub.w0;
    a.w1 = T->sub.w1;
    a.S = T->S;
    a.pos = p->sub_pos;
    return a;
}

cudaError_t sub_forward_sparse(const caxsi_plan *p, const TablePath *T, int subset, const float *f, float *g,
                               cudaStream_t s, bool &done) {
    done = false;
    const SubArgs a = sub_args(p, T, subset);
    const int64_t npix = (int64_t)p->dg.M * p->dg.N;
    int warps = 8;
    while (warps > 1 && (size_t)warps * a.np * 4 > (size_t)160 * 1024) warps /= 2;
    if ((size_t)warps * a.np * 4 > (size_t)160 * 1024) return cudaSuccess;   // too large: not done
    cudaError_t e = cudaMemsetAsync(g, 0, npix * sizeof(float), s);
    if (e != cudaSuccess || a.np == 0) {
        done = e == cudaSuccess;
        return e;
    }
    // blocks: about 4 per SM, their partial images within the forward scratch
    int blocks = (int)ceil_div64(a.R, warps);
    if (blocks > 4 * p->num_sms) blocks = 4 * p->num_sms;
    const int64_t cap = (int64_t)std::max(T->rec_chunks, T->fwd_chunks) * npix;
    if ((int64_t)blocks * a.np > cap) blocks = (int)(cap / a.np);
    const size_t smem = (size_t)warps * a.np * sizeof(float);
    e = cudaFuncSetAttribute(k_fwd_sub, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return e;
    k_fwd_sub<<<blocks, warps * 32, smem, s>>>(a, f, T->fwd_part);
    if ((e = cudaGetLastError()) != cudaSuccess) return e;
    e = launch_sum_list(T->fwd_part, blocks, a.np, p->sub_pix + p->sub_off[subset], g, s);
    done = e == cudaSuccess;
    return e;
}

cudaError_t sub_adjoint_sparse(const caxsi_plan *p, const TablePath *T, int subset, const float *w, float *f,
                               cudaStream_t s) {
    const SubArgs a = sub_args(p, T, subset);
    k_adj_sub<<<(unsigned)ceil_div64(a.R, 8), 256, 0, s>>>(a, w, f);
    return cudaGetLastError();
}
