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
// counting sort, one warp per voxel, deterministic).  The forward accumulates
// one voxel at a time into a shared-memory detector image (a pixel occurs at
// most once per voxel, so there are no conflicts).  The adjoint reduces runs
// of equal t with a warp-level segmented scan; only the runs at warp-segment
// boundaries are combined afterwards, in a fixed order.  Neither kernel uses
// atomics; both are deterministic.
//
// Record layout (structure of arrays, 12 bytes per record):
//   key = pixel | (t << 16) (uint32), w0 (float), w1 (float).
#include <cuda_bf16.h>
#include <cuda_fp16.h>

#include <vector>

#include "internal.cuh"
#include "pairgeo.cuh"
#include "table.cuh"

namespace {

constexpr int RT = 1024;                 // threads of the streaming kernels
constexpr uint32_t SENT = 0xffffffffu;   // "no run" marker
constexpr uint32_t WAIT_LIMIT = 1u << 24;
constexpr int PREF = 8;                  // record batches loaded ahead per warp

struct RecArgs {
    int R, npix, Bp, B;
    const int64_t *off;
    const uint32_t *key;
    const float *w0, *w1;
};

RecArgs rec_args(const caxsi_plan *p, const TablePath *T) {
    RecArgs a;
    a.R = p->dg.R;
    a.npix = p->dg.M * p->dg.N;
    a.Bp = T->Bp;
    a.B = T->B;
    a.off = T->rec_off;
    a.key = T->rec_key;
    a.w0 = T->rec_w0;
    a.w1 = T->rec_w1;
    return a;
}

// ---- one pair, as the on-the-fly table kernels evaluate it --------------------
struct PairRec {
    bool ok;
    int t;
    float w0, w1;
};

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

// Count the records of each voxel (one warp per voxel).
__global__ void k_rec_count(PairArgs A, TabArgs T, int64_t *cnt) {
    const DevGeo &g = A.g;
    const int lane = threadIdx.x & 31;
    const int v = (blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    if (v >= g.R) return;
    const float u_first = T.knots[0].x, u_last = T.knots[T.B - 1].x;
    const int i = v / g.J, j = v - i * g.J;
    const float4 vx = A.vox[v];
    const int npix = g.M * g.N;
    int c = 0;
    for (int p = lane; p < npix; p += 32) {
        const int m = p / g.N, n = p - m * g.N;
        c += pair_record(A, T, u_first, u_last, v, i, j, vx, m, n).ok ? 1 : 0;
    }
    for (int o = 16; o > 0; o >>= 1) c += __shfl_down_sync(0xffffffffu, c, o);
    if (lane == 0) cnt[v] = c;
}

// Fill the records of each voxel, sorted by (t, pixel): a histogram of t, its
// exclusive scan, then placement in pixel order with ranks among equal t.
__global__ void k_rec_fill(PairArgs A, TabArgs T, int wpb, const int64_t *off, uint32_t *key,
                           float *w0, float *w1) {
    extern __shared__ __align__(16) int rec_smem[];
    const DevGeo &g = A.g;
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int v = blockIdx.x * wpb + warp;
    if (warp >= wpb || v >= g.R) return;
    int *hist = rec_smem + warp * (T.B + 1);
    for (int t = lane; t <= T.B; t += 32) hist[t] = 0;
    __syncwarp();
    const float u_first = T.knots[0].x, u_last = T.knots[T.B - 1].x;
    const int i = v / g.J, j = v - i * g.J;
    const float4 vx = A.vox[v];
    const int npix = g.M * g.N;
    for (int p = lane; p < npix; p += 32) {
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
    const int64_t base = off[v];
    const unsigned lt = (1u << lane) - 1u;
    for (int pb = 0; pb < npix; pb += 32) {
        const int p = pb + lane;
        PairRec r;
        r.ok = false;
        if (p < npix) {
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
// Bounded wait: false if the phase did not complete within WAIT_LIMIT polls.
__device__ __forceinline__ bool mbar_wait(uint64_t *bar, uint32_t parity) {
    for (uint32_t k = 0; k < WAIT_LIMIT; ++k)
        if (mbar_try_wait(bar, parity)) return true;
    return false;
}

// Forward streaming kernel.  Block = 1024 threads, a chunk of voxels; the
// detector image accumulates in shared memory; each voxel's Wtab row arrives
// by a TMA bulk copy, double-buffered one voxel ahead.
__global__ void __launch_bounds__(RT, 1)
k_fwd_rec(RecArgs A, const float *__restrict__ Wtab, float *__restrict__ part, int vc, int *err) {
    extern __shared__ __align__(128) unsigned char smem_raw[];
    const int npix_al = (A.npix + 3) & ~3;
    float *g_s = reinterpret_cast<float *>(smem_raw);
    float *wbuf0 = g_s + npix_al;
    float *wbuf1 = wbuf0 + A.Bp;
    uint64_t *bar = reinterpret_cast<uint64_t *>(wbuf1 + A.Bp);
    const int tid = threadIdx.x;
    const int v0 = blockIdx.x * vc;
    const int v1 = min(v0 + vc, A.R);
    const uint32_t row_bytes = (uint32_t)A.Bp * 4u;
    for (int p = tid; p < A.npix; p += RT) g_s[p] = 0.f;
    if (tid == 0) {
        mbar_init(&bar[0], 1);
        mbar_init(&bar[1], 1);
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
        if (v0 < v1) {
            mbar_expect_tx(&bar[0], row_bytes);
            bulk_g2s(wbuf0, Wtab + (int64_t)v0 * A.Bp, row_bytes, &bar[0]);
        }
    }
    __syncthreads();
    bool ok = true;
    uint32_t ph0 = 0u, ph1 = 0u;   // mbarrier phase parity of each buffer
    for (int v = v0; v < v1; ++v) {
        const int buf = (v - v0) & 1;
        float *w_s = buf ? wbuf1 : wbuf0;
        if (tid == 0 && v + 1 < v1) {
            // the other buffer was last read by voxel v - 1, finished at the barrier below
            asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
            mbar_expect_tx(&bar[buf ^ 1], row_bytes);
            bulk_g2s(buf ? wbuf0 : wbuf1, Wtab + (int64_t)(v + 1) * A.Bp, row_bytes, &bar[buf ^ 1]);
        }
        const int late = mbar_wait(&bar[buf], buf ? ph1 : ph0) ? 0 : 1;
        if (__syncthreads_or(late)) {   // block-uniform decision
            ok = false;
            break;
        }
        if (buf) ph1 ^= 1u; else ph0 ^= 1u;
        const int64_t b = A.off[v], e = A.off[v + 1];
        for (int64_t q = b + tid; q < e; q += RT) {
            const uint32_t k = A.key[q];
            const int t = (int)(k >> 16);
            const float val = fmaf(A.w0[q], w_s[t], A.w1[q] * w_s[t + 1]);
            g_s[k & 0xffffu] += val;
        }
        __syncthreads();
    }
    if (!ok) {
        // a copy did not land in time: report, drain the copies this block issued, stop
        if (tid == 0) {
            atomicExch(err, 1);
            mbar_wait(&bar[0], ph0);
            mbar_wait(&bar[1], ph1);
        }
        return;
    }
    float *dst = part + (int64_t)blockIdx.x * A.npix;
    for (int p = tid; p < A.npix; p += RT) dst[p] = g_s[p];
}

struct Side {
    uint32_t t;
    float lo, hi;
};

// Adjoint streaming kernel.  Block = 1024 threads, a chunk of voxels; the
// input image w is staged once in shared memory.  Per voxel, warp k reduces a
// contiguous segment of the voxel's (t-sorted) records: runs of equal t are
// summed by a segmented warp scan; complete runs inside the segment are owned
// by the warp and stored directly, the first and last runs of each segment go
// to side slots that one thread adds afterwards in warp order.  Then
// V[t] = LO[t] + HI[t - 1] is written to Vtab.
__device__ __forceinline__ void store_v(float *p, float x) { *p = x; }
__device__ __forceinline__ void store_v(__nv_bfloat16 *p, float x) { *p = __float2bfloat16_rn(x); }
__device__ __forceinline__ void store_v(__half *p, float x) { *p = __float2half_rn(x); }

template <typename OutT>
__global__ void __launch_bounds__(RT, 1)
k_adj_rec(RecArgs A, const float *__restrict__ w, OutT *__restrict__ Vtab, float *__restrict__ Vlo, int vc) {
    extern __shared__ __align__(128) unsigned char smem_raw[];
    const int npix_al = (A.npix + 3) & ~3;
    float *w_s = reinterpret_cast<float *>(smem_raw);
    float *LO = w_s + npix_al;
    float *HI = LO + A.Bp;
    Side *side = reinterpret_cast<Side *>(HI + A.Bp);   // [32][2]
    Side *comp = side + 64;                              // [64] compacted side slots
    const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
    const int v0 = blockIdx.x * vc;
    const int v1 = min(v0 + vc, A.R);
    for (int p = tid; p < A.npix; p += RT) w_s[p] = w[p];
    for (int v = v0; v < v1; ++v) {
        for (int t = tid; t < A.Bp; t += RT) {
            LO[t] = 0.f;
            HI[t] = 0.f;
        }
        __syncthreads();
        const int64_t b = A.off[v], e = A.off[v + 1];
        const int64_t n = e - b;
        const int64_t seg = ((n + 31) / 32 + 31) / 32 * 32;
        const int64_t sb = min(e, b + warp * seg), se = min(e, sb + seg);
        uint32_t ct = SENT;       // carried run (warp-uniform)
        float clo = 0.f, chi = 0.f;
        bool first_pending = true;  // the segment's first run goes to side[warp][0]
        const int nbat = (int)((se - sb + 31) / 32);
        for (int g0 = 0; g0 < nbat; g0 += PREF) {
            // issue the loads of PREF batches before reducing any of them
            uint32_t kk[PREF];
            float a0[PREF], a1[PREF];
#pragma unroll
            for (int bb = 0; bb < PREF; ++bb) {
                const int64_t q = sb + (int64_t)(g0 + bb) * 32 + lane;
                kk[bb] = SENT;
                a0[bb] = a1[bb] = 0.f;
                if (g0 + bb < nbat && q < se) {
                    kk[bb] = A.key[q];
                    a0[bb] = A.w0[q];
                    a1[bb] = A.w1[q];
                }
            }
#pragma unroll
            for (int bb = 0; bb < PREF; ++bb) {
                if (g0 + bb >= nbat) break;
                const bool valid = kk[bb] != SENT;
                uint32_t t = SENT;
                float lo = 0.f, hi = 0.f;
                if (valid) {
                    t = kk[bb] >> 16;
                    const float x = w_s[kk[bb] & 0xffffu];
                    lo = a0[bb] * x;
                    hi = a1[bb] * x;
                }
                const uint32_t t0 = __shfl_sync(0xffffffffu, t, 0);
                if (ct != SENT && t0 != ct) {
                    // the carried run is complete
                    if (lane == 0) {
                        if (first_pending) side[warp * 2] = Side{ct, clo, chi};
                        else { LO[ct] = clo; HI[ct] = chi; }
                    }
                    first_pending = false;
                    ct = SENT;
                }
                if (ct != SENT && lane == 0) {
                    lo += clo;
                    hi += chi;
                }
                // inclusive segmented scan over equal t (records are sorted, runs contiguous)
#pragma unroll
                for (int o = 1; o < 32; o <<= 1) {
                    const float ylo = __shfl_up_sync(0xffffffffu, lo, o);
                    const float yhi = __shfl_up_sync(0xffffffffu, hi, o);
                    const uint32_t yt = __shfl_up_sync(0xffffffffu, t, o);
                    if (lane >= o && yt == t) {
                        lo += ylo;
                        hi += yhi;
                    }
                }
                // the run holding the batch's last valid record may continue into the
                // next batch: it becomes the carry; every run ending before it is complete
                const int last = 31 - __clz(__ballot_sync(0xffffffffu, valid));
                const uint32_t tn = __shfl_down_sync(0xffffffffu, t, 1);
                const bool run_end = valid && (lane < last) && (tn != t);
                const unsigned ends = __ballot_sync(0xffffffffu, run_end);
                if (run_end) {
                    const bool is_first = first_pending && ((ends & ((1u << lane) - 1u)) == 0);
                    if (is_first) side[warp * 2] = Side{t, lo, hi};
                    else { LO[t] = lo; HI[t] = hi; }
                }
                if (ends) first_pending = false;
                ct = __shfl_sync(0xffffffffu, t, last);
                clo = __shfl_sync(0xffffffffu, lo, last);
                chi = __shfl_sync(0xffffffffu, hi, last);
            }
        }
        if (lane == 0) {
            if (ct != SENT && first_pending) {
                side[warp * 2] = Side{ct, clo, chi};
                side[warp * 2 + 1] = Side{SENT, 0.f, 0.f};
            } else {
                if (first_pending) side[warp * 2] = Side{SENT, 0.f, 0.f};
                side[warp * 2 + 1] = ct != SENT ? Side{ct, clo, chi} : Side{SENT, 0.f, 0.f};
            }
        }
        __syncthreads();
        if (warp == 0) {
            // The side slots, read in warp order, have nondecreasing t once the empty
            // ones are dropped: compact them (order kept), then sum runs of equal t
            // with the same carry-based segmented scan and add each run once.
            int nvalid = 0;
#pragma unroll
            for (int r = 0; r < 2; ++r) {
                const Side sd = side[32 * r + lane];
                const bool val = sd.t != SENT;
                const unsigned bal = __ballot_sync(0xffffffffu, val);
                if (val) comp[nvalid + __popc(bal & ((1u << lane) - 1u))] = sd;
                nvalid += __popc(bal);
            }
            __syncwarp();
            uint32_t mt = SENT;
            float mlo = 0.f, mhi = 0.f;
            for (int r = 0; r * 32 < nvalid; ++r) {
                const int idx = 32 * r + lane;
                const bool valid = idx < nvalid;
                uint32_t t = SENT;
                float lo = 0.f, hi = 0.f;
                if (valid) {
                    const Side sd = comp[idx];
                    t = sd.t;
                    lo = sd.lo;
                    hi = sd.hi;
                }
                const uint32_t t0 = __shfl_sync(0xffffffffu, t, 0);
                if (mt != SENT && t0 != mt) {
                    if (lane == 0) { LO[mt] += mlo; HI[mt] += mhi; }
                    mt = SENT;
                }
                if (mt != SENT && lane == 0) { lo += mlo; hi += mhi; }
#pragma unroll
                for (int o = 1; o < 32; o <<= 1) {
                    const float ylo = __shfl_up_sync(0xffffffffu, lo, o);
                    const float yhi = __shfl_up_sync(0xffffffffu, hi, o);
                    const uint32_t yt = __shfl_up_sync(0xffffffffu, t, o);
                    if (lane >= o && yt == t) { lo += ylo; hi += yhi; }
                }
                const int last = 31 - __clz(__ballot_sync(0xffffffffu, valid));
                const uint32_t tn = __shfl_down_sync(0xffffffffu, t, 1);
                if (valid && lane < last && tn != t) { LO[t] += lo; HI[t] += hi; }
                mt = __shfl_sync(0xffffffffu, t, last);
                mlo = __shfl_sync(0xffffffffu, lo, last);
                mhi = __shfl_sync(0xffffffffu, hi, last);
            }
            if (mt != SENT && lane == 0) { LO[mt] += mlo; HI[mt] += mhi; }
        }
        __syncthreads();
        OutT *vrow = Vtab + (int64_t)v * A.Bp;
        if (Vlo) {
            float *lrow = Vlo + (int64_t)v * A.Bp;
            for (int t = tid; t < A.B; t += RT) {
                float h, l;
                tf32_split(LO[t] + (t > 0 ? HI[t - 1] : 0.f), h, l);
                store_v(vrow + t, h);
                lrow[t] = l;
            }
        } else {
            for (int t = tid; t < A.B; t += RT) store_v(vrow + t, LO[t] + (t > 0 ? HI[t - 1] : 0.f));
        }
        __syncthreads();
    }
}

size_t fwd_rec_smem(int npix, int Bp) {
    return (size_t)((npix + 3) & ~3) * 4 + 2 * (size_t)Bp * 4 + 16;
}
size_t adj_rec_smem(int npix, int Bp) {
    return (size_t)((npix + 3) & ~3) * 4 + 2 * (size_t)Bp * 4 + 128 * sizeof(Side);
}

}  // namespace

void records_free(TablePath *T) {
    cudaFree(T->rec_off);
    cudaFree(T->rec_key);
    cudaFree(T->rec_w0);
    cudaFree(T->rec_w1);
    T->rec_off = nullptr;
    T->rec_key = nullptr;
    T->rec_w0 = T->rec_w1 = nullptr;
    T->use_records = false;
}

// Build the records.  Returns OK without records (use_records stays false) when
// the sizes do not fit the 16-bit key fields or shared memory, or when the
// device memory is not available; the on-the-fly table kernels are used then.
caxsi_status records_build(caxsi_plan *p, TablePath *T) {
    const DevGeo &g = p->dg;
    const int npix = g.M * g.N;
    if (npix > 65536 || T->B > 65535) return CAXSI_OK;
    int smem_max = 0;
    cudaDeviceGetAttribute(&smem_max, cudaDevAttrMaxSharedMemoryPerBlockOptin, p->device);
    const size_t need = fwd_rec_smem(npix, T->Bp) > adj_rec_smem(npix, T->Bp)
                            ? fwd_rec_smem(npix, T->Bp) : adj_rec_smem(npix, T->Bp);
    int wpb = (int)((smem_max - 1024) / ((size_t)(T->B + 1) * 4));
    if (wpb > 8) wpb = 8;
    if ((size_t)smem_max < need || wpb < 1) return CAXSI_OK;

    int64_t *cnt = nullptr;
    if (cudaMalloc(&cnt, (size_t)g.R * sizeof(int64_t)) != cudaSuccess) return CAXSI_OK;
    const PairArgs pa = pair_args(p);
    const TabArgs ta = tab_args(T);
    k_rec_count<<<(unsigned)ceil_div64((int64_t)g.R * 32, 256), 256>>>(pa, ta, cnt);
    std::vector<int64_t> h(g.R + 1);
    if (cudaGetLastError() != cudaSuccess ||
        cudaMemcpy(h.data() + 1, cnt, (size_t)g.R * sizeof(int64_t), cudaMemcpyDeviceToHost) != cudaSuccess) {
        cudaFree(cnt);
        return CAXSI_ERR_CUDA;
    }
    cudaFree(cnt);
    h[0] = 0;
    for (int v = 0; v < g.R; ++v) h[v + 1] += h[v];
    const int64_t n = h[g.R];
    if (cudaMalloc(&T->rec_off, (size_t)(g.R + 1) * sizeof(int64_t)) != cudaSuccess ||
        cudaMalloc(&T->rec_key, (size_t)(n > 0 ? n : 1) * sizeof(uint32_t)) != cudaSuccess ||
        cudaMalloc(&T->rec_w0, (size_t)(n > 0 ? n : 1) * sizeof(float)) != cudaSuccess ||
        cudaMalloc(&T->rec_w1, (size_t)(n > 0 ? n : 1) * sizeof(float)) != cudaSuccess) {
        cudaGetLastError();
        records_free(T);
        return CAXSI_OK;
    }
    cudaMemcpy(T->rec_off, h.data(), (size_t)(g.R + 1) * sizeof(int64_t), cudaMemcpyHostToDevice);
    const size_t smem = (size_t)wpb * (T->B + 1) * sizeof(int);
    if (cudaFuncSetAttribute(k_rec_fill, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem) != cudaSuccess) {
        records_free(T);
        return CAXSI_ERR_CUDA;
    }
    k_rec_fill<<<(unsigned)ceil_div64(g.R, wpb), wpb * 32, smem>>>(pa, ta, wpb, T->rec_off, T->rec_key,
                                                                 T->rec_w0, T->rec_w1);
    if (cudaGetLastError() != cudaSuccess || cudaDeviceSynchronize() != cudaSuccess) {
        records_free(T);
        return CAXSI_ERR_CUDA;
    }
    T->n_rec = n;
    T->use_records = true;
    int chunks = 2 * p->num_sms;
    if (chunks > g.R) chunks = g.R;
    T->rec_vc = (int)ceil_div64(g.R, chunks);
    T->rec_chunks = (int)ceil_div64(g.R, T->rec_vc);
    p->table_bytes += n * 12 + (int64_t)(g.R + 1) * 8;
    return CAXSI_OK;
}

cudaError_t records_forward(const caxsi_plan *p, const TablePath *T, float *part, cudaStream_t s) {
    const int npix = p->dg.M * p->dg.N;
    const size_t smem = fwd_rec_smem(npix, T->Bp);
    cudaError_t e = cudaFuncSetAttribute(k_fwd_rec, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return e;
    k_fwd_rec<<<T->rec_chunks, RT, smem, s>>>(rec_args(p, T), T->tab, part, T->rec_vc, p->err_flag + 1);
    return cudaGetLastError();
}

template <typename OutT>
cudaError_t launch_adj_rec(const caxsi_plan *p, const TablePath *T, const float *w, OutT *out,
                           float *lo, cudaStream_t s) {
    const int npix = p->dg.M * p->dg.N;
    const size_t smem = adj_rec_smem(npix, T->Bp);
    cudaError_t e = cudaFuncSetAttribute(k_adj_rec<OutT>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return e;
    k_adj_rec<OutT><<<T->rec_chunks, RT, smem, s>>>(rec_args(p, T), w, out, lo, T->rec_vc);
    return cudaGetLastError();
}

cudaError_t records_adjoint(const caxsi_plan *p, const TablePath *T, const float *w, int out_kind,
                            cudaStream_t s) {
    if (out_kind == 1) return launch_adj_rec(p, T, w, reinterpret_cast<__nv_bfloat16 *>(T->v16), (float *)nullptr, s);
    if (out_kind == 2) return launch_adj_rec(p, T, w, reinterpret_cast<__half *>(T->v16), (float *)nullptr, s);
    return launch_adj_rec(p, T, w, T->tab, (float *)nullptr, s);
}
