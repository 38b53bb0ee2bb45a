// Objects of different geometries evaluated together (caxsi_multi_*): the
// direct FP32 forward and adjoint of every object of the set in one persistent
// kernel launch each.
//
// Work items.  Forward: (object, voxel chunk, detector tile of 8 x 32 pixels),
// the unit of one block of the single-plan kernel; adjoint: (object, voxel,
// detector row range), the unit of one warp of the single-plan kernel.  The
// objects' chunking is their plans' own, so each item's partial result is the
// one the single-plan call computes.
//
// Queue.  A launch has as many blocks as fit on the SMs at once; each block
// (forward) or warp (adjoint) takes the next item index with one atomic add on
// a counter until the items run out, so objects of very different sizes share
// the launch without a tail of idle SMs.  Nothing waits on anything: a pop is a
// single atomic, never a poll.
//
// Deterministic sums.  An item writes its partial result into its plan's
// partial buffer (the single call's layout), publishes it with a memory fence
// and counts itself done on the output region's counter; the item that
// completes a region (the last to arrive, whichever it is) sums the region's
// partials in ascending chunk / row-range order -- the order of the single
// call's summation kernel -- and writes the output.  So each object's result
// is bit-identical to caxsi_forward / caxsi_adjoint on its plan, whatever the
// order in which items run.
#include <math.h>

#include <algorithm>
#include <new>
#include <vector>

#include "direct_body.cuh"

namespace {

using namespace direct_impl;

// One object of the set, as the kernels see it.
struct MultiObj {
    Tables T;          // the object's geometry and plan tables
    int64_t f_off;     // its f in the packed object array (floats)
    int64_t g_off;     // its detector image in the packed image array (floats)
    float *fpart;      // its plan's forward partial images [chunks][M*N]
    float *apart;      // its plan's adjoint partials [split][R*Q] (split > 1)
    int vc, chunks, tiles_n, tiles;   // forward: voxels per chunk, chunks, tiles per row, tiles
    int split, rps;    // adjoint: detector row ranges per voxel, rows per range
    int cnt_f;         // first forward counter (one per detector tile)
    int cnt_a;         // first adjoint counter (one per voxel when split > 1)
};

// Largest b with first[b] <= it (first[0] = 0, first ascending, n entries).
__device__ __forceinline__ int find_object(const int64_t *__restrict__ first, int n, int64_t it) {
    int lo = 0, hi = n - 1;
    while (lo < hi) {
        const int mid = (lo + hi + 1) >> 1;
        if (first[mid] <= it) lo = mid;
        else hi = mid - 1;
    }
    return lo;
}

__global__ void __launch_bounds__(FWD_THREADS)
k_fwd_direct_multi(const MultiObj *__restrict__ objs, const int64_t *__restrict__ first, int nobj,
                   const float *__restrict__ f, float *__restrict__ g, unsigned *queue, unsigned *cnt) {
    extern __shared__ __align__(16) unsigned char smem_raw[];
    __shared__ MultiObj s_o;
    __shared__ int64_t s_item;
    __shared__ int s_obj;
    __shared__ bool s_last;
    const int tid = threadIdx.x;
    const int64_t total = first[nobj];
    for (;;) {
        __syncthreads();   // the previous item is done with s_o and the staging buffers
        if (tid == 0) {
            const int64_t it = (int64_t)atomicAdd(queue, 1u);
            s_item = it;
            if (it < total) {
                const int b = find_object(first, nobj, it);
                s_obj = b;
                s_o = objs[b];
            }
        }
        __syncthreads();
        const int64_t it = s_item;
        if (it >= total) break;
        const MultiObj &o = s_o;
        const int local = (int)(it - first[s_obj]);
        const int chunk = local / o.tiles, tile = local - chunk * o.tiles;
        // a register copy of the tables: the body's loops then keep the geometry in
        // registers instead of re-reading it around its shared-memory stores
        const Tables T = o.T;
        fwd_direct_body<false>(T, f + o.f_off, o.fpart, o.vc, o.tiles_n, nullptr, 0, tile, chunk, smem_raw);
        // publish this chunk's partial tile; the last chunk of the tile sums them all
        __threadfence();
        __syncthreads();
        if (tid == 0) s_last = atomicAdd(&cnt[o.cnt_f + tile], 1u) == (unsigned)(o.chunks - 1);
        __syncthreads();
        if (s_last) {
            __threadfence();
            const DevGeo &d = o.T.g;
            const int warp = tid >> 5, lane = tid & 31;
            const int tm = tile / o.tiles_n, tn = tile - tm * o.tiles_n;
            const int m = tm * FWD_WARPS + warp, n = tn * 32 + lane;
            if (m < d.M && n < d.N) {
                const int64_t npix = (int64_t)d.M * d.N, pix = (int64_t)m * d.N + n;
                float sum = 0.f;
                for (int c = 0; c < o.chunks; ++c) sum += __ldcg(o.fpart + c * npix + pix);
                g[o.g_off + pix] = sum;
            }
        }
    }
}

// Warp-level items; each warp keeps its object's description and energy table
// in its own slice of shared memory: [ADJ_WARPS] x ([kmax] float2, [(qmax+3) x 32 + 64] float).
__global__ void __launch_bounds__(ADJ_WARPS * 32)
k_adj_direct_multi(const MultiObj *__restrict__ objs, const int64_t *__restrict__ first, int nobj,
                   const float *__restrict__ w, float *__restrict__ f, unsigned *queue, unsigned *cnt, int kmax,
                   int qmax) {
    extern __shared__ __align__(16) unsigned char smem_raw[];
    __shared__ MultiObj s_o[ADJ_WARPS];
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int ke = (kmax + 1) & ~1;
    const size_t per_warp = (size_t)ke * sizeof(float2) + adj_warp_floats(qmax) * sizeof(float);
    float2 *s_en = reinterpret_cast<float2 *>(smem_raw + warp * per_warp);
    float *acc = reinterpret_cast<float *>(s_en + ke);
    const int64_t total = first[nobj];
    int cur = -1;
    for (;;) {
        int64_t it = 0;
        if (lane == 0) it = (int64_t)atomicAdd(queue, 1u);
        it = __shfl_sync(0xffffffffu, it, 0);
        if (it >= total) break;
        const int b = find_object(first, nobj, it);
        if (b != cur) {
            // the object's description and energy table into the warp's slice
            const int words = (int)(sizeof(MultiObj) / sizeof(int));
            const int *src = reinterpret_cast<const int *>(objs + b);
            int *dst = reinterpret_cast<int *>(&s_o[warp]);
            for (int k = lane; k < words; k += 32) dst[k] = src[k];
            __syncwarp();
            for (int k = lane; k < s_o[warp].T.g.K; k += 32) s_en[k] = s_o[warp].T.energy[k];
            cur = b;
        }
        const MultiObj &o = s_o[warp];
        const DevGeo &d = o.T.g;
        const int QB = d.Q + 3;
        for (int k = lane; k < QB * 32; k += 32) acc[k] = 0.f;
        __syncwarp();
        const int local = (int)(it - first[b]);
        const int v = local / o.split, sp = local - v * o.split;
        float *out = o.split > 1 ? o.apart : f + o.f_off;
        const Tables T = o.T;   // in registers (see the forward)
        adj_direct_body<false>(T, w + o.g_off, out, o.rps, nullptr, 0, v, sp, s_en, acc, lane);
        if (o.split > 1) {
            // publish this row range's partial row; the last range of the voxel sums them
            __threadfence();
            __syncwarp();
            unsigned last = 0;
            if (lane == 0) last = atomicAdd(&cnt[o.cnt_a + v], 1u) == (unsigned)(o.split - 1);
            last = __shfl_sync(0xffffffffu, last, 0);
            if (last) {
                __threadfence();
                const int64_t nf = (int64_t)d.R * d.Q;
                for (int l = lane; l < d.Q; l += 32) {
                    float sum = 0.f;
                    for (int c = 0; c < o.split; ++c) sum += __ldcg(o.apart + c * nf + (int64_t)v * d.Q + l);
                    f[o.f_off + (int64_t)v * d.Q + l] = sum;
                }
            }
        }
        __syncwarp();   // the warp's slice is read no further before the next item overwrites it
    }
}

}  // namespace

struct caxsi_multi {
    int device = 0;
    int n = 0;
    int num_sms = 0;
    std::vector<caxsi_plan *> plans;
    std::vector<int64_t> f_off, g_off;   // [n + 1] packed offsets
    int64_t f_len = 0, g_len = 0;
    int kmax = 0, qmax = 0;
    size_t smem_fwd = 0, smem_adj = 0;
    int grid_fwd = 0, grid_adj = 0;
    int n_cnt = 0;                 // counters: [0] forward queue, [1] adjoint queue, then regions
    MultiObj *objs = nullptr;      // [n] device
    int64_t *first_f = nullptr;    // [n + 1] device: first forward item of each object
    int64_t *first_a = nullptr;    // [n + 1] device: first adjoint item of each object
    unsigned *cnt = nullptr;       // [n_cnt] device
    DevGeo *geos = nullptr;        // [n] device: the objects' geometries (update kernels)
    int64_t *vox0 = nullptr;       // [n + 1] device: first voxel of each object in the packed order
    int64_t *foff = nullptr;       // [n + 1] device: first element of each object's f
    int64_t n_vox = 0;             // voxels of all objects
    float *vjp_scratch = nullptr;  // [2 f_len] device: reverse-mode scratch of the update
};

namespace {

void free_multi(caxsi_multi *m) {
    if (!m) return;
    cudaFree(m->objs);
    cudaFree(m->first_f);
    cudaFree(m->first_a);
    cudaFree(m->cnt);
    cudaFree(m->geos);
    cudaFree(m->vox0);
    cudaFree(m->foff);
    cudaFree(m->vjp_scratch);
    delete m;
}

struct DevGuard {
    int prev = -1;
    bool ok = true;
    explicit DevGuard(int dev) {
        if (cudaGetDevice(&prev) != cudaSuccess) { ok = false; return; }
        if (prev != dev && cudaSetDevice(dev) != cudaSuccess) ok = false;
    }
    ~DevGuard() {
        int cur;
        if (prev >= 0 && cudaGetDevice(&cur) == cudaSuccess && cur != prev) cudaSetDevice(prev);
    }
};

}  // namespace

// update kernels over the packed objects (recon.cu)
caxsi_status multi_update(const DevGeo *geos, const int64_t *vox0, const int64_t *foff, int nobj, int64_t n_vox,
                          int qmax, const float *f, const float *b1, const float *b2, float beta, float delta,
                          float *out, cudaStream_t s);
caxsi_status multi_update_vjp(const DevGeo *geos, const int64_t *foff, int nobj, const float *f, const float *b1,
                              const float *b2, float beta, float delta, const float *gx, float *gf, float *gb2,
                              float *scratch, int64_t n, cudaStream_t s);

extern "C" {

caxsi_status caxsi_multi_create(caxsi_plan *const *plans, int n_objects, caxsi_multi **out) {
    if (!plans || !out || n_objects < 1 || n_objects > CAXSI_MAX_MULTI) return CAXSI_ERR_INVALID;
    for (int b = 0; b < n_objects; ++b)
        if (!plans[b] || plans[b]->device != plans[0]->device) return CAXSI_ERR_INVALID;
    // each object's partial results go to its plan's scratch: a plan may serve one object only
    {
        std::vector<const caxsi_plan *> sorted(plans, plans + n_objects);
        std::sort(sorted.begin(), sorted.end());
        if (std::adjacent_find(sorted.begin(), sorted.end()) != sorted.end()) return CAXSI_ERR_INVALID;
    }
    caxsi_multi *m = new (std::nothrow) caxsi_multi();
    if (!m) return CAXSI_ERR_OOM;
    m->device = plans[0]->device;
    m->n = n_objects;
    m->num_sms = plans[0]->num_sms;
    m->plans.assign(plans, plans + n_objects);
    DevGuard dg(m->device);
    if (!dg.ok) {
        free_multi(m);
        return CAXSI_ERR_CUDA;
    }
    std::vector<MultiObj> objs(n_objects);
    std::vector<int64_t> first_f(n_objects + 1, 0), first_a(n_objects + 1, 0), vox0(n_objects + 1, 0);
    std::vector<DevGeo> geos(n_objects);
    m->f_off.assign(n_objects + 1, 0);
    m->g_off.assign(n_objects + 1, 0);
    int n_cnt = 2;
    for (int b = 0; b < n_objects; ++b) {
        const caxsi_plan *p = plans[b];
        const DevGeo &d = p->dg;
        MultiObj &o = objs[b];
        o.T = tables_of(p);
        o.f_off = m->f_off[b];
        o.g_off = m->g_off[b];
        o.fpart = p->fwd_part;
        o.apart = p->adj_part;
        o.vc = p->fwd_vc;
        o.chunks = p->fwd_chunks;
        o.tiles_n = (int)ceil_div64(d.N, 32);
        o.tiles = (int)ceil_div64(d.M, FWD_WARPS) * o.tiles_n;
        o.split = p->adj_split;
        o.rps = (int)ceil_div64(d.M, o.split);
        o.cnt_f = n_cnt;
        n_cnt += o.tiles;
        o.cnt_a = n_cnt;
        if (o.split > 1) n_cnt += d.R;
        first_f[b + 1] = first_f[b] + (int64_t)o.tiles * o.chunks;
        first_a[b + 1] = first_a[b] + (int64_t)d.R * o.split;
        vox0[b + 1] = vox0[b] + d.R;
        geos[b] = d;
        m->f_off[b + 1] = m->f_off[b] + (int64_t)d.R * d.Q;
        m->g_off[b + 1] = m->g_off[b] + (int64_t)d.M * d.N;
        m->kmax = std::max(m->kmax, d.K);
        m->qmax = std::max(m->qmax, d.Q);
        m->smem_fwd = std::max(m->smem_fwd, fwd_smem(d));
    }
    m->f_len = m->f_off[n_objects];
    m->n_vox = vox0[n_objects];
    m->g_len = m->g_off[n_objects];
    // the queues count items in 32 bits
    if (first_f[n_objects] >= (int64_t)1 << 31 || first_a[n_objects] >= (int64_t)1 << 31) {
        free_multi(m);
        return CAXSI_ERR_INVALID;
    }
    m->n_cnt = n_cnt;
    m->smem_adj = (size_t)ADJ_WARPS * (((m->kmax + 1) & ~1) * sizeof(float2) + adj_warp_floats(m->qmax) * sizeof(float));
    int smem_max = 0;
    cudaDeviceGetAttribute(&smem_max, cudaDevAttrMaxSharedMemoryPerBlockOptin, m->device);
    const size_t static_fwd = sizeof(MultiObj) + 64, static_adj = ADJ_WARPS * sizeof(MultiObj);
    if ((size_t)smem_max < m->smem_fwd + static_fwd || (size_t)smem_max < m->smem_adj + static_adj) {
        free_multi(m);
        return CAXSI_ERR_UNSUPPORTED;
    }
    caxsi_status st = CAXSI_OK;
    auto fail = [&](cudaError_t e) {
        st = e == cudaErrorMemoryAllocation ? CAXSI_ERR_OOM : CAXSI_ERR_CUDA;
        return st;
    };
    cudaError_t e;
    if ((e = cudaFuncSetAttribute(k_fwd_direct_multi, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                  (int)m->smem_fwd)) != cudaSuccess ||
        (e = cudaFuncSetAttribute(k_adj_direct_multi, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                  (int)m->smem_adj)) != cudaSuccess) {
        fail(e);
        free_multi(m);
        return st;
    }
    int occ_f = 0, occ_a = 0;
    cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ_f, k_fwd_direct_multi, FWD_THREADS, m->smem_fwd);
    cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ_a, k_adj_direct_multi, ADJ_WARPS * 32, m->smem_adj);
    m->grid_fwd = m->num_sms * std::max(1, occ_f);
    m->grid_adj = m->num_sms * std::max(1, occ_a);
    if ((e = cudaMalloc(&m->objs, n_objects * sizeof(MultiObj))) != cudaSuccess ||
        (e = cudaMalloc(&m->first_f, (n_objects + 1) * sizeof(int64_t))) != cudaSuccess ||
        (e = cudaMalloc(&m->first_a, (n_objects + 1) * sizeof(int64_t))) != cudaSuccess ||
        (e = cudaMalloc(&m->cnt, n_cnt * sizeof(unsigned))) != cudaSuccess ||
        (e = cudaMalloc(&m->geos, n_objects * sizeof(DevGeo))) != cudaSuccess ||
        (e = cudaMalloc(&m->vox0, (n_objects + 1) * sizeof(int64_t))) != cudaSuccess ||
        (e = cudaMalloc(&m->foff, (n_objects + 1) * sizeof(int64_t))) != cudaSuccess ||
        (e = cudaMemcpy(m->objs, objs.data(), n_objects * sizeof(MultiObj), cudaMemcpyHostToDevice)) != cudaSuccess ||
        (e = cudaMemcpy(m->first_f, first_f.data(), (n_objects + 1) * sizeof(int64_t), cudaMemcpyHostToDevice)) !=
            cudaSuccess ||
        (e = cudaMemcpy(m->first_a, first_a.data(), (n_objects + 1) * sizeof(int64_t), cudaMemcpyHostToDevice)) !=
            cudaSuccess ||
        (e = cudaMemcpy(m->geos, geos.data(), n_objects * sizeof(DevGeo), cudaMemcpyHostToDevice)) != cudaSuccess ||
        (e = cudaMemcpy(m->vox0, vox0.data(), (n_objects + 1) * sizeof(int64_t), cudaMemcpyHostToDevice)) !=
            cudaSuccess ||
        (e = cudaMemcpy(m->foff, m->f_off.data(), (n_objects + 1) * sizeof(int64_t), cudaMemcpyHostToDevice)) !=
            cudaSuccess) {
        fail(e);
        free_multi(m);
        return st;
    }
    *out = m;
    return CAXSI_OK;
}

void caxsi_multi_destroy(caxsi_multi *m) {
    if (!m) return;
    DevGuard dg(m->device);
    cudaDeviceSynchronize();
    free_multi(m);
}

caxsi_status caxsi_multi_forward(caxsi_multi *m, const float *f_dev, int64_t f_len, float *g_dev, int64_t g_len,
                                 int path, void *stream) {
    if (!m || !f_dev || !g_dev || f_len != m->f_len || g_len != m->g_len) return CAXSI_ERR_INVALID;
    if (path < CAXSI_PATH_DIRECT || path > CAXSI_PATH_TABLE_FP16) return CAXSI_ERR_INVALID;
    if (path != CAXSI_PATH_DIRECT) return CAXSI_ERR_UNSUPPORTED;
    DevGuard dg(m->device);
    if (!dg.ok) return CAXSI_ERR_CUDA;
    cudaStream_t s = (cudaStream_t)stream;
    caxsi_plan *p0 = m->plans[0];
    p0->launches = 0;
    CAXSI_CUDA_TRY(cudaMemsetAsync(m->cnt, 0, m->n_cnt * sizeof(unsigned), s));
    {
        CAXSI_PROF(p0, "fwd_direct_multi", s);
        k_fwd_direct_multi<<<m->grid_fwd, FWD_THREADS, m->smem_fwd, s>>>(m->objs, m->first_f, m->n, f_dev, g_dev,
                                                                         m->cnt, m->cnt);
    }
    CAXSI_LAUNCH_CHECK(p0);
    return CAXSI_OK;
}

caxsi_status caxsi_multi_adjoint(caxsi_multi *m, const float *w_dev, int64_t w_len, float *f_dev, int64_t f_len,
                                 int path, void *stream) {
    if (!m || !w_dev || !f_dev || w_len != m->g_len || f_len != m->f_len) return CAXSI_ERR_INVALID;
    if (path < CAXSI_PATH_DIRECT || path > CAXSI_PATH_TABLE_FP16) return CAXSI_ERR_INVALID;
    if (path != CAXSI_PATH_DIRECT) return CAXSI_ERR_UNSUPPORTED;
    DevGuard dg(m->device);
    if (!dg.ok) return CAXSI_ERR_CUDA;
    cudaStream_t s = (cudaStream_t)stream;
    caxsi_plan *p0 = m->plans[0];
    p0->launches = 0;
    CAXSI_CUDA_TRY(cudaMemsetAsync(m->cnt, 0, m->n_cnt * sizeof(unsigned), s));
    {
        CAXSI_PROF(p0, "adj_direct_multi", s);
        k_adj_direct_multi<<<m->grid_adj, ADJ_WARPS * 32, m->smem_adj, s>>>(m->objs, m->first_a, m->n, w_dev, f_dev,
                                                                            m->cnt + 1, m->cnt, m->kmax, m->qmax);
    }
    CAXSI_LAUNCH_CHECK(p0);
    return CAXSI_OK;
}

caxsi_status caxsi_multi_em_update(caxsi_multi *m, const float *f_dev, const float *b1_dev, const float *b2_dev,
                                   float beta, float delta, float *f_out_dev, int64_t f_len, void *stream) {
    if (!m || !f_dev || !b1_dev || !b2_dev || !f_out_dev || f_len != m->f_len) return CAXSI_ERR_INVALID;
    if (!isfinite(beta) || beta < 0.f || !isfinite(delta) || delta < 0.f) return CAXSI_ERR_INVALID;
    const uintptr_t a = reinterpret_cast<uintptr_t>(f_dev), o = reinterpret_cast<uintptr_t>(f_out_dev);
    const uintptr_t len = (uintptr_t)f_len * sizeof(float);
    if (o < a + len && a < o + len) return CAXSI_ERR_INVALID;   // the stencil reads f while f_out is written
    DevGuard dg(m->device);
    if (!dg.ok) return CAXSI_ERR_CUDA;
    caxsi_plan *p0 = m->plans[0];
    p0->launches = 0;
    caxsi_status st;
    {
        CAXSI_PROF(p0, "em_update_multi", (cudaStream_t)stream);
        st = multi_update(m->geos, m->vox0, m->foff, m->n, m->n_vox, m->qmax, f_dev, b1_dev, b2_dev, beta, delta,
                          f_out_dev, (cudaStream_t)stream);
    }
    if (st == CAXSI_OK) p0->launches++;
    return st;
}

caxsi_status caxsi_multi_em_update_vjp(caxsi_multi *m, const float *f_dev, const float *b1_dev, const float *b2_dev,
                                       float beta, float delta, const float *grad_out_dev, float *grad_f_dev,
                                       float *grad_b2_dev, int64_t f_len, void *stream) {
    if (!m || !f_dev || !b1_dev || !b2_dev || !grad_out_dev || !grad_f_dev || !grad_b2_dev || f_len != m->f_len)
        return CAXSI_ERR_INVALID;
    if (!isfinite(beta) || beta < 0.f || !isfinite(delta) || delta < 0.f) return CAXSI_ERR_INVALID;
    const uintptr_t len = (uintptr_t)f_len * sizeof(float);
    auto ov = [&](const void *x, const void *y) {
        const uintptr_t a = reinterpret_cast<uintptr_t>(x), b = reinterpret_cast<uintptr_t>(y);
        return a < b + len && b < a + len;
    };
    for (const void *outp : {(const void *)grad_f_dev, (const void *)grad_b2_dev})
        for (const void *in : {(const void *)f_dev, (const void *)b1_dev, (const void *)b2_dev,
                               (const void *)grad_out_dev})
            if (ov(outp, in)) return CAXSI_ERR_INVALID;
    if (ov(grad_f_dev, grad_b2_dev)) return CAXSI_ERR_INVALID;
    DevGuard dg(m->device);
    if (!dg.ok) return CAXSI_ERR_CUDA;
    if (!m->vjp_scratch) CAXSI_CUDA_TRY(cudaMalloc(&m->vjp_scratch, 2 * (size_t)m->f_len * sizeof(float)));
    caxsi_plan *p0 = m->plans[0];
    p0->launches = 0;
    caxsi_status st;
    {
        CAXSI_PROF(p0, "em_update_vjp_multi", (cudaStream_t)stream);
        st = multi_update_vjp(m->geos, m->foff, m->n, f_dev, b1_dev, b2_dev, beta, delta, grad_out_dev, grad_f_dev,
                              grad_b2_dev, m->vjp_scratch, f_len, (cudaStream_t)stream);
    }
    if (st == CAXSI_OK) p0->launches += 2;
    return st;
}

caxsi_status caxsi_multi_layout(const caxsi_multi *m, int64_t *f_offsets, int64_t *g_offsets) {
    if (!m || !f_offsets || !g_offsets) return CAXSI_ERR_INVALID;
    for (int b = 0; b <= m->n; ++b) {
        f_offsets[b] = m->f_off[b];
        g_offsets[b] = m->g_off[b];
    }
    return CAXSI_OK;
}

}  // extern "C"
