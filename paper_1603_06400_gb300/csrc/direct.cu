// Direct FP32 evaluation of the forward model (Eq. 3-4, Algorithm 1) and its
// transpose (Algorithm 3): every (voxel, pixel) pair computes its scatter
// angle and sums the K energy bins of the source spectrum.
//
// Forward: a block owns a tile of 8 detector rows x 32 columns (one warp per
// row, one lane per pixel) and a chunk of voxels; the chunk's q rows are
// staged in shared memory as (f_l, f_{l+1} - f_l) pairs so that one 8-byte
// load gives both interpolation nodes.  Each chunk writes a private partial
// image; a second kernel sums the partials in a fixed order (deterministic,
// no atomics).
//
// Adjoint: a warp owns one voxel (optionally a range of detector rows of it);
// lanes walk the pixels; every lane scatters its energy terms into a
// lane-private row of Q+3 q bins in shared memory laid out [bin][lane] (bank
// = lane, so the scatter is conflict-free), and the 32 private rows are
// summed at the end with a rotated read (also conflict-free).  No atomics.
//
// Subset operators (ordered subsets, Sec. VI): both kernels take a list of
// detector pixels instead of the whole detector (LIST): the forward gives one
// thread to each listed pixel and writes compact partial sums, which are summed
// and scattered to the listed pixels; the adjoint's lanes walk the list.  The
// cost of a subset operator is then that of its pairs.
#include <mutex>

#include "direct_body.cuh"

namespace {

using namespace direct_impl;

template <bool LIST>
__global__ void __launch_bounds__(FWD_THREADS)
k_fwd_direct(Tables T, const float *__restrict__ f, float *__restrict__ part, int vc, int tiles_n,
             const int *__restrict__ list, int np) {
    extern __shared__ __align__(16) unsigned char smem_raw[];
    fwd_direct_body<LIST>(T, f, part, vc, tiles_n, list, np, blockIdx.x, blockIdx.y, smem_raw);
}

// out[list[e]] = sum_c part[c * np + e], c ascending: the listed pixels' sums of
// the compact partial images.
__global__ void k_sum_list(const float *__restrict__ part, int nparts, int np, const int *__restrict__ list,
                           float *__restrict__ out) {
    const int e = blockIdx.x * blockDim.x + threadIdx.x;
    if (e >= np) return;
    float s = 0.f;
    for (int c = 0; c < nparts; ++c) s += part[(int64_t)c * np + e];
    out[list[e]] = s;
}

// out[idx] = sum_c part[c * stride + idx], c ascending (the loads of 32 terms are
// issued before they are added, in the same order).
__global__ void k_sum_parts(const float *__restrict__ part, int nparts, int64_t stride,
                            float *__restrict__ out, int64_t n) {
    int64_t idx = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (idx >= n) return;
    float s = 0.f;
    int c = 0;
    for (; c + 32 <= nparts; c += 32) {
        float v[32];
#pragma unroll
        for (int k = 0; k < 32; ++k) v[k] = part[(int64_t)(c + k) * stride + idx];
#pragma unroll
        for (int k = 0; k < 32; ++k) s += v[k];
    }
    for (; c < nparts; ++c) s += part[(int64_t)c * stride + idx];
    out[idx] = s;
}


template <bool LIST>
__global__ void __launch_bounds__(ADJ_WARPS * 32)
k_adj_direct(Tables T, const float *__restrict__ w, float *__restrict__ out, int split,
             int rows_per_split, const int *__restrict__ list, int np) {
    extern __shared__ __align__(16) unsigned char smem_raw[];
    const DevGeo &g = T.g;
    const int QB = g.Q + 3;  // bins l' = l + 1 in [0, Q + 2]; 1..Q are real
    float2 *s_en = reinterpret_cast<float2 *>(smem_raw);
    float *s_acc = reinterpret_cast<float *>(s_en + ((g.K + 1) & ~1));

    const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
    const int item = blockIdx.x * ADJ_WARPS + warp;
    const int v = item / split, sp = item - (item / split) * split;
    for (int k = tid; k < g.K; k += blockDim.x) s_en[k] = T.energy[k];
    float *acc = s_acc + (int64_t)warp * adj_warp_floats(g.Q);
    for (int b = lane; b < QB * 32; b += 32) acc[b] = 0.f;
    __syncthreads();
    if (v >= g.R) return;
    adj_direct_body<LIST>(T, w, out, rows_per_split, list, np, v, sp, s_en, acc, lane);
}


}  // namespace

cudaError_t launch_sum_list(const float *part, int nparts, int np, const int *list, float *g, cudaStream_t s) {
    k_sum_list<<<(unsigned)ceil_div64(np, 256), 256, 0, s>>>(part, nparts, np, list, g);
    return cudaGetLastError();
}

cudaError_t launch_sum_parts(const float *part, int nparts, int64_t stride, float *out,
                             int64_t n, cudaStream_t s) {
    k_sum_parts<<<(unsigned)ceil_div64(n, 256), 256, 0, s>>>(part, nparts, stride, out, n);
    return cudaGetLastError();
}

void direct_configure(caxsi_plan *p) {
    const DevGeo &g = p->dg;
    const int tiles = (int)(ceil_div64(g.M, FWD_WARPS) * ceil_div64(g.N, 32));
    const int target = 16 * p->num_sms;
    int chunks = (int)ceil_div64(target, tiles);
    if (chunks > g.R) chunks = g.R;
    int vc = (int)ceil_div64(g.R, chunks);
    if (vc < 8) vc = 8;
    p->fwd_vc = vc;
    p->fwd_chunks = (int)ceil_div64(g.R, vc);
    int split = (int)ceil_div64(16 * p->num_sms, g.R);
    if (split > g.M) split = g.M;
    if (split < 1) split = 1;
    int rps = (int)ceil_div64(g.M, split);
    p->adj_split = (int)ceil_div64(g.M, rps);
}

size_t direct_fwd_smem(const caxsi_plan *p) { return fwd_smem(p->dg); }
size_t direct_adj_smem(const caxsi_plan *p) { return adj_smem(p->dg); }

caxsi_status direct_forward(caxsi_plan *p, const float *f, float *g_out, cudaStream_t s) {
    if (p->online_mask) return symmask_forward(p, f, g_out, s);
    const DevGeo &g = p->dg;
    const int tiles_n = (int)ceil_div64(g.N, 32);
    const int tiles = (int)ceil_div64(g.M, FWD_WARPS) * tiles_n;
    const size_t sm = fwd_smem(g);
    CAXSI_CUDA_TRY(cudaFuncSetAttribute(k_fwd_direct<false>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm));
    dim3 grid(tiles, p->fwd_chunks);
    {
        CAXSI_PROF(p, "fwd_direct", s);
        k_fwd_direct<false><<<grid, FWD_THREADS, sm, s>>>(tables_of(p), f, p->fwd_part, p->fwd_vc, tiles_n, nullptr, 0);
    }
    CAXSI_LAUNCH_CHECK(p);
    const int64_t npix = (int64_t)g.M * g.N;
    {
        CAXSI_PROF(p, "sum_parts", s);
        k_sum_parts<<<(unsigned)ceil_div64(npix, 256), 256, 0, s>>>(p->fwd_part, p->fwd_chunks, npix, g_out, npix);
    }
    CAXSI_LAUNCH_CHECK(p);
    return CAXSI_OK;
}

caxsi_status direct_adjoint(caxsi_plan *p, const float *w, float *f_out, cudaStream_t s) {
    if (p->online_mask) return symmask_adjoint(p, w, f_out, s);
    const DevGeo &g = p->dg;
    const size_t sm = adj_smem(g);
    CAXSI_CUDA_TRY(cudaFuncSetAttribute(k_adj_direct<false>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm));
    const int split = p->adj_split;
    const int rps = (int)ceil_div64(g.M, split);
    const int64_t items = (int64_t)g.R * split;
    float *dst = split > 1 ? p->adj_part : f_out;
    {
        CAXSI_PROF(p, "adj_direct", s);
        k_adj_direct<false><<<(unsigned)ceil_div64(items, ADJ_WARPS), ADJ_WARPS * 32, sm, s>>>(tables_of(p), w, dst,
                                                                                          split, rps, nullptr, 0);
    }
    CAXSI_LAUNCH_CHECK(p);
    if (split > 1) {
        const int64_t nf = (int64_t)g.R * g.Q;
        {
            CAXSI_PROF(p, "sum_parts", s);
            k_sum_parts<<<(unsigned)ceil_div64(nf, 256), 256, 0, s>>>(p->adj_part, split, nf, f_out, nf);
        }
        CAXSI_LAUNCH_CHECK(p);
    }
    return CAXSI_OK;
}

// Subset operators: the pixels sub_pix[sub_off[subset] .. sub_off[subset + 1]).
caxsi_status direct_forward_subset(caxsi_plan *p, const float *f, float *g_out, int subset, cudaStream_t s) {
    const DevGeo &g = p->dg;
    const int np = p->sub_off[subset + 1] - p->sub_off[subset];
    const int *list = p->sub_pix + p->sub_off[subset];
    const int64_t npix = (int64_t)g.M * g.N;
    CAXSI_CUDA_TRY(cudaMemsetAsync(g_out, 0, npix * sizeof(float), s));
    if (np == 0) return CAXSI_OK;
    // voxel chunks so that about 4 blocks per SM run; their compact partial
    // images fit the plan's forward scratch (fwd_chunks full images)
    const int xb = (int)ceil_div64(np, FWD_THREADS);
    int chunks = (int)ceil_div64(4 * p->num_sms, xb);
    if (chunks > g.R) chunks = g.R;
    if ((int64_t)chunks * np > (int64_t)p->fwd_chunks * npix) chunks = (int)((int64_t)p->fwd_chunks * npix / np);
    const int vc = (int)ceil_div64(g.R, chunks);
    chunks = (int)ceil_div64(g.R, vc);
    const size_t sm = fwd_smem(g);
    CAXSI_CUDA_TRY(cudaFuncSetAttribute(k_fwd_direct<true>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm));
    {
        CAXSI_PROF(p, "fwd_direct_subset", s);
        k_fwd_direct<true><<<dim3(xb, chunks), FWD_THREADS, sm, s>>>(tables_of(p), f, p->fwd_part, vc, 0, list, np);
    }
    CAXSI_LAUNCH_CHECK(p);
    {
        CAXSI_PROF(p, "sum_list", s);
        k_sum_list<<<(unsigned)ceil_div64(np, 256), 256, 0, s>>>(p->fwd_part, chunks, np, list, g_out);
    }
    CAXSI_LAUNCH_CHECK(p);
    return CAXSI_OK;
}

caxsi_status direct_adjoint_subset(caxsi_plan *p, const float *w, float *f_out, int subset, cudaStream_t s) {
    const DevGeo &g = p->dg;
    const int np = p->sub_off[subset + 1] - p->sub_off[subset];
    const int *list = p->sub_pix + p->sub_off[subset];
    const size_t sm = adj_smem(g);
    CAXSI_CUDA_TRY(cudaFuncSetAttribute(k_adj_direct<true>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm));
    {
        CAXSI_PROF(p, "adj_direct_subset", s);
        k_adj_direct<true><<<(unsigned)ceil_div64(g.R, ADJ_WARPS), ADJ_WARPS * 32, sm, s>>>(tables_of(p), w, f_out, 1,
                                                                                         g.M, list, np);
    }
    CAXSI_LAUNCH_CHECK(p);
    return CAXSI_OK;
}

// ---------------------------------------------------------------------------
// Forward model with scratch in a static device array (allocates nothing).
//
// The chunked forward above keeps its per-chunk partial images in plan-owned
// scratch.  This variant keeps them in a fixed file-scope device array instead,
// so a call performs no device allocation of any kind: it is for callers that
// must not allocate device memory at the point of the call -- for example code
// running while another thread captures a CUDA graph in global capture mode
// (where cudaMalloc fails), real-time loops that forbid allocation after
// start-up, or hosts whose memory pool owns all device memory.
// ---------------------------------------------------------------------------
namespace {

// Partial images of the forward chunks; every GPU that loads the library holds
// this array until the process exits.
static __device__ __align__(256) float g_static_fwd_scratch[CAXSI_STATIC_SCRATCH_FLOATS];

// Device address of the array, looked up once per device (with that device
// current) on the first call that uses the device.
std::mutex g_static_scratch_mu;
float *g_static_scratch_ptr[CAXSI_MAX_DEVICES] = {};

cudaError_t static_scratch_address(int dev, float **out) {
    if (dev < 0 || dev >= CAXSI_MAX_DEVICES) return cudaErrorInvalidDevice;
    std::lock_guard<std::mutex> lk(g_static_scratch_mu);
    if (!g_static_scratch_ptr[dev]) {
        void *ptr = nullptr;
        cudaError_t e = cudaGetSymbolAddress(&ptr, g_static_fwd_scratch);
        if (e != cudaSuccess) return e;
        g_static_scratch_ptr[dev] = static_cast<float *>(ptr);
    }
    *out = g_static_scratch_ptr[dev];
    return cudaSuccess;
}

}  // namespace

caxsi_status direct_forward_static_scratch(caxsi_plan *p, const float *f, float *g_out,
                                           cudaStream_t s) {
    const DevGeo &g = p->dg;
    const int64_t npix = (int64_t)g.M * g.N;
    const int64_t max_chunks = (int64_t)CAXSI_STATIC_SCRATCH_FLOATS / npix;
    if (max_chunks < 1) return CAXSI_ERR_SCRATCH_LIMIT;
    int chunks = p->fwd_chunks < max_chunks ? p->fwd_chunks : (int)max_chunks;
    const int vc = (int)ceil_div64(g.R, chunks);
    chunks = (int)ceil_div64(g.R, vc);
    float *part = nullptr;
    CAXSI_CUDA_TRY(static_scratch_address(p->device, &part));
    const int tiles_n = (int)ceil_div64(g.N, 32);
    const int tiles = (int)ceil_div64(g.M, FWD_WARPS) * tiles_n;
    const size_t sm = fwd_smem(g);
    CAXSI_CUDA_TRY(cudaFuncSetAttribute(k_fwd_direct<false>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm));
    // every chunk overwrites its whole partial image, so nothing needs clearing
    k_fwd_direct<false><<<dim3(tiles, chunks), FWD_THREADS, sm, s>>>(tables_of(p), f, part, vc, tiles_n, nullptr, 0);
    CAXSI_LAUNCH_CHECK(p);
    k_sum_parts<<<(unsigned)ceil_div64(npix, 256), 256, 0, s>>>(part, chunks, npix, g_out, npix);
    CAXSI_LAUNCH_CHECK(p);
    return CAXSI_OK;
}
