// C ABI entry points: validation, plan ownership, dispatch.
#include <math.h>
#include <new>
#include <string.h>

#include "internal.cuh"

size_t direct_fwd_smem(const caxsi_plan *p);
size_t direct_adj_smem(const caxsi_plan *p);

namespace {

// Makes the plan's device current for the duration of a call.
struct DeviceGuard {
    int prev = -1;
    bool ok = true;
    explicit DeviceGuard(int dev) {
        if (cudaGetDevice(&prev) != cudaSuccess) { ok = false; return; }
        if (prev != dev && cudaSetDevice(dev) != cudaSuccess) ok = false;
    }
    ~DeviceGuard() {
        int cur;
        if (prev >= 0 && cudaGetDevice(&cur) == cudaSuccess && cur != prev) cudaSetDevice(prev);
    }
};

bool finite_pos(double v) { return isfinite(v) && v > 0.0; }

caxsi_status validate(const caxsi_geometry *g) {
    if (g->X < 1 || g->J < 1 || g->M < 1 || g->N < 1 || g->K < 1 || g->Q < 2 || g->rho_y < 1)
        return CAXSI_ERR_INVALID;
    if (g->K > CAXSI_MAX_K || g->mask_rows < 1 || g->mask_cols < 1) return CAXSI_ERR_INVALID;
    if (!finite_pos(g->dx) || !finite_pos(g->p_y) || !finite_pos(g->p_z) ||
        !finite_pos(g->mask_cell) || !finite_pos(g->hc) || !finite_pos(g->E_min))
        return CAXSI_ERR_INVALID;
    if (!isfinite(g->x_center) || !isfinite(g->X_det) || !isfinite(g->X_mask) ||
        !isfinite(g->q_min) || !isfinite(g->q_max) || !isfinite(g->E_max) || !isfinite(g->C) ||
        !isfinite(g->mask_y0) || !isfinite(g->mask_z0))
        return CAXSI_ERR_INVALID;
    if (!(g->q_max > g->q_min) || !(g->E_max > g->E_min)) return CAXSI_ERR_INVALID;
    const double x_lo = g->x_center - 0.5 * (g->X - 1) * g->dx;
    const double x_hi = g->x_center + 0.5 * (g->X - 1) * g->dx;
    if (!(x_lo > 0.0) || !(x_hi < g->X_mask) || !(g->X_mask < g->X_det)) return CAXSI_ERR_INVALID;
    // sizes: every table index below 2^31 per dimension product used in int arithmetic
    const double R = (double)g->X * g->J;
    if (R * g->Q > 2e9 || (double)g->M * g->N > 2e9 ||
        (double)g->J * g->rho_y + g->N > 1e7 || (double)g->N > 4e6)
        return CAXSI_ERR_INVALID;
    return CAXSI_OK;
}

void free_plan(caxsi_plan *p) {
    if (!p) return;
    for (auto &r : p->prof.recs) { cudaEventDestroy(r.a); cudaEventDestroy(r.b); }
    for (auto e : p->prof.pool) cudaEventDestroy(e);
    table_destroy(p);
    cudaFree(p->vox);
    cudaFree(p->zrow);
    cudaFree(p->god);
    cudaFree(p->tbits);
    cudaFree(p->mask01);
    cudaFree(p->energy);
    cudaFree(p->fwd_part);
    cudaFree(p->adj_part);
    cudaFree(p->gtmp);
    cudaFree(p->ratio);
    cudaFree(p->ones);
    for (int k = 0; k < 4; ++k) cudaFree(p->b1[k]);
    for (int k = 0; k < 4; ++k) cudaFree(p->b1_sub[k]);
    cudaFree(p->sub_pix);
    cudaFree(p->sub_of_pix);
    cudaFree(p->sub_pos);
    cudaFree(p->vjp_scratch);
    cudaFree(p->b2);
    cudaFree(p->fnew);
    cudaFree(p->nll_part);
    cudaFree(p->nll_dev);
    cudaFree(p->err_flag);
    cudaFree(p->stage_in);
    cudaFree(p->stage_out);
    if (p->copy_stream) {
        cudaEventDestroy(p->pipe_ev[0]);
        cudaEventDestroy(p->pipe_ev[1]);
        cudaStreamDestroy(p->copy_stream);
    }
    delete p;
}

__global__ void k_fill(float *a, float v, int64_t n) {
    int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i < n) a[i] = v;
}

caxsi_status alloc_scratch(caxsi_plan *p) {
    const DevGeo &g = p->dg;
    const int64_t npix = (int64_t)g.M * g.N, nf = (int64_t)g.R * g.Q;
    CAXSI_CUDA_TRY(cudaMalloc(&p->fwd_part, (size_t)p->fwd_chunks * npix * sizeof(float)));
    if (p->adj_split > 1)
        CAXSI_CUDA_TRY(cudaMalloc(&p->adj_part, (size_t)p->adj_split * nf * sizeof(float)));
    CAXSI_CUDA_TRY(cudaMalloc(&p->gtmp, npix * sizeof(float)));
    CAXSI_CUDA_TRY(cudaMalloc(&p->ratio, npix * sizeof(float)));
    CAXSI_CUDA_TRY(cudaMalloc(&p->ones, npix * sizeof(float)));
    CAXSI_CUDA_TRY(cudaMalloc(&p->b2, nf * sizeof(float)));
    CAXSI_CUDA_TRY(cudaMalloc(&p->fnew, nf * sizeof(float)));
    p->nll_blocks = (int)(ceil_div64(npix, NLL_THREADS) < 2 * p->num_sms ? ceil_div64(npix, NLL_THREADS)
                                                                         : 2 * p->num_sms);
    if (p->nll_blocks < 1) p->nll_blocks = 1;
    CAXSI_CUDA_TRY(cudaMalloc(&p->nll_part, p->nll_blocks * sizeof(double)));
    CAXSI_CUDA_TRY(cudaMalloc(&p->nll_dev, sizeof(double)));
    CAXSI_CUDA_TRY(cudaMalloc(&p->err_flag, 3 * sizeof(int)));
    CAXSI_CUDA_TRY(cudaMemset(p->err_flag, 0, 3 * sizeof(int)));
    k_fill<<<(unsigned)ceil_div64(npix, 256), 256>>>(p->ones, 1.f, npix);
    CAXSI_CUDA_TRY(cudaGetLastError());
    CAXSI_CUDA_TRY(cudaDeviceSynchronize());
    p->table_bytes += (int64_t)p->fwd_chunks * npix * 4 + (p->adj_split > 1 ? p->adj_split * nf * 4 : 0) +
                      3 * npix * 4 + 2 * nf * 4;
    return CAXSI_OK;
}

bool path_ok(int path) { return path >= CAXSI_PATH_DIRECT && path <= CAXSI_PATH_TABLE_FP16; }

// subset < 0: the full operator; else the rows of that detector subset (table paths).
caxsi_status run_forward(caxsi_plan *p, const float *f, float *g, int path, cudaStream_t s, int subset = -1) {
    if (path == CAXSI_PATH_DIRECT) return subset < 0 ? direct_forward(p, f, g, s) : direct_forward_subset(p, f, g, subset, s);
    return table_forward(p, f, g, path, subset, s);
}

caxsi_status run_adjoint(caxsi_plan *p, const float *w, float *f, int path, cudaStream_t s, int subset = -1) {
    if (path == CAXSI_PATH_DIRECT) return subset < 0 ? direct_adjoint(p, w, f, s) : direct_adjoint_subset(p, w, f, subset, s);
    return table_adjoint(p, w, f, path, subset, s);
}

void drop_subset_sensitivities(caxsi_plan *p) {
    for (int k = 0; k < 4; ++k) {
        cudaFree(p->b1_sub[k]);
        p->b1_sub[k] = nullptr;
        p->b1_sub_ok[k].clear();
    }
}

bool subset_ok(const caxsi_plan *p, int subset) { return subset >= 0 && subset < p->n_subsets; }

// [a, a + n) and [b, b + n) (floats) share an element
bool overlaps(const void *a, const void *b, int64_t n) {
    const uintptr_t x = reinterpret_cast<uintptr_t>(a), y = reinterpret_cast<uintptr_t>(b);
    const uintptr_t len = (uintptr_t)n * sizeof(float);
    return x < y + len && y < x + len;
}

}  // namespace

extern "C" {

caxsi_status caxsi_plan_create(const caxsi_geometry *geom, const double *phi_host,
                               const uint8_t *mask_host, caxsi_plan **out) {
    if (!geom || !phi_host || !mask_host || !out) return CAXSI_ERR_INVALID;
    caxsi_status st = validate(geom);
    if (st != CAXSI_OK) return st;
    for (int k = 0; k < geom->K; ++k)
        if (!isfinite(phi_host[k])) return CAXSI_ERR_INVALID;
    int dev;
    if (cudaGetDevice(&dev) != cudaSuccess) return CAXSI_ERR_CUDA;
    caxsi_plan *p = new (std::nothrow) caxsi_plan();
    if (!p) return CAXSI_ERR_OOM;
    p->g = *geom;
    p->device = dev;
    p->phi.assign(phi_host, phi_host + geom->K);
    if (cudaDeviceGetAttribute(&p->num_sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess) {
        delete p;
        return CAXSI_ERR_CUDA;
    }
    DevGeo &d = p->dg;
    d.X = geom->X; d.J = geom->J; d.Q = geom->Q; d.M = geom->M; d.N = geom->N; d.K = geom->K;
    d.rho_y = geom->rho_y;
    d.R = geom->X * geom->J;
    d.ND = geom->N + geom->rho_y * (geom->J - 1);
    d.d_min = -geom->rho_y * (geom->J - 1);
    d.Nw = (geom->N + 31) / 32;
    d.p_y = (float)geom->p_y;
    d.Xd = (float)geom->X_det;
    d.cN = 0.5f * (float)(geom->N - 1);
    const double dq = (geom->q_max - geom->q_min) / (geom->Q - 1);
    d.b = (float)(geom->q_min / dq);
    d.Qf = (float)geom->Q;
    {
        const double dE = (geom->E_max - geom->E_min) / geom->K;
        d.a0 = (float)((geom->E_min + 0.5 * dE) / (geom->hc * dq));
        d.da = (float)(dE / (geom->hc * dq));
    }

    direct_configure(p);
    int smem_max = 0;
    cudaDeviceGetAttribute(&smem_max, cudaDevAttrMaxSharedMemoryPerBlockOptin, dev);
    if ((size_t)smem_max < direct_adj_smem(p) || (size_t)smem_max < direct_fwd_smem(p) ||
        (size_t)smem_max < symmask_fwd_smem(p->dg) || (size_t)smem_max < symmask_adj_smem(p->dg)) {
        delete p;
        return CAXSI_ERR_UNSUPPORTED;
    }
    st = plan_build_tables(p, phi_host, mask_host);
    if (st == CAXSI_OK) st = alloc_scratch(p);
    if (st != CAXSI_OK) {
        free_plan(p);
        return st;
    }
    *out = p;
    return CAXSI_OK;
}

void caxsi_plan_destroy(caxsi_plan *plan) {
    if (!plan) return;
    DeviceGuard dg(plan->device);
    cudaDeviceSynchronize();
    free_plan(plan);
}

caxsi_status caxsi_forward(caxsi_plan *p, const float *f_dev, int64_t f_len, float *g_dev,
                           int64_t g_len, int path, void *stream) {
    if (!p || !f_dev || !g_dev || !path_ok(path)) return CAXSI_ERR_INVALID;
    if (f_len != (int64_t)p->dg.R * p->dg.Q || g_len != (int64_t)p->dg.M * p->dg.N)
        return CAXSI_ERR_INVALID;
    DeviceGuard dg(p->device);
    if (!dg.ok) return CAXSI_ERR_CUDA;
    p->launches = 0;
    return run_forward(p, f_dev, g_dev, path, (cudaStream_t)stream);
}

caxsi_status caxsi_adjoint(caxsi_plan *p, const float *w_dev, int64_t w_len, float *f_dev,
                           int64_t f_len, int path, void *stream) {
    if (!p || !f_dev || !w_dev || !path_ok(path)) return CAXSI_ERR_INVALID;
    if (f_len != (int64_t)p->dg.R * p->dg.Q || w_len != (int64_t)p->dg.M * p->dg.N)
        return CAXSI_ERR_INVALID;
    DeviceGuard dg(p->device);
    if (!dg.ok) return CAXSI_ERR_CUDA;
    p->launches = 0;
    return run_adjoint(p, w_dev, f_dev, path, (cudaStream_t)stream);
}

caxsi_status caxsi_recon_step(caxsi_plan *p, const float *y_dev, const float *r_dev, float *f_dev,
                              int64_t f_len, float beta, float delta, int path, double *nll_out,
                              void *stream) {
    if (!p || !y_dev || !f_dev || !path_ok(path)) return CAXSI_ERR_INVALID;
    if (f_len != (int64_t)p->dg.R * p->dg.Q) return CAXSI_ERR_INVALID;
    if (!isfinite(beta) || beta < 0.f || !isfinite(delta) || delta < 0.f) return CAXSI_ERR_INVALID;
    DeviceGuard dg(p->device);
    if (!dg.ok) return CAXSI_ERR_CUDA;
    cudaStream_t s = (cudaStream_t)stream;
    p->launches = 0;
    const int64_t nf = (int64_t)p->dg.R * p->dg.Q;
    caxsi_status st;
    if (!p->b1[path]) {
        // b1 = A^T 1, cached only once it has been computed
        float *b1 = nullptr;
        CAXSI_CUDA_TRY(cudaMalloc(&b1, nf * sizeof(float)));
        if ((st = run_adjoint(p, p->ones, b1, path, s)) != CAXSI_OK) {
            cudaStreamSynchronize(s);
            cudaFree(b1);
            return st;
        }
        p->b1[path] = b1;
        p->table_bytes += nf * 4;
    }
    // z = A f + r, ratio = y / z, and L(f) in FP64 when asked for
    if ((st = run_forward(p, f_dev, p->gtmp, path, s)) != CAXSI_OK) return st;
    if ((st = recon_ratio(p, y_dev, r_dev, nullptr, -1, nll_out != nullptr, s)) != CAXSI_OK) return st;
    if (nll_out) {
        int64_t keep = p->launches;
        st = recon_nll_fetch(p, nll_out, s);
        p->launches = keep;
        if (st != CAXSI_OK) return st;
    }
    // b2 = A^T (y / z), then the closed-form update
    if ((st = run_adjoint(p, p->ratio, p->b2, path, s)) != CAXSI_OK) return st;
    if ((st = recon_update(p, f_dev, beta, delta, p->b1[path], s)) != CAXSI_OK) return st;
    CAXSI_CUDA_TRY(cudaMemcpyAsync(f_dev, p->fnew, nf * sizeof(float), cudaMemcpyDeviceToDevice, s));
    return CAXSI_OK;
}

caxsi_status caxsi_plan_set_subsets(caxsi_plan *p, int n_subsets, const int32_t *subset_of_pixel) {
    if (!p || !subset_of_pixel) return CAXSI_ERR_INVALID;
    const int64_t npix = (int64_t)p->dg.M * p->dg.N;
    if (n_subsets < 1 || n_subsets > CAXSI_MAX_SUBSETS || n_subsets > npix) return CAXSI_ERR_INVALID;
    for (int64_t k = 0; k < npix; ++k)
        if (subset_of_pixel[k] < 0 || subset_of_pixel[k] >= n_subsets) return CAXSI_ERR_INVALID;
    DeviceGuard dg(p->device);
    if (!dg.ok) return CAXSI_ERR_CUDA;
    // subset calls in flight on any stream may still read the lists and records
    CAXSI_CUDA_TRY(cudaDeviceSynchronize());
    p->n_subsets = 0;
    drop_subset_sensitivities(p);
    // the partition and its pixel lists (counting sort of the pixels by subset)
    p->sub_host.assign(subset_of_pixel, subset_of_pixel + npix);
    p->sub_off.assign(n_subsets + 1, 0);
    std::vector<int> pix(npix), pos(npix);
    for (int64_t k = 0; k < npix; ++k) p->sub_off[subset_of_pixel[k] + 1]++;
    for (int s = 0; s < n_subsets; ++s) p->sub_off[s + 1] += p->sub_off[s];
    {
        std::vector<int> fill(p->sub_off.begin(), p->sub_off.end() - 1);
        for (int64_t k = 0; k < npix; ++k) {
            const int s = subset_of_pixel[k];
            pos[k] = fill[s] - p->sub_off[s];
            pix[fill[s]++] = (int)k;
        }
    }
    if (!p->sub_pix) CAXSI_CUDA_TRY(cudaMalloc(&p->sub_pix, npix * sizeof(int)));
    if (!p->sub_of_pix) CAXSI_CUDA_TRY(cudaMalloc(&p->sub_of_pix, npix * sizeof(int)));
    if (!p->sub_pos) CAXSI_CUDA_TRY(cudaMalloc(&p->sub_pos, npix * sizeof(int)));
    CAXSI_CUDA_TRY(cudaMemcpy(p->sub_pix, pix.data(), npix * sizeof(int), cudaMemcpyHostToDevice));
    CAXSI_CUDA_TRY(cudaMemcpy(p->sub_of_pix, subset_of_pixel, npix * sizeof(int), cudaMemcpyHostToDevice));
    CAXSI_CUDA_TRY(cudaMemcpy(p->sub_pos, pos.data(), npix * sizeof(int), cudaMemcpyHostToDevice));
    ++p->sub_gen;
    p->n_subsets = n_subsets;
    // the table paths' grouped records now if the table exists, else on first use;
    // a geometry without pair records keeps the partition for the direct path (its
    // table-path subset calls then return UNSUPPORTED)
    caxsi_status st = p->table ? table_set_subsets(p) : CAXSI_OK;
    if (st == CAXSI_ERR_UNSUPPORTED) st = CAXSI_OK;
    if (st != CAXSI_OK) p->n_subsets = 0;
    return st;
}

caxsi_status caxsi_forward_subset(caxsi_plan *p, int subset, const float *f_dev, int64_t f_len, float *g_dev,
                                  int64_t g_len, int path, void *stream) {
    if (!p || !f_dev || !g_dev || !path_ok(path) || !subset_ok(p, subset)) return CAXSI_ERR_INVALID;
    if (f_len != (int64_t)p->dg.R * p->dg.Q || g_len != (int64_t)p->dg.M * p->dg.N)
        return CAXSI_ERR_INVALID;
    DeviceGuard dg(p->device);
    if (!dg.ok) return CAXSI_ERR_CUDA;
    p->launches = 0;
    return run_forward(p, f_dev, g_dev, path, (cudaStream_t)stream, subset);
}

caxsi_status caxsi_adjoint_subset(caxsi_plan *p, int subset, const float *w_dev, int64_t w_len, float *f_dev,
                                  int64_t f_len, int path, void *stream) {
    if (!p || !f_dev || !w_dev || !path_ok(path) || !subset_ok(p, subset)) return CAXSI_ERR_INVALID;
    if (f_len != (int64_t)p->dg.R * p->dg.Q || w_len != (int64_t)p->dg.M * p->dg.N)
        return CAXSI_ERR_INVALID;
    DeviceGuard dg(p->device);
    if (!dg.ok) return CAXSI_ERR_CUDA;
    p->launches = 0;
    return run_adjoint(p, w_dev, f_dev, path, (cudaStream_t)stream, subset);
}

caxsi_status caxsi_recon_step_subset(caxsi_plan *p, int subset, const float *y_dev, const float *r_dev,
                                     float *f_dev, int64_t f_len, float beta, float delta, int path,
                                     double *nll_out, void *stream) {
    if (!p || !y_dev || !f_dev || !path_ok(path) || !subset_ok(p, subset)) return CAXSI_ERR_INVALID;
    if (f_len != (int64_t)p->dg.R * p->dg.Q) return CAXSI_ERR_INVALID;
    if (!isfinite(beta) || beta < 0.f || !isfinite(delta) || delta < 0.f) return CAXSI_ERR_INVALID;
    DeviceGuard dg(p->device);
    if (!dg.ok) return CAXSI_ERR_CUDA;
    cudaStream_t s = (cudaStream_t)stream;
    p->launches = 0;
    const int64_t nf = (int64_t)p->dg.R * p->dg.Q;
    caxsi_status st;
    if (!p->b1_sub[path]) {
        CAXSI_CUDA_TRY(cudaMalloc(&p->b1_sub[path], (size_t)p->n_subsets * nf * sizeof(float)));
        p->b1_sub_ok[path].assign(p->n_subsets, 0);
        p->table_bytes += p->n_subsets * nf * 4;
    }
    float *b1p = p->b1_sub[path] + (int64_t)subset * nf;
    if (!p->b1_sub_ok[path][subset]) {
        // b1_p = A_p^T 1: the subset adjoint reads only the subset's pixels of `ones`
        if ((st = run_adjoint(p, p->ones, b1p, path, s, subset)) != CAXSI_OK) return st;
        p->b1_sub_ok[path][subset] = 1;
    }
    // z_p = A_p f + r_p, ratio on the subset's pixels, and L_p(f) in FP64 when asked for
    if ((st = run_forward(p, f_dev, p->gtmp, path, s, subset)) != CAXSI_OK) return st;
    if ((st = recon_ratio(p, y_dev, r_dev, p->sub_of_pix, subset, nll_out != nullptr, s)) != CAXSI_OK) return st;
    if (nll_out) {
        int64_t keep = p->launches;
        st = recon_nll_fetch(p, nll_out, s);
        p->launches = keep;
        if (st != CAXSI_OK) return st;
    }
    // b2_p = A_p^T (y_p / z_p), then the closed-form update with b1_p
    if ((st = run_adjoint(p, p->ratio, p->b2, path, s, subset)) != CAXSI_OK) return st;
    if ((st = recon_update(p, f_dev, beta, delta, b1p, s)) != CAXSI_OK) return st;
    CAXSI_CUDA_TRY(cudaMemcpyAsync(f_dev, p->fnew, nf * sizeof(float), cudaMemcpyDeviceToDevice, s));
    return CAXSI_OK;
}

static caxsi_status batch_args(const caxsi_plan *p, int nb, const int32_t *ranges, const void *in, int64_t in_len,
                               const void *out, int64_t out_len, bool fwd) {
    if (!p || !ranges || !in || !out || nb < 1 || nb > CAXSI_MAX_BATCH) return CAXSI_ERR_INVALID;
    const int64_t nf = (int64_t)p->dg.R * p->dg.Q, ng = (int64_t)p->dg.M * p->dg.N;
    if (in_len != nb * (fwd ? nf : ng) || out_len != nb * (fwd ? ng : nf)) return CAXSI_ERR_INVALID;
    for (int b = 0; b < nb; ++b)
        if (ranges[2 * b] < 0 || ranges[2 * b] > ranges[2 * b + 1] || ranges[2 * b + 1] > p->dg.R)
            return CAXSI_ERR_INVALID;
    return CAXSI_OK;
}

caxsi_status caxsi_forward_batch(caxsi_plan *p, int n_objects, const int32_t *voxel_ranges, const float *f_dev,
                                 int64_t f_len, float *g_dev, int64_t g_len, int path, void *stream) {
    caxsi_status st = batch_args(p, n_objects, voxel_ranges, f_dev, f_len, g_dev, g_len, true);
    if (st != CAXSI_OK) return st;
    if (!path_ok(path)) return CAXSI_ERR_INVALID;
    DeviceGuard dg(p->device);
    if (!dg.ok) return CAXSI_ERR_CUDA;
    p->launches = 0;
    return table_forward_batch(p, n_objects, voxel_ranges, f_dev, g_dev, path, (cudaStream_t)stream);
}

caxsi_status caxsi_adjoint_batch(caxsi_plan *p, int n_objects, const int32_t *voxel_ranges, const float *w_dev,
                                 int64_t w_len, float *f_dev, int64_t f_len, int path, void *stream) {
    caxsi_status st = batch_args(p, n_objects, voxel_ranges, w_dev, w_len, f_dev, f_len, false);
    if (st != CAXSI_OK) return st;
    if (!path_ok(path)) return CAXSI_ERR_INVALID;
    DeviceGuard dg(p->device);
    if (!dg.ok) return CAXSI_ERR_CUDA;
    p->launches = 0;
    return table_adjoint_batch(p, n_objects, voxel_ranges, w_dev, f_dev, path, (cudaStream_t)stream);
}

caxsi_status caxsi_em_update(caxsi_plan *p, const float *f_dev, const float *b1_dev, const float *b2_dev,
                             float beta, float delta, float *f_out_dev, int64_t f_len, void *stream) {
    if (!p || !f_dev || !b1_dev || !b2_dev || !f_out_dev) return CAXSI_ERR_INVALID;
    const int64_t nf = (int64_t)p->dg.R * p->dg.Q;
    if (f_len < nf || f_len % nf) return CAXSI_ERR_INVALID;
    // the update reads the neighbours of every element of f while writing f_out
    if (overlaps(f_out_dev, f_dev, f_len)) return CAXSI_ERR_INVALID;
    if (!isfinite(beta) || beta < 0.f || !isfinite(delta) || delta < 0.f) return CAXSI_ERR_INVALID;
    DeviceGuard dg(p->device);
    if (!dg.ok) return CAXSI_ERR_CUDA;
    p->launches = 0;
    return recon_update_ext(p, f_dev, b1_dev, b2_dev, beta, delta, f_out_dev, f_len, (cudaStream_t)stream);
}

caxsi_status caxsi_em_update_vjp(caxsi_plan *p, const float *f_dev, const float *b1_dev, const float *b2_dev,
                                 float beta, float delta, const float *grad_out_dev, float *grad_f_dev,
                                 float *grad_b2_dev, int64_t f_len, void *stream) {
    if (!p || !f_dev || !b1_dev || !b2_dev || !grad_out_dev || !grad_f_dev || !grad_b2_dev)
        return CAXSI_ERR_INVALID;
    const int64_t nf = (int64_t)p->dg.R * p->dg.Q;
    if (f_len < nf || f_len % nf) return CAXSI_ERR_INVALID;
    // both passes read f, b1, b2 and grad_out (the second pass at the neighbours too)
    // while writing grad_f and grad_b2
    for (const float *out : {(const float *)grad_f_dev, (const float *)grad_b2_dev})
        for (const float *in : {f_dev, b1_dev, b2_dev, grad_out_dev})
            if (overlaps(out, in, f_len)) return CAXSI_ERR_INVALID;
    if (overlaps(grad_f_dev, grad_b2_dev, f_len)) return CAXSI_ERR_INVALID;
    if (!isfinite(beta) || beta < 0.f || !isfinite(delta) || delta < 0.f) return CAXSI_ERR_INVALID;
    DeviceGuard dg(p->device);
    if (!dg.ok) return CAXSI_ERR_CUDA;
    p->launches = 0;
    return recon_update_vjp(p, f_dev, b1_dev, b2_dev, beta, delta, grad_out_dev, grad_f_dev, grad_b2_dev, f_len,
                            (cudaStream_t)stream);
}

caxsi_status caxsi_ratio(caxsi_plan *p, const float *g_dev, const float *y_dev, const float *r_dev,
                         float *ratio_dev, int64_t n, void *stream) {
    if (!p || !g_dev || !y_dev || !ratio_dev || n < 1) return CAXSI_ERR_INVALID;
    DeviceGuard dg(p->device);
    if (!dg.ok) return CAXSI_ERR_CUDA;
    p->launches = 0;
    return recon_ratio_ext(p, g_dev, y_dev, r_dev, ratio_dev, n, (cudaStream_t)stream);
}

caxsi_status caxsi_ratio_vjp(caxsi_plan *p, const float *g_dev, const float *y_dev, const float *r_dev,
                             const float *grad_ratio_dev, float *grad_g_dev, int64_t n, void *stream) {
    if (!p || !g_dev || !y_dev || !grad_ratio_dev || !grad_g_dev || n < 1) return CAXSI_ERR_INVALID;
    DeviceGuard dg(p->device);
    if (!dg.ok) return CAXSI_ERR_CUDA;
    p->launches = 0;
    return recon_ratio_vjp(p, g_dev, y_dev, r_dev, grad_ratio_dev, grad_g_dev, n, (cudaStream_t)stream);
}

static caxsi_status host_call(caxsi_plan *p, const float *in_host, int64_t in_len, float *out_host,
                              int64_t out_len, int path, bool fwd) {
    if (!p || !in_host || !out_host || !path_ok(path)) return CAXSI_ERR_INVALID;
    const int64_t nf = (int64_t)p->dg.R * p->dg.Q, ng = (int64_t)p->dg.M * p->dg.N;
    if (in_len != (fwd ? nf : ng) || out_len != (fwd ? ng : nf)) return CAXSI_ERR_INVALID;
    DeviceGuard dg(p->device);
    if (!dg.ok) return CAXSI_ERR_CUDA;
    const int64_t big = nf > ng ? nf : ng;
    if (!p->stage_in) {
        CAXSI_CUDA_TRY(cudaMalloc(&p->stage_in, big * sizeof(float)));
        p->table_bytes += big * 4;
    }
    if (!p->stage_out) {
        CAXSI_CUDA_TRY(cudaMalloc(&p->stage_out, big * sizeof(float)));
        p->table_bytes += big * 4;
    }
    p->launches = 0;
    cudaStream_t s = 0;
    // the FP32 table path overlaps the copy of f with part of the contraction: the
    // forward contracts the first quarter of the rows while the rest of f arrives
    const int64_t part = (p->dg.R / 4) & ~int64_t(127);
    const bool piped = path == CAXSI_PATH_TABLE_FP32 && part > 0;
    if (piped && !p->copy_stream) {
        CAXSI_CUDA_TRY(cudaStreamCreateWithFlags(&p->copy_stream, cudaStreamNonBlocking));
        if (cudaEventCreateWithFlags(&p->pipe_ev[0], cudaEventDisableTiming) != cudaSuccess ||
            cudaEventCreateWithFlags(&p->pipe_ev[1], cudaEventDisableTiming) != cudaSuccess) {
            cudaStreamDestroy(p->copy_stream);
            p->copy_stream = nullptr;
            return CAXSI_ERR_CUDA;
        }
    }
    HostPipe pipe{part, p->copy_stream, p->pipe_ev[0], p->pipe_ev[1], out_host, 0};
    if (piped && fwd) {
        // the first part of f, then the rest on the copy stream (one after the other:
        // they share the link) while the first part's contraction runs
        const int64_t n1 = part * p->dg.Q;
        CAXSI_CUDA_TRY(cudaMemcpyAsync(p->stage_in, in_host, n1 * sizeof(float), cudaMemcpyHostToDevice, s));
        CAXSI_CUDA_TRY(cudaEventRecord(pipe.out_half, s));
        CAXSI_CUDA_TRY(cudaStreamWaitEvent(pipe.cs, pipe.out_half, 0));
        CAXSI_CUDA_TRY(cudaMemcpyAsync(p->stage_in + n1, in_host + n1, (in_len - n1) * sizeof(float),
                                       cudaMemcpyHostToDevice, pipe.cs));
        CAXSI_CUDA_TRY(cudaEventRecord(pipe.in_ready, pipe.cs));
    } else {
        CAXSI_CUDA_TRY(cudaMemcpyAsync(p->stage_in, in_host, in_len * sizeof(float), cudaMemcpyHostToDevice, s));
    }
    p->pipe = piped ? &pipe : nullptr;
    caxsi_status st = fwd ? run_forward(p, p->stage_in, p->stage_out, path, s)
                          : run_adjoint(p, p->stage_in, p->stage_out, path, s);
    p->pipe = nullptr;
    if (st == CAXSI_OK) {
        // the part of the result that the adjoint has not sent already
        const int64_t from = fwd ? 0 : pipe.out_from * p->dg.Q;
        if (cudaMemcpyAsync(out_host + from, p->stage_out + from, (out_len - from) * sizeof(float),
                            cudaMemcpyDeviceToHost, s) != cudaSuccess)
            st = CAXSI_ERR_CUDA;
    }
    // both streams are drained before returning, also after an error
    if (cudaStreamSynchronize(s) != cudaSuccess) st = CAXSI_ERR_CUDA;
    if (piped && cudaStreamSynchronize(pipe.cs) != cudaSuccess) st = CAXSI_ERR_CUDA;
    return st;
}

caxsi_status caxsi_forward_host(caxsi_plan *p, const float *f_host, int64_t f_len, float *g_host,
                                int64_t g_len, int path) {
    return host_call(p, f_host, f_len, g_host, g_len, path, true);
}

caxsi_status caxsi_adjoint_host(caxsi_plan *p, const float *w_host, int64_t w_len, float *f_host,
                                int64_t f_len, int path) {
    return host_call(p, w_host, w_len, f_host, f_len, path, false);
}

caxsi_status caxsi_plan_info(caxsi_plan *p, caxsi_plan_info_t *info) {
    if (!p || !info) return CAXSI_ERR_INVALID;
    DeviceGuard dg(p->device);
    int e = 0;
    if (cudaDeviceSynchronize() != cudaSuccess ||
        cudaMemcpy(&e, p->err_flag + 1, sizeof(int), cudaMemcpyDeviceToHost) != cudaSuccess)
        return CAXSI_ERR_CUDA;
    if (e) cudaMemset(p->err_flag + 1, 0, sizeof(int));
    info->device_error = e;
    info->n_offsets = p->dg.ND;
    info->table_bytes = p->table_bytes;
    info->n_breakpoints = table_breakpoints(p);
    info->kernel_launches = p->launches;
    info->n_open_pairs = p->open_pairs;
    info->n_records = table_records(p);
    info->n_sym_records = table_sym_records(p);
    info->mask_symmetric = p->mask_symmetric;
    return CAXSI_OK;
}

caxsi_status caxsi_forward_static_scratch(caxsi_plan *p, const float *f_dev, int64_t f_len,
                                          float *g_dev, int64_t g_len, void *stream) {
    if (!p || !f_dev || !g_dev) return CAXSI_ERR_INVALID;
    if (f_len != (int64_t)p->dg.R * p->dg.Q || g_len != (int64_t)p->dg.M * p->dg.N)
        return CAXSI_ERR_INVALID;
    DeviceGuard dg(p->device);
    if (!dg.ok) return CAXSI_ERR_CUDA;
    p->launches = 0;
    return direct_forward_static_scratch(p, f_dev, g_dev, (cudaStream_t)stream);
}

caxsi_status caxsi_plan_set_option(caxsi_plan *p, int key, int value) {
    if (!p) return CAXSI_ERR_INVALID;
    if (key == CAXSI_OPT_GEMM_ENGINE && (value == CAXSI_GEMM_TCGEN05 || value == CAXSI_GEMM_CUBLAS)) {
        p->gemm_engine = value;
        return CAXSI_OK;
    }
    if (key == CAXSI_OPT_SYMMETRY && (value == 0 || value == 1)) {
        p->no_symmetry = !value;
        return CAXSI_OK;
    }
    if (key == CAXSI_OPT_SPARSE_SUBSETS && (value == 0 || value == 1)) {
        p->no_sparse_subsets = !value;
        return CAXSI_OK;
    }
    if (key == CAXSI_OPT_GEMM_BANDS && (value == 0 || value == 1)) {
        p->no_bands = !value;
        return CAXSI_OK;
    }
    if (key == CAXSI_OPT_ONLINE_MASK && (value == 0 || value == 1)) {
        if (value && !p->mask_symmetric) return CAXSI_ERR_UNSUPPORTED;
        p->online_mask = value;
        return CAXSI_OK;
    }
    if (key == CAXSI_OPT_TEST_WAIT_LIMIT && value >= 0) {
        p->test_wait_limit = (uint32_t)value;
        return CAXSI_OK;
    }
    if (key == CAXSI_OPT_TEST_WITHHOLD_COPY && (value == 0 || value == 1)) {
        p->test_withhold = value;
        return CAXSI_OK;
    }
    if (key == CAXSI_OPT_U_SAMPLES && (value == 0 || (value >= 2 && value <= CAXSI_MAX_U_SAMPLES))) {
        if (p->table && value != p->u_samples) return CAXSI_ERR_INVALID;   // fixed once the table is built
        p->u_samples = value;
        return CAXSI_OK;
    }
    return CAXSI_ERR_INVALID;
}

static void prof_clear(caxsi_plan *p) {
    for (auto &r : p->prof.recs) {
        cudaEventSynchronize(r.b);
        p->prof.pool.push_back(r.a);
        p->prof.pool.push_back(r.b);
    }
    p->prof.recs.clear();
}

caxsi_status caxsi_profile_enable(caxsi_plan *p, int enable) {
    if (!p) return CAXSI_ERR_INVALID;
    DeviceGuard dg(p->device);
    prof_clear(p);
    p->prof.on = enable != 0;
    return CAXSI_OK;
}

caxsi_status caxsi_profile_read(caxsi_plan *p, caxsi_kernel_stat *out, int capacity, int *count) {
    if (!p || !count || capacity < 0 || (capacity > 0 && !out)) return CAXSI_ERR_INVALID;
    DeviceGuard dg(p->device);
    int n = 0;
    caxsi_status st = CAXSI_OK;
    for (auto &r : p->prof.recs) {
        if (cudaEventSynchronize(r.b) != cudaSuccess) { st = CAXSI_ERR_CUDA; continue; }
        float ms = 0.f;
        if (cudaEventElapsedTime(&ms, r.a, r.b) != cudaSuccess) { st = CAXSI_ERR_CUDA; continue; }
        int k = 0;
        while (k < n && strncmp(out[k].name, r.name, sizeof(out[k].name) - 1) != 0) ++k;
        if (k == n) {
            if (n >= capacity) continue;
            memset(&out[n], 0, sizeof(out[n]));
            strncpy(out[n].name, r.name, sizeof(out[n].name) - 1);
            ++n;
        }
        out[k].launches += 1;
        out[k].total_ms += ms;
    }
    prof_clear(p);
    *count = n;
    return st;
}

caxsi_status caxsi_os_partition(int M, int N, int rho_y, int rho_z, int sigma_y, int32_t *subset_of_pixel) {
    if (!subset_of_pixel || M < 2 || N < 1 || rho_y < 1 || rho_z < 1) return CAXSI_ERR_INVALID;
    if (sigma_y <= 0) sigma_y = rho_y % 2 == 0 ? rho_y : 16 * rho_y;
    // rows: the upper half in rho_z classes of step rho_z, each row's mirror image
    // about z = 0 in its class; columns: classes of step sigma_y, each column's
    // mirror image about y = 0 in its class (sigma_y / 2 column classes)
    if (M % 2 || (M / 2) % rho_z) return CAXSI_ERR_INVALID;
    if (sigma_y < 2 || sigma_y % 2 || N % sigma_y || sigma_y % rho_y) return CAXSI_ERR_INVALID;
    const int cols = sigma_y / 2;
    for (int m = 0; m < M; ++m) {
        const int row_class = (m < M / 2 ? m : M - 1 - m) % rho_z;
        for (int n = 0; n < N; ++n) {
            const int c = n % sigma_y;
            const int col_class = c < sigma_y - 1 - c ? c : sigma_y - 1 - c;
            subset_of_pixel[(int64_t)m * N + n] = row_class * cols + col_class;
        }
    }
    return CAXSI_OK;
}

const char *caxsi_status_string(caxsi_status s) {
    switch (s) {
        case CAXSI_OK: return "ok";
        case CAXSI_ERR_INVALID: return "invalid argument";
        case CAXSI_ERR_CUDA: return "CUDA error";
        case CAXSI_ERR_OOM: return "out of device memory";
        case CAXSI_ERR_NONPOS_MEAN: return "positive count with non-positive mean";
        case CAXSI_ERR_INTERNAL: return "internal consistency check failed";
        case CAXSI_ERR_UNSUPPORTED: return "unsupported option";
        case CAXSI_ERR_SCRATCH_LIMIT: return "problem exceeds the static scratch array";
    }
    return "unknown status";
}

}  // extern "C"
