// Plan tables (FP64 kernels, stored as FP32 / bits).
//
// * voxel table: position, y in units of the detector pitch, C * G_so
//   (G_so = x/(x^2+y^2)^1.5, Appendix A) and |r|^2;
// * offset table: G_od(s) * dtheta(s) for every scatter vector
//   s = (X_det - x_i, y'_n - y_j, z'_m).  With the object y pitch equal to
//   rho_y detector pitches, s depends on (i, d = n - rho_y j, m) only
//   (translation symmetry, Sec. III-A), so one entry serves all (j, n) pairs
//   with the same offset d;
// * mask factor bits: T(r, r') for every pair, the binary mask value where
//   the ray crosses the mask plane (Appendix A), precomputed as the paper
//   precomputes its mask factors (Sec. III-C).  The cell decision is taken in
//   FP64 with explicitly rounded operations (no fused multiply-add), so it is
//   the IEEE double result of the ray-plane intersection formula.
#include <math.h>
#include <stdio.h>

#include "internal.cuh"
#include "maskgeo.cuh"

namespace {

__global__ void k_plan_voxels(PlanGeo64 g, float4 *vox) {
    int v = blockIdx.x * blockDim.x + threadIdx.x;
    if (v >= g.X * g.J) return;
    int i = v / g.J, j = v % g.J;
    double x = vox_x(g, i), y = vox_y(g, j);
    double r2 = x * x + y * y;
    double gso = x / (r2 * sqrt(r2));
    float Y = (float)(((double)j - 0.5 * (g.J - 1)) * g.rho_y);  // exact half-integer
    vox[v] = make_float4((float)x, Y, (float)(g.C * gso), (float)r2);
}

__global__ void k_plan_rows(PlanGeo64 g, float *zrow) {
    int m = blockIdx.x * blockDim.x + threadIdx.x;
    if (m < g.M) zrow[m] = (float)pix_z(g, m);
}

// G_od * dtheta per (i, m, d); s_y = p_y (d + c0) with c0 = rho_y (J-1)/2 - (N-1)/2.
__global__ void k_plan_offsets(PlanGeo64 g, float *god) {
    int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    int64_t total = (int64_t)g.X * g.M * g.ND;
    if (t >= total) return;
    int dd = (int)(t % g.ND);
    int m = (int)((t / g.ND) % g.M);
    int i = (int)(t / ((int64_t)g.ND * g.M));
    double c0 = 0.5 * g.rho_y * (g.J - 1) - 0.5 * (g.N - 1);
    double sx = g.Xd - vox_x(g, i);
    double sy = ((double)(dd + g.d_min) + c0) * g.py;
    double sz = pix_z(g, m);
    double s2 = sx * sx + sy * sy + sz * sz;
    double g_od = fabs(sx) / (s2 * sqrt(s2));
    // angle between s+ = s + (0,0,h) and s- = s - (0,0,h), h = p_z / 2
    double h = 0.5 * g.pz;
    double a0 = sx, a1 = sy, a2 = sz + h;
    double b0 = sx, b1 = sy, b2 = sz - h;
    double cx = a1 * b2 - a2 * b1, cy = a2 * b0 - a0 * b2, cz = a0 * b1 - a1 * b0;
    double dth = atan2(sqrt(cx * cx + cy * cy + cz * cz), a0 * b0 + a1 * b1 + a2 * b2);
    god[t] = (float)(g_od * dth);
}

__global__ void k_plan_mask_rows(PlanGeo64 g, int *rowidx) {
    int t = blockIdx.x * blockDim.x + threadIdx.x;
    if (t >= g.X * g.M) return;
    int i = t / g.M, m = t % g.M;
    rowidx[t] = mask_row(g, i, m);
}

__global__ void k_plan_mask_cols(PlanGeo64 g, int *colidx) {
    int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (t >= (int64_t)g.X * g.J * g.N) return;
    int n = (int)(t % g.N);
    int j = (int)((t / g.N) % g.J);
    int i = (int)(t / ((int64_t)g.N * g.J));
    colidx[t] = mask_col(g, i, j, n);
}

// One 32-bit word of mask factor bits per thread: voxel v, row m, word w.
__global__ void k_plan_tbits(PlanGeo64 g, int Nw, const int *rowidx, const int *colidx,
                             const uint8_t *mask, uint32_t *tbits) {
    int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    int64_t total = (int64_t)g.X * g.J * g.M * Nw;
    if (t >= total) return;
    int w = (int)(t % Nw);
    int m = (int)((t / Nw) % g.M);
    int64_t v = t / ((int64_t)Nw * g.M);
    int i = (int)(v / g.J);
    int row = rowidx[i * g.M + m];
    uint32_t bits = 0;
    if (row >= 0) {
        const int *cols = colidx + v * g.N;
        const uint8_t *mrow = mask + (int64_t)row * g.cols;
        for (int b = 0; b < 32; ++b) {
            int n = w * 32 + b;
            if (n >= g.N) break;
            int c = cols[n];
            if (c >= 0 && mrow[c]) bits |= (1u << b);
        }
    }
    tbits[t] = bits;
}

// Number of set mask-factor bits (plan statistics only).
__global__ void k_popcount(const uint32_t *bits, int64_t n, unsigned long long *out) {
    unsigned long long c = 0;
    for (int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; t < n;
         t += (int64_t)gridDim.x * blockDim.x)
        c += __popc(bits[t]);
    for (int o = 16; o > 0; o >>= 1) c += __shfl_down_sync(0xffffffffu, c, o);
    if ((threadIdx.x & 31) == 0) atomicAdd(out, c);
}

}  // namespace

caxsi_status plan_build_tables(caxsi_plan *p, const double *phi_host, const uint8_t *mask_host) {
    const caxsi_geometry &G = p->g;
    DevGeo &d = p->dg;
    const PlanGeo64 g = plan_geo64(p);

    const int64_t R = (int64_t)G.X * G.J;
    const int64_t n_off = (int64_t)G.X * G.M * d.ND;
    const int64_t n_bits = R * G.M * d.Nw;
    CAXSI_CUDA_TRY(cudaMalloc(&p->vox, R * sizeof(float4)));
    CAXSI_CUDA_TRY(cudaMalloc(&p->zrow, G.M * sizeof(float)));
    CAXSI_CUDA_TRY(cudaMalloc(&p->god, n_off * sizeof(float)));
    CAXSI_CUDA_TRY(cudaMalloc(&p->tbits, n_bits * sizeof(uint32_t)));
    CAXSI_CUDA_TRY(cudaMalloc(&p->energy, G.K * sizeof(float2)));
    p->table_bytes += R * sizeof(float4) + G.M * sizeof(float) + n_off * sizeof(float) +
                      n_bits * sizeof(uint32_t) + G.K * sizeof(float2);

    // energy constants: a_k = E_k / (hc dq), c_k = Phi_k E_k dE / hc^2 (energy form of Eq. 4)
    {
        float2 en[CAXSI_MAX_K];
        double dE = (G.E_max - G.E_min) / G.K;
        double dq = (G.q_max - G.q_min) / (G.Q - 1);
        for (int k = 0; k < G.K; ++k) {
            double E = G.E_min + (k + 0.5) * dE;
            en[k] = make_float2((float)(E / (G.hc * dq)), (float)(phi_host[k] * E * dE / (G.hc * G.hc)));
        }
        CAXSI_CUDA_TRY(cudaMemcpy(p->energy, en, G.K * sizeof(float2), cudaMemcpyHostToDevice));
    }

    const int T = 256;
    k_plan_voxels<<<(unsigned)ceil_div64(R, T), T>>>(g, p->vox);
    CAXSI_CUDA_TRY(cudaGetLastError());
    k_plan_rows<<<(unsigned)ceil_div64(G.M, T), T>>>(g, p->zrow);
    CAXSI_CUDA_TRY(cudaGetLastError());
    k_plan_offsets<<<(unsigned)ceil_div64(n_off, T), T>>>(g, p->god);
    CAXSI_CUDA_TRY(cudaGetLastError());

    // mask factor bits via temporary FP64 cell-index tables
    uint8_t *mask_dev = nullptr;
    int *rowidx = nullptr, *colidx = nullptr;
    const int64_t n_mask = (int64_t)G.mask_rows * G.mask_cols;
    const int64_t n_cols = R * G.N;
    caxsi_status st = CAXSI_OK;
    do {
        cudaError_t e;
        if ((e = cudaMalloc(&mask_dev, n_mask)) != cudaSuccess ||
            (e = cudaMalloc(&rowidx, (size_t)G.X * G.M * sizeof(int))) != cudaSuccess ||
            (e = cudaMalloc(&colidx, (size_t)(n_cols < 2 ? 2 : n_cols) * sizeof(int))) != cudaSuccess) {
            st = e == cudaErrorMemoryAllocation ? CAXSI_ERR_OOM : CAXSI_ERR_CUDA;
            break;
        }
        // normalise the mask to 0/1 on the host copy path
        uint8_t *m01 = (uint8_t *)malloc((size_t)n_mask);
        if (!m01) { st = CAXSI_ERR_OOM; break; }
        for (int64_t q = 0; q < n_mask; ++q) m01[q] = mask_host[q] ? 1 : 0;
        // mirror symmetry about the central ray: cells centred on y = 0 and z = 0 and
        // the pattern equal to its left-right and up-down images; with J, M, N even
        // the pairs related by the mirrors then share their mask factor
        bool sym = G.J % 2 == 0 && G.M % 2 == 0 && G.N % 2 == 0 &&
                   G.mask_y0 == -0.5 * G.mask_cols * G.mask_cell && G.mask_z0 == -0.5 * G.mask_rows * G.mask_cell;
        for (int r = 0; r < G.mask_rows && sym; ++r)
            for (int c = 0; c < G.mask_cols && sym; ++c) {
                const uint8_t a = m01[(int64_t)r * G.mask_cols + c];
                sym = a == m01[(int64_t)r * G.mask_cols + (G.mask_cols - 1 - c)] &&
                      a == m01[(int64_t)(G.mask_rows - 1 - r) * G.mask_cols + c];
            }
        p->mask_symmetric = sym ? 1 : 0;
        e = cudaMemcpy(mask_dev, m01, (size_t)n_mask, cudaMemcpyHostToDevice);
        free(m01);
        if (e != cudaSuccess) { st = CAXSI_ERR_CUDA; break; }
        k_plan_mask_rows<<<(unsigned)ceil_div64((int64_t)G.X * G.M, T), T>>>(g, rowidx);
        k_plan_mask_cols<<<(unsigned)ceil_div64(n_cols, T), T>>>(g, colidx);
        k_plan_tbits<<<(unsigned)ceil_div64(n_bits, T), T>>>(g, d.Nw, rowidx, colidx, mask_dev, p->tbits);
        if (cudaGetLastError() != cudaSuccess || cudaDeviceSynchronize() != cudaSuccess) {
            st = CAXSI_ERR_CUDA;
            break;
        }
        // reuse the column-index buffer (allocated with >= 8 bytes) as the counter
        unsigned long long *cnt = reinterpret_cast<unsigned long long *>(colidx);
        unsigned long long h = 0;
        if (cudaMemset(cnt, 0, sizeof(h)) != cudaSuccess) { st = CAXSI_ERR_CUDA; break; }
        k_popcount<<<2 * p->num_sms, 256>>>(p->tbits, n_bits, cnt);
        if (cudaGetLastError() != cudaSuccess ||
            cudaMemcpy(&h, cnt, sizeof(h), cudaMemcpyDeviceToHost) != cudaSuccess) {
            st = CAXSI_ERR_CUDA;
            break;
        }
        p->open_pairs = (int64_t)h;
    } while (0);
    // the 0 / 1 mask stays with the plan (the online mask factor reads it)
    if (st == CAXSI_OK) {
        p->mask01 = mask_dev;
        p->table_bytes += n_mask;
    } else {
        cudaFree(mask_dev);
    }
    cudaFree(rowidx);
    cudaFree(colidx);
    return st;
}
