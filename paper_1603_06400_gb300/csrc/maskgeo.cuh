// FP64 positions of voxels and pixels and the mask cell a scattered ray crosses
// (Appendix A: the ray from voxel r to pixel r' meets the mask plane x = X_mask at
// t = (X_mask - x) / (X_det - x)), each operation rounded as written (no fused
// multiply-add), so the cell decision is the IEEE double result of the formula.
// Shared by the plan builder (precomputed mask factor bits) and the kernels that
// compute the mask factor online.
#pragma once

#include "internal.cuh"

struct PlanGeo64 {
    int X, J, M, N, rho_y, rows, cols, ND, d_min;
    double xc, dx, py, pz, Xd, Xm, C, cell, y0, z0;
};

inline PlanGeo64 plan_geo64(const caxsi_plan *p) {
    const caxsi_geometry &G = p->g;
    PlanGeo64 g;
    g.X = G.X; g.J = G.J; g.M = G.M; g.N = G.N; g.rho_y = G.rho_y;
    g.rows = G.mask_rows; g.cols = G.mask_cols; g.ND = p->dg.ND; g.d_min = p->dg.d_min;
    g.xc = G.x_center; g.dx = G.dx; g.py = G.p_y; g.pz = G.p_z; g.Xd = G.X_det;
    g.Xm = G.X_mask; g.C = G.C; g.cell = G.mask_cell; g.y0 = G.mask_y0; g.z0 = G.mask_z0;
    return g;
}


static __device__ __forceinline__ double vox_x(const PlanGeo64 &g, int i) {
    return __dadd_rn(g.xc, __dmul_rn((double)i - 0.5 * (g.X - 1), g.dx));
}
static __device__ __forceinline__ double vox_y(const PlanGeo64 &g, int j) {
    return __dmul_rn(__dmul_rn((double)j - 0.5 * (g.J - 1), (double)g.rho_y), g.py);
}
static __device__ __forceinline__ double pix_y(const PlanGeo64 &g, int n) {
    return __dmul_rn((double)n - 0.5 * (g.N - 1), g.py);
}
static __device__ __forceinline__ double pix_z(const PlanGeo64 &g, int m) {
    return __dmul_rn((double)m - 0.5 * (g.M - 1), g.pz);
}

// Mask cell indices in FP64, rounded step by step as written.
static __device__ __forceinline__ double plane_t(const PlanGeo64 &g, double x) {
    return __ddiv_rn(__dsub_rn(g.Xm, x), __dsub_rn(g.Xd, x));
}

// Mask row crossed by the rays from depth i to detector row m, -1 outside the mask.
static __device__ __forceinline__ int mask_row(const PlanGeo64 &g, int i, int m) {
    const double tt = plane_t(g, vox_x(g, i));
    const double zm = __dmul_rn(tt, pix_z(g, m));
    const double rf = floor(__ddiv_rn(__dsub_rn(zm, g.z0), g.cell));
    return (rf < 0 || rf >= g.rows) ? -1 : (int)rf;
}

// Mask column crossed by the rays from voxel (i, j) to detector column n, -1 outside.
static __device__ __forceinline__ int mask_col(const PlanGeo64 &g, int i, int j, int n) {
    const double x = vox_x(g, i), y = vox_y(g, j);
    const double tt = plane_t(g, x);
    const double ym = __dadd_rn(y, __dmul_rn(tt, __dsub_rn(pix_y(g, n), y)));
    const double cf = floor(__ddiv_rn(__dsub_rn(ym, g.y0), g.cell));
    return (cf < 0 || cf >= g.cols) ? -1 : (int)cf;
}

// The same cell decisions from an FP32 estimate, falling back to the FP64 formula
// when the estimate is within MASK_EDGE cell widths of a cell edge.  The FP32
// estimate's error is far below MASK_EDGE (a few ulps of coordinates below 10^3
// cell widths), so away from the edges the floor of the estimate is the floor of
// the exact value, and next to them the FP64 formula decides: the result equals
// mask_row / mask_col.
#define MASK_EDGE 4e-3f

struct MaskGeo32 {
    float xc, dx, ymul, py, pz, Xd, Xm, inv_cell, y0, z0;
    float hx, hj, hn, hm;   // (X-1)/2, (J-1)/2, (N-1)/2, (M-1)/2
};

inline MaskGeo32 mask_geo32(const PlanGeo64 &g) {
    MaskGeo32 m;
    m.xc = (float)g.xc; m.dx = (float)g.dx; m.ymul = (float)(g.rho_y * g.py); m.py = (float)g.py;
    m.pz = (float)g.pz; m.Xd = (float)g.Xd; m.Xm = (float)g.Xm; m.inv_cell = (float)(1.0 / g.cell);
    m.y0 = (float)g.y0; m.z0 = (float)g.z0;
    m.hx = 0.5f * (float)(g.X - 1); m.hj = 0.5f * (float)(g.J - 1); m.hn = 0.5f * (float)(g.N - 1);
    m.hm = 0.5f * (float)(g.M - 1);
    return m;
}

static __device__ __forceinline__ bool near_edge(float u) { return fabsf(u - rintf(u)) < MASK_EDGE; }

static __device__ __forceinline__ int mask_row_fast(const PlanGeo64 &g, const MaskGeo32 &h, int i, int m) {
    const float x = fmaf((float)i - h.hx, h.dx, h.xc);
    const float t = (h.Xm - x) / (h.Xd - x);
    const float u = (t * (((float)m - h.hm) * h.pz) - h.z0) * h.inv_cell;
    if (near_edge(u)) return mask_row(g, i, m);
    const float r = floorf(u);
    return (r < 0.f || r >= (float)g.rows) ? -1 : (int)r;
}

static __device__ __forceinline__ int mask_col_fast(const PlanGeo64 &g, const MaskGeo32 &h, int i, int j, int n) {
    const float x = fmaf((float)i - h.hx, h.dx, h.xc);
    const float t = (h.Xm - x) / (h.Xd - x);
    const float y = ((float)j - h.hj) * h.ymul, yn = ((float)n - h.hn) * h.py;
    const float u = (fmaf(t, yn - y, y) - h.y0) * h.inv_cell;
    if (near_edge(u)) return mask_col(g, i, j, n);
    const float c = floorf(u);
    return (c < 0.f || c >= (float)g.cols) ? -1 : (int)c;
}
