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
