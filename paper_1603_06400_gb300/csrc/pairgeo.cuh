// Scatter angle of one (voxel, pixel) pair in FP32 (Sec. II: theta is the
// angle between r = (x, y, 0) and s = r' - r).
//
// Returns u = sin(theta/2) and the angular factor (1 + cos^2 theta) cos(theta/2)
// of the spectral factor S(theta, q).  For Bragg's law q = E u / hc the
// interpolation position needs u to a few ulps even for theta ~ 1e-3 rad,
// where 1 - cos(theta) cancels.  So the angle is built from the exact scalar
// products:
//   Dt = r . s,  |r x s|^2 = s_z^2 |r|^2 + D^2,  D = x s_y - y s_x,
//   P^2 = Dt^2 + |r x s|^2 (= |r|^2 |s|^2),
//   u = |r x s| / sqrt(2 P (P + Dt)),  cos(theta/2) = sqrt((P + Dt) / (2 P)).
// The y coordinates are carried in units of the detector pitch p_y, where
// voxel and pixel centres are exact half-integers: Y = y/p_y, S_y = s_y/p_y.
// Then D = p_y (x S_y - Y s_x), and the 2x2 determinant is evaluated with an
// FMA-compensated product (Kahan's method), so D keeps its relative accuracy
// when x S_y and Y s_x nearly cancel (pixels close to the continuation of the
// incident ray).  s_x = X_det - x is exact in FP32 when X_det/2 <= x <= X_det.
#pragma once

__device__ __forceinline__ void pair_u_angular(float x, float Y, float r2, float Npix, float sz,
                                               float py, float Xd, float &u, float &ang) {
    const float sx = Xd - x;
    const float Sy = Npix - Y;
    const float w = Y * sx;
    const float e = fmaf(Y, sx, -w);
    const float Dp = fmaf(x, Sy, -w) - e;
    const float D = py * Dp;
    const float Dt = fmaf(x, sx, (py * Y) * (py * Sy));
    const float Cr2 = fmaf(sz * sz, r2, D * D);
    const float P2 = fmaf(Dt, Dt, Cr2);
    const float P = sqrtf(P2);
    const float q1 = P + Dt;
    const float twoP = 2.f * P;
    u = sqrtf(Cr2 / (twoP * q1));
    const float c = Dt / P;
    ang = fmaf(c, c, 1.f) * sqrtf(q1 / twoP);
}
