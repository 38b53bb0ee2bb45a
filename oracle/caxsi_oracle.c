/*
 * FP64 CPU oracle for the fan-beam coded-aperture coherent-scatter forward
 * model g = A f and its adjoint (backward model) f = A^T w.
 *
 * TEST INFRASTRUCTURE ONLY.  Only the test suite, the smoke check and the
 * benchmark's CPU-baseline leg load this library.  It shares no code, header
 * or table with the CUDA library and does not include anything from it.
 *
 * What it computes (Odinaka et al., "Joint System and Algorithm Design for
 * Computationally Efficient Fan Beam Coded Aperture X-ray Coherent Scatter
 * Imaging"):
 *
 *   g(r') = C sum_r G_so(r) G_od(s) T(r, r') dtheta W(r, theta)      (Eq. 3)
 *   W(r, theta) = int S(theta, q) f(r, q) dq                          (Eq. 4)
 *
 * with G_so = x/(x^2+y^2)^1.5, G_od = |n_d . s_hat|/s^2 (Eq. 2 and
 * Appendix A, n_d = x_hat), the scatter angle theta between r and
 * s = r' - r (Sec. II), dtheta the angle between the scatter vectors to the
 * midpoints of the pixel's two z edges (Appendix A), and T the binary mask
 * value where the ray r -> r' crosses the mask plane (Appendix A).
 *
 * The q integral of Eq. 4 is evaluated in its energy form: substituting
 * E = hc q / sin(theta/2) (Bragg's law, Appendix A) into S(theta, q) dq gives
 * (1 + cos^2 theta) cos(theta/2) Phi(E) E / (hc)^2 dE, and the energy integral
 * is taken over K midpoint bins:
 *
 *   W(r, theta) = (1 + cos^2 theta) cos(theta/2)
 *                 * sum_k Phi_k E_k dE / hc^2 * f~(r, q_k),
 *   q_k = E_k sin(theta/2) / hc,
 *
 * where f~ is the linear interpolation of the q-grid samples f(r, q_l),
 * q_l = q_min + l dq, extended by a zero sample one step beyond each end of
 * the grid (equivalently f~ = sum_l f_l hat((q - q_l)/dq)).
 *
 * The forward loop follows Algorithm 1 (object point, detector point, then
 * the spectral sum) with the detector points distributed over threads; the
 * adjoint follows Algorithm 3 (object point, then detector point, spectral
 * weights transposed onto the q bins) with the object points distributed
 * over threads.  Nothing is tabulated, blocked or reused between pairs.
 */
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>
#ifdef _OPENMP
#include <omp.h>
#endif

typedef struct {
    int X, J, Q, M, N, K, rho_y, mask_rows, mask_cols;
    double x_center, dx, p_y, p_z, X_det, X_mask;
    double q_min, q_max, E_min, E_max, hc, C;
    double mask_cell, mask_y0, mask_z0;
} og_geom;

/* Per-pair factors, returned to the tests through oracle_pair(). */
typedef struct {
    double x, y, yp, zp;      /* object point (x, y, 0), detector point (X_d, yp, zp) */
    double Gso, God, dtheta;  /* geometric factors */
    double theta, u;          /* scatter angle and u = sin(theta/2) */
    double T;                 /* mask transmission (0 or 1) */
    double mask_y, mask_z;    /* crossing point on the mask plane */
    double angular;           /* (1 + cos^2 theta) cos(theta/2) */
} og_pair;

/* Voxel and pixel centres: the source sits at the origin, the fan in z = 0,
 * the object region and the detector are centred on the central ray (Sec. II,
 * Sec. III-A), the object pitch along y is rho_y detector pitches. */
static double vox_x(const og_geom *g, int i) { return g->x_center + (i - 0.5 * (g->X - 1)) * g->dx; }
static double vox_y(const og_geom *g, int j) { return (j - 0.5 * (g->J - 1)) * g->rho_y * g->p_y; }
static double pix_y(const og_geom *g, int n) { return (n - 0.5 * (g->N - 1)) * g->p_y; }
static double pix_z(const og_geom *g, int m) { return (m - 0.5 * (g->M - 1)) * g->p_z; }

static double norm3(double a, double b, double c) { return sqrt(a * a + b * b + c * c); }

/* Angle between two 3-vectors: atan2(|a x b|, a . b). */
static double angle_between(const double a[3], const double b[3]) {
    double cx = a[1] * b[2] - a[2] * b[1];
    double cy = a[2] * b[0] - a[0] * b[2];
    double cz = a[0] * b[1] - a[1] * b[0];
    double dot = a[0] * b[0] + a[1] * b[1] + a[2] * b[2];
    return atan2(norm3(cx, cy, cz), dot);
}

/* Binary mask value where the ray from r to r' crosses the plane x = X_mask;
 * zero outside the mask array (Appendix A). */
static double mask_value(const og_geom *g, const uint8_t *mask, double x, double y,
                         double yp, double zp, double *my, double *mz) {
    double t = (g->X_mask - x) / (g->X_det - x);
    double ym = y + t * (yp - y);
    double zm = t * zp;
    *my = ym;
    *mz = zm;
    double cf = floor((ym - g->mask_y0) / g->mask_cell);
    double rf = floor((zm - g->mask_z0) / g->mask_cell);
    if (cf < 0 || rf < 0 || cf >= g->mask_cols || rf >= g->mask_rows) return 0.0;
    return mask[(long)rf * g->mask_cols + (long)cf] ? 1.0 : 0.0;
}

static void pair_factors(const og_geom *g, const uint8_t *mask, int i, int j, int m, int n,
                         og_pair *o) {
    double x = vox_x(g, i), y = vox_y(g, j), yp = pix_y(g, n), zp = pix_z(g, m);
    double r[3] = {x, y, 0.0};
    double s[3] = {g->X_det - x, yp - y, zp};
    double slen = norm3(s[0], s[1], s[2]);
    o->x = x; o->y = y; o->yp = yp; o->zp = zp;
    /* G_so = x / (x^2 + y^2)^1.5 */
    o->Gso = x / pow(x * x + y * y, 1.5);
    /* G_od = |n_d . s_hat| / s^2 with n_d = x_hat */
    o->God = fabs(s[0]) / (slen * slen * slen);
    /* dtheta: angle between the scatter vectors to the two z edges of the pixel */
    double h = 0.5 * g->p_z;
    double sp[3] = {s[0], s[1], s[2] + h};
    double sm[3] = {s[0], s[1], s[2] - h};
    o->dtheta = angle_between(sp, sm);
    /* scatter angle between r_hat and s_hat */
    o->theta = angle_between(r, s);
    o->u = sin(0.5 * o->theta);
    o->angular = (1.0 + cos(o->theta) * cos(o->theta)) * cos(0.5 * o->theta);
    o->T = mask_value(g, mask, x, y, yp, zp, &o->mask_y, &o->mask_z);
}

/* Linear interpolation of the q samples at fractional bin tau, with a zero
 * sample one step beyond each end of the grid. */
static double f_interp(const double *frow, int Q, double tau) {
    if (!(tau > -1.0 && tau < (double)Q)) return 0.0;
    double lf = floor(tau);
    int l = (int)lf;
    double a = tau - lf;
    double f0 = (l >= 0 && l <= Q - 1) ? frow[l] : 0.0;
    double f1 = (l + 1 >= 0 && l + 1 <= Q - 1) ? frow[l + 1] : 0.0;
    return (1.0 - a) * f0 + a * f1;
}

static double energy_k(const og_geom *g, int k) {
    double dE = (g->E_max - g->E_min) / g->K;
    return g->E_min + (k + 0.5) * dE;
}

/* Effective spectral factor W(r, theta) of Eq. 4 in energy form. */
static double w_energy(const og_geom *g, const double *phi, const double *frow, const og_pair *p) {
    double dE = (g->E_max - g->E_min) / g->K;
    double dq = (g->q_max - g->q_min) / (g->Q - 1);
    double acc = 0.0;
    for (int k = 0; k < g->K; ++k) {
        double E = energy_k(g, k);
        double q = E * p->u / g->hc;               /* Bragg's law */
        double ck = phi[k] * E * dE / (g->hc * g->hc);
        acc += ck * f_interp(frow, g->Q, (q - g->q_min) / dq);
    }
    return p->angular * acc;
}

static void set_threads(int nthreads) {
#ifdef _OPENMP
    if (nthreads > 0) omp_set_num_threads(nthreads);
#else
    (void)nthreads;
#endif
}

int oracle_max_threads(void) {
#ifdef _OPENMP
    return omp_get_max_threads();
#else
    return 1;
#endif
}

void oracle_pair(const og_geom *g, const uint8_t *mask, int i, int j, int m, int n, og_pair *out) {
    pair_factors(g, mask, i, j, m, n, out);
}

/* W(r, theta) for one pair and one q row (exposed for the change-of-variables pin). */
double oracle_w_energy(const og_geom *g, const double *phi, const uint8_t *mask,
                       const double *frow, int i, int j, int m, int n) {
    og_pair p;
    pair_factors(g, mask, i, j, m, n, &p);
    return w_energy(g, phi, frow, &p);
}

/* Forward model (Algorithm 1) for a list of detector pixels p = m*N + n. */
void oracle_forward_pixels(const og_geom *g, const double *phi, const uint8_t *mask,
                           const double *f, const long *pix, long npix, double *out,
                           int nthreads) {
    set_threads(nthreads);
#pragma omp parallel for schedule(dynamic, 1)
    for (long t = 0; t < npix; ++t) {
        int m = (int)(pix[t] / g->N), n = (int)(pix[t] % g->N);
        double acc = 0.0;
        for (int i = 0; i < g->X; ++i)
            for (int j = 0; j < g->J; ++j) {
                og_pair p;
                pair_factors(g, mask, i, j, m, n, &p);
                const double *frow = f + ((long)i * g->J + j) * g->Q;
                double W = w_energy(g, phi, frow, &p);
                acc += p.Gso * p.God * p.T * p.dtheta * W;
            }
        out[t] = g->C * acc;
    }
}

void oracle_forward(const og_geom *g, const double *phi, const uint8_t *mask, const double *f,
                    double *out, int nthreads) {
    long npix = (long)g->M * g->N;
    long *pix = (long *)malloc(sizeof(long) * npix);
    for (long t = 0; t < npix; ++t) pix[t] = t;
    oracle_forward_pixels(g, phi, mask, f, pix, npix, out, nthreads);
    free(pix);
}

/* Backward model (Algorithm 3) for a list of voxels v = i*J + j; out is
 * [nvox][Q].  For every pixel and energy the interpolation weights of f~ are
 * transposed onto the two q bins they touch. */
void oracle_adjoint_voxels(const og_geom *g, const double *phi, const uint8_t *mask,
                           const double *w, const long *vox, long nvox, double *out,
                           int nthreads) {
    set_threads(nthreads);
    double dE = (g->E_max - g->E_min) / g->K;
    double dq = (g->q_max - g->q_min) / (g->Q - 1);
#pragma omp parallel for schedule(dynamic, 1)
    for (long t = 0; t < nvox; ++t) {
        int i = (int)(vox[t] / g->J), j = (int)(vox[t] % g->J);
        double *frow = out + t * g->Q;
        for (int l = 0; l < g->Q; ++l) frow[l] = 0.0;
        for (int m = 0; m < g->M; ++m)
            for (int n = 0; n < g->N; ++n) {
                og_pair p;
                pair_factors(g, mask, i, j, m, n, &p);
                double base = p.Gso * p.God * p.T * p.dtheta * p.angular * w[(long)m * g->N + n];
                if (base == 0.0) continue;
                for (int k = 0; k < g->K; ++k) {
                    double E = energy_k(g, k);
                    double q = E * p.u / g->hc;
                    double ck = phi[k] * E * dE / (g->hc * g->hc);
                    double tau = (q - g->q_min) / dq;
                    if (!(tau > -1.0 && tau < (double)g->Q)) continue;
                    double lf = floor(tau);
                    int l = (int)lf;
                    double a = tau - lf;
                    if (l >= 0 && l <= g->Q - 1) frow[l] += base * ck * (1.0 - a);
                    if (l + 1 >= 0 && l + 1 <= g->Q - 1) frow[l + 1] += base * ck * a;
                }
            }
        for (int l = 0; l < g->Q; ++l) frow[l] *= g->C;
    }
}

void oracle_adjoint(const og_geom *g, const double *phi, const uint8_t *mask, const double *w,
                    double *out, int nthreads) {
    long nvox = (long)g->X * g->J;
    long *vox = (long *)malloc(sizeof(long) * nvox);
    for (long t = 0; t < nvox; ++t) vox[t] = t;
    oracle_adjoint_voxels(g, phi, mask, w, vox, nvox, out, nthreads);
    free(vox);
}

/* Dense system matrix H[p][v*Q + l] (Eq. 5's H_{i,j} with the image ordered
 * lexicographically as voxel-major, q-minor), formed entry by entry: each
 * entry is the forward model applied to the unit vector e_{v,l}.  Only for
 * tiny instances. */
void oracle_assemble_H(const og_geom *g, const double *phi, const uint8_t *mask, double *H) {
    long P = (long)g->M * g->N, V = (long)g->X * g->J;
    long cols = V * g->Q;
    double *e = (double *)calloc((size_t)g->Q, sizeof(double));
    for (long p = 0; p < P; ++p) {
        int m = (int)(p / g->N), n = (int)(p % g->N);
        for (long v = 0; v < V; ++v) {
            int i = (int)(v / g->J), j = (int)(v % g->J);
            og_pair pr;
            pair_factors(g, mask, i, j, m, n, &pr);
            for (int l = 0; l < g->Q; ++l) {
                e[l] = 1.0;
                double W = w_energy(g, phi, e, &pr);
                e[l] = 0.0;
                H[p * cols + v * g->Q + l] = g->C * pr.Gso * pr.God * pr.T * pr.dtheta * W;
            }
        }
    }
    free(e);
}
