/*
 * caxsi.h -- C ABI of the GB300 (sm_103a) library for the fan-beam
 * coded-aperture X-ray coherent-scatter forward model g = A f and its
 * adjoint f = A^T w (Odinaka et al., arXiv:1603.06400).
 *
 * Model (Sec. II, Eq. 1-4, Appendix A).  With the source at the origin and
 * the fan in the plane z = 0, object voxel (i, j) sits at r = (x_i, y_j, 0)
 * and detector pixel (m, n) at r' = (X_det, y'_n, z'_m); s = r' - r.  Then
 *
 *   g[m][n] = C sum_{i,j} G_so(r) G_od(s) T(r, r') dtheta(s) W(r, theta),
 *   W(r, theta) = (1 + cos^2 theta) cos(theta/2)
 *                 * sum_k Phi_k E_k dE / hc^2 * f~(r, E_k sin(theta/2) / hc),
 *
 * G_so = x/(x^2+y^2)^1.5, G_od = |s_x|/|s|^3, theta the angle between r and
 * s, dtheta the angle between the scatter vectors to the pixel's two z edges,
 * T the binary mask value where the ray crosses the mask plane x = X_mask,
 * E_k the midpoints of K equal energy bins on [E_min, E_max] (the energy form
 * of Eq. 4 under Bragg's law q = E sin(theta/2)/hc), and f~ the linear
 * interpolation of the samples f[i][j][l] at q_l = q_min + l dq,
 * dq = (q_max - q_min)/(Q - 1), with a zero sample one step beyond each end.
 *
 * Layouts (all row-major, float32 on the device unless stated):
 *   f : [X][J][Q]  voxel i along the central ray, j across the fan, q fastest
 *       (the lexicographic voxel-by-channel order of Eq. 5).
 *   g, w, y, r : [M][N]  detector row m (z), column n (y), n fastest.
 *
 * Centres: x_i = x_center + (i - (X-1)/2) dx, y_j = (j - (J-1)/2) rho_y p_y,
 *          y'_n = (n - (N-1)/2) p_y, z'_m = (m - (M-1)/2) p_z.
 * The object pitch along y is rho_y detector pitches (Sec. III-A translation
 * symmetry).  Mask cell (row, col) covers
 *   [mask_z0 + row*cell, +cell) x [mask_y0 + col*cell, +cell) on the mask plane;
 * the transmission is 0 outside the mask array.
 *
 * Ownership and streams.  The caller owns every buffer passed in and the
 * stream (a cudaStream_t passed as void*, NULL = legacy default stream).
 * A plan owns its device tables and its scratch; entry points that take
 * device pointers are asynchronous on the given stream unless stated.  Calls
 * that share one plan must be ordered (same stream, or synchronised by the
 * caller): they share the plan's scratch memory.
 *
 * Errors.  Every entry point returns a caxsi_status; nothing is thrown across
 * the ABI and nothing aborts.  Null pointers, wrong lengths and invalid
 * geometry give CAXSI_ERR_INVALID without launching anything.  A CUDA
 * failure gives CAXSI_ERR_CUDA.
 */
#ifndef CAXSI_H
#define CAXSI_H

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef struct caxsi_plan caxsi_plan;

typedef enum {
    CAXSI_OK = 0,
    CAXSI_ERR_INVALID = 1,      /* bad argument: null pointer, length, geometry */
    CAXSI_ERR_CUDA = 2,         /* a CUDA runtime call or launch failed */
    CAXSI_ERR_OOM = 3,          /* device allocation failed */
    CAXSI_ERR_NONPOS_MEAN = 4,  /* a positive count met a non-positive mean A f + r */
    CAXSI_ERR_INTERNAL = 5,     /* a device-side consistency check failed */
    CAXSI_ERR_UNSUPPORTED = 6,  /* option not available for this plan */
    CAXSI_ERR_SCRATCH_LIMIT = 7 /* problem larger than a fixed scratch array allows */
} caxsi_status;

/* How A and A^T are evaluated.
 * DIRECT: the energy sum of Eq. 4 per (voxel, pixel) pair in FP32 (Alg. 1 / 3
 *   structure, all factors computed or fetched per pair).
 * TABLE_FP32: the same operator evaluated exactly through the piecewise-
 *   linear structure of W in u = sin(theta/2): W(r, u) is tabulated per voxel
 *   at every u where some energy bin crosses a q-grid node (so that linear
 *   interpolation in u between table entries is exact), the table is a
 *   contraction over q, and each pair interpolates it (forward) or scatters
 *   into its transposed table (adjoint).  FP32 arithmetic throughout.
 * TABLE_BF16 / TABLE_FP16: as TABLE_FP32 with the contraction over q on
 *   tensor cores with bf16 / fp16 operands and FP32 accumulation (reduced
 *   precision; the error against FP64 is measured, not bounded to 1e-5).  The
 *   tables the contractions produce and consume (W and V, one row per voxel) are
 *   kept in 16 bits where the mirror-symmetric records are used (bf16 for
 *   TABLE_BF16's W and V, fp16 for TABLE_FP16's V; TABLE_FP16's W stays FP32,
 *   as fp16's range would not hold every value).  TABLE_BF16's adjoint also
 *   streams the mirror-symmetric adjoint records' pair weights w0, w1 as bf16 (a
 *   copy that the plan keeps beside the FP32 one); the knot interval of each
 *   pair, the mask factors, the forward's pair weights and all accumulations
 *   stay exact / FP32. */
typedef enum {
    CAXSI_PATH_DIRECT = 0,
    CAXSI_PATH_TABLE_FP32 = 1,
    CAXSI_PATH_TABLE_BF16 = 2,
    CAXSI_PATH_TABLE_FP16 = 3
} caxsi_path;

/* System description; lengths in mm, energies in keV, q in nm^-1 (so that
 * hc = 1.23984193 keV nm).  Requirements: X, J, M, N, K >= 1; Q >= 2;
 * rho_y >= 1; K <= 1024; dx, p_y, p_z, mask_cell > 0; 0 < x_i < X_mask <
 * X_det for every voxel; q_min < q_max; 0 < E_min < E_max; hc > 0. */
typedef struct {
    int32_t X, J, Q, M, N, K, rho_y, mask_rows, mask_cols;
    double x_center, dx, p_y, p_z, X_det, X_mask;
    double q_min, q_max, E_min, E_max, hc, C;
    double mask_cell, mask_y0, mask_z0;
} caxsi_geometry;

/* Build a plan on the current CUDA device: validates the geometry, uploads the
 * spectrum and mask, and builds the device tables in FP64 kernels (per-voxel
 * position and G_so, per-offset G_od * dtheta -- one entry per scatter vector,
 * shared by all voxel/pixel pairs related by the translation symmetry of
 * Sec. III-A -- and the precomputed binary mask factor of every pair, as the
 * paper precomputes its mask factors offline, Sec. III-C).
 *   geom      host pointer, read during the call.
 *   phi_host  host pointer to K doubles: the bin-averaged spectrum Phi_k.
 *   mask_host host pointer to mask_rows * mask_cols bytes, 0 = opaque,
 *             nonzero = open, row = z cell, col = y cell.
 *   out       receives the plan; unchanged on error.
 * Synchronous.  Errors: INVALID, OOM, CUDA. */
caxsi_status caxsi_plan_create(const caxsi_geometry *geom, const double *phi_host,
                               const uint8_t *mask_host, caxsi_plan **out);

/* Release a plan and all device memory it owns (synchronises the device
 * first).  NULL is ignored. */
void caxsi_plan_destroy(caxsi_plan *plan);

/* Forward model g = A f (Eq. 3 with Eq. 4; Algorithm 1's sum over object
 * points, detector points and the spectrum).
 *   f_dev  device, f_len = X*J*Q floats, layout [X][J][Q].
 *   g_dev  device, g_len = M*N floats, layout [M][N]; overwritten.
 *   path   a caxsi_path.
 * Asynchronous on stream.  Errors: INVALID, UNSUPPORTED, CUDA, OOM. */
caxsi_status caxsi_forward(caxsi_plan *plan, const float *f_dev, int64_t f_len,
                           float *g_dev, int64_t g_len, int path, void *stream);

/* Backward model f = A^T w (the exact transpose of caxsi_forward; Algorithm 3
 * of Sec. IV with the spectral interpolation weights transposed onto the q
 * bins).
 *   w_dev  device, w_len = M*N floats.
 *   f_dev  device, f_len = X*J*Q floats; overwritten.
 * Asynchronous on stream.  Errors: INVALID, UNSUPPORTED, CUDA, OOM. */
caxsi_status caxsi_adjoint(caxsi_plan *plan, const float *w_dev, int64_t w_len,
                           float *f_dev, int64_t f_len, int path, void *stream);

/* One iteration of the EM-type algorithm of Sec. VI (Algorithm 4) for the
 * penalised Poisson likelihood of Sec. V:
 *   z = A f + r;  b2 = A^T (y / z);  f <- positive root of
 *   chi1 f^2 + chi2 f - chi3 = 0 (Eq. 10, Appendices B and C) with
 *   b1 = A^T 1 (computed on first use, cached in the plan), Huber potential
 *   psi_delta on the 4 spatial neighbours (i +- 1, j +- 1) of each voxel and
 *   q channel, unit weights.  beta = 0 gives the MLEM update f b2 / b1.
 *   y_dev     device, M*N counts (float, >= 0).
 *   r_dev     device, M*N background (>= 0) or NULL for r = 0.
 *   f_dev     device, X*J*Q, in/out (f >= 0).
 *   nll_out   host pointer or NULL.  When non-NULL the call synchronises the
 *             stream and stores the negative log-likelihood
 *             L(f_in) = sum_i z_i - y_i ln z_i + ln y_i! accumulated in FP64.
 * Edge rules: y_i = z_i = 0 contributes ratio 0 and likelihood 0; y_i > 0 with
 * z_i <= 0 gives CAXSI_ERR_NONPOS_MEAN (detected when nll_out is non-NULL, or
 * on the next call otherwise; f is then left unchanged by this call only if
 * nll_out is non-NULL).  A voxel/channel with b1 = 0 and beta = 0 keeps its
 * value.  Errors: INVALID, NONPOS_MEAN, CUDA, OOM. */
caxsi_status caxsi_recon_step(caxsi_plan *plan, const float *y_dev, const float *r_dev,
                              float *f_dev, int64_t f_len, float beta, float delta,
                              int path, double *nll_out, void *stream);

/* ---- Ordered subsets (Sec. VI, Algorithm 5) ------------------------------------
 * The detector is split into P disjoint pixel subsets; A_p is A restricted to
 * the rows (pixels) of subset p.  The paper's symmetry-preserving choice groups
 * every pixel with its left-right and up-down mirror images and with the
 * pixels a multiple of the translation step away; any partition is accepted
 * here (the Python binding builds the paper's one).  CAXSI_PATH_DIRECT
 * evaluates only the pairs of the subset's pixels, so a subset operator costs
 * about 1/P of the full one (the point of the algorithm).  The table paths
 * stream only the subset's pair records (records grouped by subset).  In FP32,
 * when the subsets average at most a few hundred records per voxel and Q is a
 * multiple of 4 up to 128, each record is contracted with its two rows of the
 * spectral matrix directly, so a subset operator costs about 1/P of a full one
 * there too; otherwise (the 16-bit paths, denser subsets) the q contractions
 * stay whole-object and a subset operator costs most of a full one.
 */
#define CAXSI_MAX_SUBSETS 1024

/* The symmetry-preserving partition of Sec. VI, as a map pixel -> subset for
 * caxsi_plan_set_subsets.  Rows: the upper half of the detector (m < M/2) is
 * split into rho_z classes of row step rho_z, and every row's mirror image about
 * the centre line z = 0 (row M-1-m) joins its class.  Columns: classes of step
 * sigma_y, every column's mirror image about y = 0 (column c -> sigma_y-1-c
 * within the step) joining its class, so sigma_y / 2 column classes.  Subset of
 * pixel (m, n) = row class * (sigma_y / 2) + column class; n_subsets =
 * rho_z * sigma_y / 2.  sigma_y keeps the translation symmetry when it is a
 * multiple of the translation step rho_y; sigma_y <= 0 picks rho_y when rho_y is
 * even and 16 rho_y otherwise (the paper's example uses a column step of 16).
 *   subset_of_pixel  host, M*N int32, written row-major in (m, n).
 * Host only (no device work).  Errors: INVALID when the output is NULL, M is
 * odd, rho_z does not divide M/2, or sigma_y is odd, does not divide N or is
 * not a multiple of rho_y. */
caxsi_status caxsi_os_partition(int M, int N, int rho_y, int rho_z, int sigma_y, int32_t *subset_of_pixel);

/* Set (or replace) the partition.  subset_of_pixel: host, M*N int32 in
 * [0, n_subsets), row-major (m, n).  Synchronises the device first (work in
 * flight may still read the old partition), uploads the subsets' pixel lists,
 * drops the cached subset sensitivities and builds the table paths' records
 * grouped by subset if the plan's tables exist already; otherwise the first
 * table-path subset call builds them (that call then synchronises).
 * Errors: INVALID (sizes, an index out of range, n_subsets outside
 * [1, min(CAXSI_MAX_SUBSETS, M*N)]), CUDA, OOM.  Where the geometry has no pair
 * records (more than 65536 pixels or knots) the partition still serves the
 * direct path, and the table paths' subset calls return UNSUPPORTED. */
caxsi_status caxsi_plan_set_subsets(caxsi_plan *plan, int n_subsets, const int32_t *subset_of_pixel);

/* g = A_p f: g_dev (M*N, device) holds the subset's pixels of A f and 0 at every
 * other pixel.  Same arguments and errors as caxsi_forward, plus subset in
 * [0, n_subsets) (INVALID otherwise or before caxsi_plan_set_subsets). */
caxsi_status caxsi_forward_subset(caxsi_plan *plan, int subset, const float *f_dev, int64_t f_len,
                                  float *g_dev, int64_t g_len, int path, void *stream);

/* f = A_p^T w: only the subset's pixels of w_dev are read.  Arguments and
 * errors as caxsi_forward_subset. */
caxsi_status caxsi_adjoint_subset(caxsi_plan *plan, int subset, const float *w_dev, int64_t w_len,
                                  float *f_dev, int64_t f_len, int path, void *stream);

/* One inner step of the ordered-subset EM-type algorithm (Algorithm 5):
 *   z_p = A_p f + r_p;  b2_p = A_p^T (y_p / z_p);  f <- Eq. 10 with b1_p = A_p^T 1
 *   (computed on first use per subset and path, cached in the plan).
 * Only the subset's pixels of y_dev and r_dev are read; nll_out receives the
 * subset's likelihood L_p(f_in).  beta is the penalty weight of this step: the
 * ordered-subset pass of the Python binding passes beta / P, so that the
 * subset's data term stands for 1/P of the full one.  Edge rules and errors as
 * caxsi_recon_step, plus those of caxsi_forward_subset. */
caxsi_status caxsi_recon_step_subset(caxsi_plan *plan, int subset, const float *y_dev, const float *r_dev,
                                     float *f_dev, int64_t f_len, float beta, float delta, int path,
                                     double *nll_out, void *stream);

/* ---- Batches of objects ------------------------------------------------------
 * n_objects objects share the plan's geometry, spectrum and mask; object b is
 * the voxel range [voxel_ranges[2b], voxel_ranges[2b+1]) of the voxel index
 * v = i*J + j (depth slabs of uneven extent), with its own f block
 * f_dev + b*X*J*Q ([X][J][Q], voxels outside its range are not read) and its own
 * detector image g_dev + b*M*N.  The paper has no batched operator: it serves
 * training and many-object reconstruction (one launch per stage for the whole
 * batch).  The q contraction is one GEMM over the packed rows of all objects'
 * voxels, and the pair streaming runs per voxel chunk of each object, so each
 * object's result is bit-identical to caxsi_forward / caxsi_adjoint on that
 * object alone with f = 0 outside its range (the adjoint's f is 0 outside the
 * range; the single forward with CAXSI_OPT_SYMMETRY 0, since batches stream one
 * record per open pair).  CAXSI_PATH_TABLE_FP32 with the tcgen05 engine only (UNSUPPORTED
 * otherwise).  voxel_ranges is host memory; the call is asynchronous on stream
 * after a synchronous upload when the layout changes.  Errors: INVALID (sizes,
 * ranges outside [0, X*J], n_objects outside [1, CAXSI_MAX_BATCH]),
 * UNSUPPORTED, CUDA, OOM. */
#define CAXSI_MAX_BATCH 4096
caxsi_status caxsi_forward_batch(caxsi_plan *plan, int n_objects, const int32_t *voxel_ranges,
                                 const float *f_dev, int64_t f_len, float *g_dev, int64_t g_len, int path,
                                 void *stream);
caxsi_status caxsi_adjoint_batch(caxsi_plan *plan, int n_objects, const int32_t *voxel_ranges,
                                 const float *w_dev, int64_t w_len, float *f_dev, int64_t f_len, int path,
                                 void *stream);

/* ---- Objects of different geometries in one launch -----------------------------
 * A multi-object set groups n_objects plans, each with its own geometry (object
 * extents X, J, Q, detector, spectrum, mask), so that the forward model or the
 * adjoint of every object runs in ONE persistent kernel launch: the launch's
 * blocks (forward) or warps (adjoint) take work items -- an object's voxel chunk
 * and 8 x 32 detector tile for A, an object's voxel and detector row range for
 * A^T, the units of the single-plan direct kernels -- from an atomic counter
 * until none is left (no waits: a pop never polls), and the item that completes
 * an output region sums its partial results in ascending order.  Each object's
 * result is bit-identical to caxsi_forward / caxsi_adjoint on its own plan with
 * CAXSI_PATH_DIRECT, whatever the order the items ran in.  The paper evaluates
 * one object at a time; the set serves batched and differentiable
 * reconstruction of objects of uneven sizes (training data, unrolled
 * iterations).
 *
 * Packed layouts: object b's f is the X_b*J_b*Q_b floats ([X_b][J_b][Q_b]) at
 * offset F_b = sum_{c<b} X_c J_c Q_c of f_dev, its detector image the M_b*N_b
 * floats at offset G_b = sum_{c<b} M_c N_c of g_dev / w_dev (caxsi_multi_layout
 * returns F_0..F_n and G_0..G_n).
 *
 * The set refers to the plans (it does not own them) and uses their scratch:
 * destroy it before them, and order its calls with the plans' own calls.  All
 * plans must be on one device, and a plan may appear only once (its scratch holds
 * its object's partial results).  Errors: INVALID (NULL, lengths, plans on
 * different devices, a plan given twice, n_objects outside [1, CAXSI_MAX_MULTI]), UNSUPPORTED (a
 * path other than CAXSI_PATH_DIRECT; shared memory too small for the largest
 * K and Q), CUDA, OOM. */
#define CAXSI_MAX_MULTI 4096
typedef struct caxsi_multi caxsi_multi;
caxsi_status caxsi_multi_create(caxsi_plan *const *plans, int n_objects, caxsi_multi **out);
void caxsi_multi_destroy(caxsi_multi *multi);
/* f_offsets, g_offsets: host arrays of n_objects + 1 entries, filled with F_b, G_b. */
caxsi_status caxsi_multi_layout(const caxsi_multi *multi, int64_t *f_offsets, int64_t *g_offsets);
/* g = A f for every object (f_len = F_n, g_len = G_n); one launch.  Asynchronous. */
caxsi_status caxsi_multi_forward(caxsi_multi *multi, const float *f_dev, int64_t f_len, float *g_dev,
                                 int64_t g_len, int path, void *stream);
/* f = A^T w for every object (w_len = G_n, f_len = F_n); one launch.  Asynchronous. */
caxsi_status caxsi_multi_adjoint(caxsi_multi *multi, const float *w_dev, int64_t w_len, float *f_dev,
                                 int64_t f_len, int path, void *stream);
/* The update of Eq. 10 (as caxsi_em_update) for every object with its own
 * geometry and neighbourhoods, f_len = F_n, one launch; and its reverse mode (as
 * caxsi_em_update_vjp), two launches.  Outputs must not overlap inputs (INVALID). */
caxsi_status caxsi_multi_em_update(caxsi_multi *multi, const float *f_dev, const float *b1_dev,
                                   const float *b2_dev, float beta, float delta, float *f_out_dev,
                                   int64_t f_len, void *stream);
caxsi_status caxsi_multi_em_update_vjp(caxsi_multi *multi, const float *f_dev, const float *b1_dev,
                                       const float *b2_dev, float beta, float delta,
                                       const float *grad_out_dev, float *grad_f_dev, float *grad_b2_dev,
                                       int64_t f_len, void *stream);

/* ---- The update step as a differentiable function ------------------------------
 * caxsi_em_update: f_out = the closed-form update of Eq. 10 (the Lemma's positive
 * root with the Huber penalty of caxsi_recon_step) from f, b1 = A^T 1 and
 * b2 = A^T (y / z), elementwise with the 4-neighbour stencil; f_len is a multiple
 * of X*J*Q (objects of this geometry back to back, each with its own
 * neighbourhoods).  All pointers device; f_out must not overlap f (INVALID).
 * caxsi_em_update_vjp: the reverse mode of caxsi_em_update: given grad_out =
 * dL/df_out, writes grad_f = dL/df and grad_b2 = dL/db2 (b1 is treated as a
 * constant), by implicit differentiation of the root
 * ((2 chi1 x + chi2) dx = dchi3 - x dchi2 - x^2 dchi1) through the Huber terms
 * (derivatives taken one-sided at |f_j - f_k| = delta).  Used with A and A^T to
 * unroll the reconstruction under automatic differentiation; the paper has no
 * such step.  grad_f and grad_b2 must not overlap each other or any input
 * (INVALID).  Errors: INVALID, CUDA, OOM. */
caxsi_status caxsi_em_update(caxsi_plan *plan, const float *f_dev, const float *b1_dev, const float *b2_dev,
                             float beta, float delta, float *f_out_dev, int64_t f_len, void *stream);
caxsi_status caxsi_em_update_vjp(caxsi_plan *plan, const float *f_dev, const float *b1_dev,
                                 const float *b2_dev, float beta, float delta, const float *grad_out_dev,
                                 float *grad_f_dev, float *grad_b2_dev, int64_t f_len, void *stream);

/* ---- The likelihood ratio as a differentiable function ------------------------
 * caxsi_ratio: ratio = y / z with z = g + r (the ratio of Algorithm 4, whose
 * adjoint gives b2), elementwise over n elements (any number of detector images
 * back to back).  z > 0: y / z in FP32.  z <= 0: 0; if y > 0 there as well the
 * plan's error word is set, and the next call of this plan that returns the
 * likelihood (caxsi_recon_step with nll_out) reports CAXSI_ERR_NONPOS_MEAN.
 * caxsi_ratio_vjp: its reverse mode with respect to g: grad_g = -grad_ratio y / z^2
 * where z > 0, 0 elsewhere.  The paper has no reverse mode; it serves unrolled
 * reconstructions under automatic differentiation.
 *   g_dev, y_dev, grad_ratio_dev  device, n floats;  r_dev  device, n floats, or
 *   NULL for r = 0;  ratio_dev / grad_g_dev  device, n floats, overwritten.
 * Asynchronous on stream.  Errors: INVALID (NULL pointers, n < 1), CUDA. */
caxsi_status caxsi_ratio(caxsi_plan *plan, const float *g_dev, const float *y_dev, const float *r_dev,
                         float *ratio_dev, int64_t n, void *stream);
caxsi_status caxsi_ratio_vjp(caxsi_plan *plan, const float *g_dev, const float *y_dev, const float *r_dev,
                             const float *grad_ratio_dev, float *grad_g_dev, int64_t n, void *stream);

/* Host-buffer forms: copy the input from host memory to plan-owned device
 * staging buffers, evaluate, copy the result back to host memory, and
 * synchronise before returning.  Pinned host memory gives the fastest copies.
 * Same lengths and layouts as the device forms, and the same results bit for
 * bit.  On TABLE_FP32 the contraction over q runs in two launches over two parts
 * of the voxel rows, so that the copy of one part of f overlaps the other part's
 * contraction (forward: the last three quarters of f are copied in while the
 * first quarter is contracted; adjoint: the rows of the first wave of output tiles are copied
 * out while the rest are contracted), on a second stream that the plan creates
 * at the first such call. */
caxsi_status caxsi_forward_host(caxsi_plan *plan, const float *f_host, int64_t f_len,
                                float *g_host, int64_t g_len, int path);
caxsi_status caxsi_adjoint_host(caxsi_plan *plan, const float *w_host, int64_t w_len,
                                float *f_host, int64_t f_len, int path);

/* Plan facts for callers and benchmarks: entries of the per-offset table,
 * bytes of device tables, and the number of u breakpoints of the table paths
 * (0 until a table path is first used). */
typedef struct {
    int64_t n_offsets;        /* N + rho_y (J - 1) */
    int64_t table_bytes;      /* device bytes held by the plan */
    int64_t n_breakpoints;    /* u breakpoints of the table paths */
    int64_t kernel_launches;  /* kernels launched by the last forward/adjoint/recon call */
    int64_t n_open_pairs;     /* (voxel, pixel) pairs whose mask factor T is 1 */
    int64_t n_records;        /* precomputed pair records of the table paths (0 until built) */
    int64_t device_error;     /* 1 if a kernel of this plan gave up a bounded wait (copy or
                                 tensor-core pipeline); reading it synchronises the device
                                 and clears it */
    int64_t n_sym_records;    /* records of the mirror-symmetric adjoint, each serving up to
                                 four pairs (0 until built, or when the geometry has no
                                 mirror symmetry) */
    int64_t mask_symmetric;   /* 1 if the mask is mirror-symmetric about the central ray in
                                 y and z and J, M, N are even (CAXSI_OPT_ONLINE_MASK applies) */
} caxsi_plan_info_t;

caxsi_status caxsi_plan_info(caxsi_plan *plan, caxsi_plan_info_t *info);

/* Plan options (CAXSI_OPT_SYMMETRY below).
 *   CAXSI_OPT_GEMM_ENGINE: how the table paths evaluate their contractions
 *     over q: CAXSI_GEMM_TCGEN05 (default; this library's tcgen05 tensor-core
 *     kernel, 3xTF32 for TABLE_FP32, single pass for TABLE_BF16/FP16) or
 *     CAXSI_GEMM_CUBLAS (cuBLAS: bf16x9 emulation for TABLE_FP32).
 * Errors: INVALID for an unknown key or value. */
#define CAXSI_OPT_GEMM_ENGINE 1
#define CAXSI_GEMM_TCGEN05 0
#define CAXSI_GEMM_CUBLAS 1
/*   CAXSI_OPT_SYMMETRY: 1 (default) or 0.  With 1, the table paths' full
 *     forward and adjoint use the left-right and up-down mirror symmetries of
 *     the geometry (Sec. III-A) when J, M and N are even: one precomputed record
 *     serves a pair and its mirror images (each with its own mask factor), which
 *     about halves the bytes streamed per call.  0 streams one record per open
 *     pair.  The subset and batched operators always stream one record per open
 *     pair. */
#define CAXSI_OPT_SYMMETRY 2
/*   CAXSI_OPT_U_SAMPLES: 0 (default) or N in [2, CAXSI_MAX_U_SAMPLES].  With 0
 *     the table paths interpolate W(r, u) between the exact knots, where it is
 *     piecewise linear (exact up to rounding).  With N they sample it at N
 *     uniformly spaced u over the same range and interpolate linearly between
 *     the samples: an approximation of A (and the exact transpose of that
 *     approximation as the adjoint), the table-path counterpart of the paper's
 *     scatter-angle interpolation (Sec. III-B), with N/B of the table bytes and
 *     of the contraction work.  It must be set before the first table-path call
 *     of the plan (INVALID afterwards, unless the value is unchanged). */
#define CAXSI_OPT_U_SAMPLES 3
#define CAXSI_MAX_U_SAMPLES 8192
/*   CAXSI_OPT_GEMM_BANDS: 1 (default) or 0.  The spectral matrix S~ that the
 *     table paths contract with is zero outside a band (a knot's energies reach
 *     only a range of q bins); with 1 the tcgen05 contractions skip the product
 *     blocks that meet only those zeros.  The skipped products are exact zeros:
 *     results are unchanged, only the work shrinks.  0 multiplies everything. */
#define CAXSI_OPT_GEMM_BANDS 4
/*   CAXSI_OPT_SPARSE_SUBSETS: 1 (default) or 0.  With 1 the FP32 table path's
 *     subset operators contract only at the knots of the subset's pairs, per
 *     pair record against the rows of S~ (a subset operator then costs about
 *     1/P of a full one); 0 runs the whole-object contractions as the full
 *     operators do.  Equal up to FP32 rounding. */
#define CAXSI_OPT_SPARSE_SUBSETS 5
/*   CAXSI_OPT_ONLINE_MASK: 0 (default) or 1.  For a secondary mask that is
 *     mirror-symmetric about the central ray in y and in z (cells centred on the
 *     ray, pattern equal to its left-right and up-down images; caxsi_plan_info
 *     reports it, and J, M, N must be even), 1 makes CAXSI_PATH_DIRECT exploit
 *     the symmetric system design of Sec. III-A / III-C: the four pairs related
 *     by the left-right and up-down mirrors share geometry AND mask factor, so the
 *     forward computes each group's geometry and mask factor once and the energy
 *     sums of the two mirrored voxel columns (Algorithm 2's W_L, W_R and four
 *     detector quadrants), the adjoint one energy scatter per up-down pixel pair;
 *     the mask factor is computed online from the mask array (FP64 cell decision,
 *     as the plan builder takes it) instead of read from the per-pair bits.
 *     UNSUPPORTED for a mask without that symmetry.  The multi-object set, the
 *     subset operators and the static-scratch forward keep the per-pair bits. */
#define CAXSI_OPT_ONLINE_MASK 8
/*   CAXSI_OPT_TEST_WAIT_LIMIT, CAXSI_OPT_TEST_WITHHOLD_COPY: test hooks of the
 *     failure path, 0 in normal use.  Every wait of the record kernels for a
 *     bulk copy is bounded; WAIT_LIMIT sets the record forward's bound in polls
 *     (0 = the default, about a second), and WITHHOLD_COPY = 1 makes the record
 *     forward (CAXSI_PATH_TABLE_FP32 with CAXSI_OPT_SYMMETRY 0) skip each block's
 *     first row copy, so that the wait for it runs out: the kernel then records
 *     the error (device_error of caxsi_plan_info; CAXSI_ERR_INTERNAL from the
 *     next call that reports the likelihood), waits for the copies it did issue
 *     and returns, leaving the context usable; the call's output is then
 *     undefined.  Nothing is withheld by any other kernel. */
#define CAXSI_OPT_TEST_WAIT_LIMIT 6
#define CAXSI_OPT_TEST_WITHHOLD_COPY 7
caxsi_status caxsi_plan_set_option(caxsi_plan *plan, int key, int value);

/* Kernel timing (tracing).  When enabled, every kernel the plan launches is
 * bracketed by CUDA events recorded on its launch stream; caxsi_profile_read
 * synchronises on those events, returns per-kernel launch counts and total
 * device milliseconds (up to `capacity` distinct kernels, count in *count),
 * and clears the record.  Enabling or disabling clears the record too.
 * The event pairs add a few microseconds of host work per launch. */
typedef struct {
    char name[32];
    int64_t launches;
    double total_ms;
} caxsi_kernel_stat;

caxsi_status caxsi_profile_enable(caxsi_plan *plan, int enable);
caxsi_status caxsi_profile_read(caxsi_plan *plan, caxsi_kernel_stat *out, int capacity,
                                int *count);

/* Forward model g = A f (DIRECT path arithmetic) whose scratch lives in a
 * fixed static device array of CAXSI_STATIC_SCRATCH_FLOATS floats (4 MiB per
 * GPU that loads the library, held until the process exits) instead of the
 * plan.  The paper has no counterpart: this entry point exists for callers
 * that must not allocate device memory at the point of the call -- code that
 * runs while another thread captures a CUDA graph in global capture mode
 * (cudaMalloc fails there), real-time loops that forbid allocation after
 * start-up, or hosts whose memory pool owns all device memory.  It calls no
 * cudaMalloc, cudaFree or allocating library routine.
 *   plan      an existing plan (created beforehand, at set-up time).
 *   f_dev     device, f_len = X*J*Q floats.   g_dev  device, g_len = M*N floats.
 * The scratch holds one partial image of M*N floats per chunk of voxels, at
 * least one chunk: M*N > CAXSI_STATIC_SCRATCH_FLOATS is rejected with
 * CAXSI_ERR_SCRATCH_LIMIT before anything is launched.  The first call on a
 * device looks up the array's device address with that device current, so
 * make that first call before any stream capture.  Every call shares the one
 * array (each call overwrites all of it that it reads, so nothing carries over
 * between calls); calls that overlap on the GPU -- on several streams, several
 * plans or several host threads -- race on it and must be serialised by the
 * caller.  Asynchronous on stream.
 * Errors: INVALID, SCRATCH_LIMIT, CUDA. */
#define CAXSI_STATIC_SCRATCH_FLOATS (1 << 20)
caxsi_status caxsi_forward_static_scratch(caxsi_plan *plan, const float *f_dev, int64_t f_len,
                                          float *g_dev, int64_t g_len, void *stream);

/* Human-readable name of a status code (static storage). */
const char *caxsi_status_string(caxsi_status status);

#ifdef __cplusplus
}
#endif

#endif /* CAXSI_H */
