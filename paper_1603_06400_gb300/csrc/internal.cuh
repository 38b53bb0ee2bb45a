// Internal declarations of the caxsi CUDA library (sm_103a).
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include <vector>

#include "caxsi.h"

#define CAXSI_MAX_K 1024
#define CAXSI_MAX_DEVICES 64

// Geometry scalars needed by the kernels, derived once per plan.
struct DevGeo {
    int X, J, Q, M, N, K, rho_y;
    int R;        // X * J voxels
    int ND;       // offsets d = n - rho_y j: N + rho_y (J - 1)
    int d_min;    // -rho_y (J - 1)
    int Nw;       // 32-bit words per detector row of mask bits
    float p_y;    // detector pitch along y (mm)
    float Xd;     // detector plane x (mm)
    float cN;     // (N - 1) / 2
    float b;      // q_min / dq
    float Qf;     // (float)Q
    float a0, da; // a_k = E_k / (hc dq) = a0 + k da (uniform energy bins)
};

// Optional per-kernel timing with CUDA events recorded on the launch stream
// around every kernel of the library (off by default).
struct KernelProfiler {
    bool on = false;
    struct Rec { const char *name; cudaEvent_t a, b; };
    std::vector<Rec> recs;
    std::vector<cudaEvent_t> pool;
    cudaEvent_t get() {
        if (!pool.empty()) { cudaEvent_t e = pool.back(); pool.pop_back(); return e; }
        cudaEvent_t e = nullptr;
        cudaEventCreate(&e);
        return e;
    }
};

// Threads per block of the likelihood-ratio kernel (recon.cu); the plan sizes
// its per-block partial sums with it.
constexpr int NLL_THREADS = 64;

// Table-path data (piecewise-linear structure of W in u); built on first use.
struct TablePath;

// A host-buffer call on the FP32 table path runs the contraction over q in two
// launches over two parts of the voxel rows, so that one part's copy overlaps the
// other part's contraction: forward -- the rows split at `rows` (a quarter of them,
// a whole number of 128-row tiles); the second part of f arrives on copy_stream and
// `in_ready` records its end (the forward waits for it before the second part, or
// before anything when it does not split); adjoint -- the first part is one wave
// of 128-row tiles (one per SM) when there are more; after its contraction the
// adjoint records `out_half`, copies that part of f to out_host on copy_stream
// and sets `out_from` to its rows, so that the caller copies only the rest.  Each
// output row is computed exactly as without the split.
struct HostPipe {
    int64_t rows;
    cudaStream_t cs;
    cudaEvent_t in_ready, out_half;
    float *out_host;
    int64_t out_from;
};

struct caxsi_plan {
    caxsi_geometry g;
    DevGeo dg;
    int device;
    int num_sms;

    // device tables (built by FP64 kernels)
    float4 *vox;        // [R] {x_i, Y_j = y_j/p_y, C*G_so, x_i^2 + y_j^2}
    float *zrow;        // [M] z'_m
    float *god;         // [X][M][ND] G_od * dtheta per scatter vector
    uint32_t *tbits;    // [R][M][Nw] mask factor bits per pair
    float2 *energy;     // [K] {a_k = E_k/(hc dq), c_k = Phi_k E_k dE / hc^2}

    // scratch (plan-owned)
    float *fwd_part;    // [fwd_chunks][M*N] forward partial sums
    int fwd_chunks;
    int fwd_vc;         // voxels per forward chunk
    float *adj_part;    // [adj_split][R*Q] adjoint partials (adj_split > 1)
    int adj_split;
    float *gtmp;        // [M*N]
    float *ratio;       // [M*N]
    float *ones;        // [M*N]
    float *b1[4];       // [R*Q] A^T 1 per path, lazily
    int n_subsets;      // detector subsets of the ordered-subset operators (0 = none)
    std::vector<int32_t> sub_host;  // [M*N] subset of each pixel (host copy of the partition)
    std::vector<int> sub_off;   // [n_subsets + 1] each subset's range in sub_pix (host)
    int *sub_pix;       // [M*N] the pixels grouped by subset, ascending within a subset (device)
    int *sub_of_pix;    // [M*N] subset of each pixel (device)
    int *sub_pos;       // [M*N] position of each pixel in its subset's list (device)
    int sub_gen;        // incremented by every new partition
    float *b1_sub[4];   // [n_subsets][R*Q] A_p^T 1 per path, lazily
    std::vector<unsigned char> b1_sub_ok[4];   // which subsets of b1_sub are computed
    float *vjp_scratch;   // [2][vjp_cap] reverse-mode scratch of the update
    int64_t vjp_cap;
    float *b2;          // [R*Q]
    float *fnew;        // [R*Q]
    double *nll_part;   // [nll_blocks]
    double *nll_dev;    // [1]
    int nll_blocks;
    int *err_flag;      // [3] device words: [0] non-positive mean, [1] copy wait timed out,
                        // [2] completion counter of the likelihood blocks
    float *stage_in, *stage_out;  // host-API staging, lazily
    // Host-buffer calls on the FP32 table path overlap their large copy with the
    // contraction: set only during such a call (see HostPipe).
    struct HostPipe *pipe;
    cudaStream_t copy_stream;     // lazily, with the two events below
    cudaEvent_t pipe_ev[2];

    TablePath *table;

    int64_t table_bytes;
    int64_t launches;   // kernels launched by the current / last call
    int64_t open_pairs; // (voxel, pixel) pairs with mask factor 1
    std::vector<double> phi;  // host copy of the spectrum Phi_k
    int gemm_engine;          // table-path contractions: 0 = tcgen05 kernel, 1 = cuBLAS
    int no_symmetry;          // 1: the table forward streams the ordinary records, not the mirror-symmetric ones
    int u_samples;            // table paths: 0 = the exact knots; N >= 2: N uniform samples of u (approximate)
    int no_bands;             // 1: the tcgen05 contractions multiply the zeros outside the band of S~ too
    int no_sparse_subsets;    // 1: the FP32 subset operators use the whole-object contractions too
    uint8_t *mask01;          // [mask_rows][mask_cols] the mask as 0 / 1 (device)
    int mask_symmetric;       // 1: the mask is mirror-symmetric about the central ray in y and z, J, M, N even
    int online_mask;          // 1: the direct path uses the symmetric-mask kernels (mask factor online)
    uint32_t test_wait_limit; // test hook: polls of the record forward's copy waits (0 = default)
    int test_withhold;        // test hook: the record forward withholds each block's first row copy
    KernelProfiler prof;
};

// ---- plan.cu -----------------------------------------------------------------
caxsi_status plan_build_tables(caxsi_plan *p, const double *phi_host, const uint8_t *mask_host);

// ---- direct.cu ---------------------------------------------------------------
caxsi_status direct_forward(caxsi_plan *p, const float *f, float *g, cudaStream_t s);
caxsi_status direct_adjoint(caxsi_plan *p, const float *w, float *f, cudaStream_t s);
// symmask.cu: the direct operators for a mirror-symmetric mask, mask factor online
caxsi_status symmask_forward(caxsi_plan *p, const float *f, float *g, cudaStream_t s);
caxsi_status symmask_adjoint(caxsi_plan *p, const float *w, float *f, cudaStream_t s);
size_t symmask_fwd_smem(const DevGeo &g);
size_t symmask_adj_smem(const DevGeo &g);
void direct_configure(caxsi_plan *p);
caxsi_status direct_forward_static_scratch(caxsi_plan *p, const float *f, float *g, cudaStream_t s);
// g[list[e]] = sum over the nparts compact partial images part[c * np + e], c ascending
cudaError_t launch_sum_list(const float *part, int nparts, int np, const int *list, float *g, cudaStream_t s);
// subset operators over the pixel lists of caxsi_plan_set_subsets
caxsi_status direct_forward_subset(caxsi_plan *p, const float *f, float *g, int subset, cudaStream_t s);
caxsi_status direct_adjoint_subset(caxsi_plan *p, const float *w, float *f, int subset, cudaStream_t s);

// ---- table.cu ----------------------------------------------------------------
// subset < 0: the full operator; else the rows (pixels) of that detector subset.
caxsi_status table_forward(caxsi_plan *p, const float *f, float *g, int path, int subset, cudaStream_t s);
caxsi_status table_adjoint(caxsi_plan *p, const float *w, float *f, int path, int subset, cudaStream_t s);
// the table paths' records grouped by the plan's current partition (no-op when
// they are up to date; synchronous when it builds them)
caxsi_status table_set_subsets(caxsi_plan *p);
// nb objects = voxel ranges [ranges[2b], ranges[2b+1]) of the shared geometry
caxsi_status table_forward_batch(caxsi_plan *p, int nb, const int32_t *ranges, const float *f, float *g,
                                 int path, cudaStream_t s);
caxsi_status table_adjoint_batch(caxsi_plan *p, int nb, const int32_t *ranges, const float *w, float *f,
                                 int path, cudaStream_t s);

void table_destroy(caxsi_plan *p);
int64_t table_breakpoints(const caxsi_plan *p);
int64_t table_records(const caxsi_plan *p);
int64_t table_sym_records(const caxsi_plan *p);

// ---- recon.cu ----------------------------------------------------------------
// sub != null: only pixels with sub[i] == subset enter (ratio 0 and no
// likelihood term elsewhere).
// ratio = y / (g + r); with nll, the FP64 negative log-likelihood too (in nll_dev)
caxsi_status recon_ratio(caxsi_plan *p, const float *y, const float *r, const int *sub, int subset, bool nll,
                         cudaStream_t s);
caxsi_status recon_update(caxsi_plan *p, const float *f_old, float beta, float delta,
                          const float *b1, cudaStream_t s);
caxsi_status recon_nll_fetch(caxsi_plan *p, double *out, cudaStream_t s);
// n = nobj * R * Q elements (objects back to back)
caxsi_status recon_update_ext(caxsi_plan *p, const float *f, const float *b1, const float *b2, float beta,
                              float delta, float *out, int64_t n, cudaStream_t s);
// ratio = y / (g + r) over n elements of caller buffers, and its reverse mode
caxsi_status recon_ratio_ext(caxsi_plan *p, const float *g, const float *y, const float *r, float *ratio, int64_t n,
                             cudaStream_t s);
caxsi_status recon_ratio_vjp(caxsi_plan *p, const float *g, const float *y, const float *r, const float *gr,
                             float *gg, int64_t n, cudaStream_t s);
caxsi_status recon_update_vjp(caxsi_plan *p, const float *f, const float *b1, const float *b2, float beta,
                              float delta, const float *gx, float *gf, float *gb2, int64_t n, cudaStream_t s);

// ---- helpers -----------------------------------------------------------------
#define CAXSI_CUDA_TRY(expr)                                   \
    do {                                                       \
        cudaError_t _e = (expr);                               \
        if (_e != cudaSuccess) {                               \
            return _e == cudaErrorMemoryAllocation ? CAXSI_ERR_OOM : CAXSI_ERR_CUDA; \
        }                                                      \
    } while (0)

#define CAXSI_LAUNCH_CHECK(p)                                  \
    do {                                                       \
        (p)->launches++;                                       \
        cudaError_t _e = cudaGetLastError();                   \
        if (_e != cudaSuccess) return CAXSI_ERR_CUDA;          \
    } while (0)

// Bracket one kernel launch with profiler events (no-op when profiling is off).
struct ProfScope {
    caxsi_plan *p;
    const char *name;
    cudaStream_t s;
    cudaEvent_t a = nullptr;
    ProfScope(caxsi_plan *p_, const char *n, cudaStream_t s_) : p(p_), name(n), s(s_) {
        if (p->prof.on) { a = p->prof.get(); cudaEventRecord(a, s); }
    }
    ~ProfScope() {
        if (a) {
            cudaEvent_t b = p->prof.get();
            cudaEventRecord(b, s);
            p->prof.recs.push_back({name, a, b});
        }
    }
};
#define CAXSI_PROF(p, name, s) ProfScope _prof_scope_##__LINE__((p), (name), (s))

static inline int64_t ceil_div64(int64_t a, int64_t b) { return (a + b - 1) / b; }
