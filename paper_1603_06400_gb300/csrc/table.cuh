// Shared state and device helpers of the table paths (see table.cu).
#pragma once

#include <cublas_v2.h>

#include <vector>

#include "internal.cuh"

// One set of pair records: P groups per voxel (P = 1 for the full operator).
struct RecSet {
    int P = 0;                  // groups per voxel; 0 = not built
    int64_t n = 0;              // records, without the quad padding
    int64_t *off = nullptr;     // [R * P + 1] record range of each (voxel, group), whole quads
    uint32_t *key = nullptr;    // pixel | (t << 16)
    float *w0 = nullptr;        // c (1 - alpha)
    float *w1 = nullptr;        // c alpha
};

// Buffers and layout of the batched operators (objects = voxel ranges of the
// shared geometry; the rows of all objects' voxels are packed).
struct BatchState {
    std::vector<int32_t> ranges;   // the layout the device arrays below describe
    int nb = 0, n_items = 0;
    int64_t rows = 0;
    int4 *items = nullptr;         // [n_items] {obj, v0, v1, packed row of v0}
    int64_t *rowmap = nullptr;     // [rows] source row obj * R + v of each packed row
    int2 *obj_items = nullptr;     // [nb] {first item, items} of each object (chunk order)
    int items_cap = 0, nb_cap = 0;
    int64_t rows_cap = 0, part_cap = 0;
    float *tab = nullptr;          // [rows][Bp] W / V rows
    float *f_hi = nullptr;         // [rows][Qp] packed forward input rows
    float *fpk = nullptr;          // [rows][Q] adjoint output rows
    float *part = nullptr;         // [n_items][M*N] forward partial images
};

// Mirror-symmetric records for the forward model.  The geometry is symmetric
// under the left-right mirror (j, n) -> (J-1-j, N-1-n) and the up-down mirror
// m -> M-1-m (Sec. III-A): mirrored pairs share u, the interval, alpha and c;
// only their mask factors differ.  One record per voxel pair (j, J-1-j) and
// quadrant pixel (m < M/2, n < N/2) holds the two geometry classes of its 8
// pairs -- A: (v, m, n) and its mirrors, B: (v, m, N-1-n) and its mirrors --
// and the 8 mask bits, so that the record owns its 4 pixels for both voxels.
struct SymSet {
    bool ok = false;
    int R2 = 0;                // voxel pairs X * J/2
    int nrec = 0;              // records per voxel pair (M/2)(N/2)
    uint32_t *tt = nullptr;    // [R2 * nrec] interval of class A | class B << 16
    uint8_t *tb = nullptr;     // [R2 * nrec] mask bits (see k_sym_build)
    float4 *w = nullptr;       // [R2 * nrec] {w0 A, w1 A, w0 B, w1 B}
    int chunks = 0, vc = 0;    // forward blocks, voxel pairs per block
    // The adjoint's lists, one per voxel pair s (group 0 of "voxel" s), sorted by
    // t: a record stands for the four pairs (v, m, n), (v, M-1-m, n),
    // (v', m, N-1-n), (v', M-1-m, N-1-n) of one quadrant row m < M/2 and any
    // column n, which share the interval and the weights; key = the four mask
    // bits in the order of the quadrant pixel (m, n0)'s images (m, n0),
    // (M-1-m, n0), (m, N-1-n0), (M-1-m, N-1-n0) | class << 4 (0: n = n0, 1: n =
    // N-1-n0) | quadrant pixel m (N/2) + n0 << 5 | t << 18.  Records whose four
    // pairs are all closed are left out.  adj.P = 0 when the sizes do not fit the
    // key ((M/2)(N/2) > 8192 or B > 16383) or shared memory.
    RecSet adj;
    uint16_t *adj_w0_16 = nullptr, *adj_w1_16 = nullptr;   // adj.w0 / adj.w1 as bf16 (the bf16 path), or null
    // the adjoint's work items: (pair s, knot segment [sg L, (sg + 1) L)), with the
    // quad range of the records that reach the segment (first | end << 16)
    int adj_L = 0, adj_nseg = 0;
    uint32_t *adj_seg = nullptr;   // [R2 * adj_nseg]
};

struct TablePath {
    int B = 0;          // knots
    int Qp = 0;         // q row length of the 16-bit / TF32-split operand copies (multiple of 8)
    int Bp = 0;         // padded row length of Wtab / Vtab (>= B + 1, multiple of 4)
    int NB = 0;         // buckets
    float u0 = 0.f, inv_h = 0.f;
    float2 *knots = nullptr;    // [B] {u_t, 1/(u_{t+1} - u_t)}; last {u_B, 0}
    uint16_t *bstart = nullptr; // [NB] last knot index at or below the bucket start
    float *S = nullptr;         // [B][Q] S~ (FP32)
    float *tab = nullptr;       // [R][Bp] Wtab (forward) / Vtab (adjoint)
    float *fwd_part = nullptr;  // [fwd_chunks][M*N]
    int fwd_chunks = 0, fwd_vc = 0, ppt = 1, threads = 1024, pix_chunks = 1;
    int adj_chunks = 0, adj_vc = 0;
    size_t smem_fwd = 0, smem_adj = 0;
    size_t smem_adj_fx = 0;     // shared memory of the deterministic on-the-fly adjoint (0: does not fit)
    float cmax = 0.f;           // bound of one pair's factor C G_so G_od dtheta (1+cos^2)cos (on-the-fly adjoint)
    unsigned *wmax = nullptr;   // [1] device: max |w| of the current adjoint call (float bits)

    // Pair records (precomputed per-pair interval and weights), voxel-major.
    // rec: every open pair, sorted by (knot interval t, pixel) within each voxel.
    // sub: the same pairs grouped by detector subset within each voxel, then
    //      sorted by (t, pixel): the ordered-subset operators (built on request).
    bool use_records = false;
    RecSet rec, sub;
    SymSet sym;
    int sub_gen = 0;             // the plan partition sub was built for (plan sub_gen)
    BatchState batch;
    int rec_chunks = 0, rec_vc = 0;

    // Contractions over q on tensor cores (cuBLAS): FP32-accurate via the
    // bf16x9 emulation, or single-pass bf16 / fp16 operands with FP32 accumulation.
    cublasHandle_t blas = nullptr;
    void *blas_ws = nullptr;
    size_t blas_ws_bytes = 0;
    void *S16[2] = {nullptr, nullptr};  // S~ as bf16 / fp16, [B][Qp]
    void *f16 = nullptr;                // [R][Qp] 16-bit copy of the forward input
    void *v16 = nullptr;                // [R][Bp] 16-bit adjoint rows

    // Hand-written tcgen05 GEMM operands: TF32 high/low splits (3xTF32) and the
    // transposed spectral matrix S~^T [Q][Bp] for the adjoint contraction.
    float *S_hi = nullptr, *S_lo = nullptr;     // [B][Qp]
    float *St_hi = nullptr, *St_lo = nullptr;   // [Q][Bp]
    void *St16[2] = {nullptr, nullptr};         // [Q][Bp] bf16 / fp16
    float *f_hi = nullptr;                      // [R][Qp] padded copy of the forward input (rows not 16-byte multiples)
    // Band tables of S~ for those GEMMs (device): per n-tile of the forward the
    // q k-blocks to keep, per K-chunk of the adjoint the q quarters to keep;
    // [0] for the TF32 operands, [1] for the 16-bit ones.
    int2 *kband[2] = {nullptr, nullptr};
    int2 *nband[2] = {nullptr, nullptr};
};


struct PairArgs {
    DevGeo g;
    const float4 *vox;
    const float *zrow;
    const float *god;
    const uint32_t *tbits;
};

inline PairArgs pair_args(const caxsi_plan *p) {
    PairArgs a;
    a.g = p->dg;
    a.vox = p->vox;
    a.zrow = p->zrow;
    a.god = p->god;
    a.tbits = p->tbits;
    return a;
}

// Interval t with u_t <= u < u_{t+1} (u inside [u_1, u_B]).
static __device__ __forceinline__ int find_interval(float u, const float2 *kn, const uint16_t *bstart,
                                             int B, int NB, float u0, float inv_h) {
    int bk = (int)((u - u0) * inv_h);
    bk = min(max(bk, 0), NB - 1);
    int t = bstart[bk];
    while (t + 1 < B && kn[t + 1].x <= u) ++t;
    while (t > 0 && kn[t].x > u) --t;
    return t;
}

struct TabArgs {
    int B, NB, Bp;
    float u0, inv_h;
    const float2 *knots;
    const uint16_t *bstart;
};

inline TabArgs tab_args(const TablePath *T) {
    TabArgs a;
    a.B = T->B;
    a.NB = T->NB;
    a.Bp = T->Bp;
    a.u0 = T->u0;
    a.inv_h = T->inv_h;
    a.knots = T->knots;
    a.bstart = T->bstart;
    return a;
}

// records.cu
caxsi_status records_build(caxsi_plan *p, TablePath *T);
caxsi_status records_build_subsets(caxsi_plan *p, TablePath *T, int P, const int32_t *sub_host);
caxsi_status sym_build(caxsi_plan *p, TablePath *T);
// w16: the knot rows are bf16 (in T->v16) instead of FP32 (in T->tab)
cudaError_t sym_forward(const caxsi_plan *p, const TablePath *T, float *part, cudaStream_t s, bool w16 = false);
// out_kind as for records_adjoint
cudaError_t sym_adjoint(const caxsi_plan *p, const TablePath *T, const float *w, int out_kind, cudaStream_t s);
cudaError_t records_forward(const caxsi_plan *p, const TablePath *T, int subset, float *part, cudaStream_t s);
// Sparse subset operators (FP32, per-record contractions against the rows of S~);
// sub_sparse_ok says whether they apply to these arrays and pay at this density
// (average records per voxel and subset up to max_per_voxel); the forward sets
// done = false (and does nothing) when the subset's image does not fit shared
// memory.
bool sub_sparse_ok(const caxsi_plan *p, const void *a, const void *b, int max_per_voxel);
cudaError_t sub_forward_sparse(const caxsi_plan *p, const TablePath *T, int subset, const float *f, float *g,
                               cudaStream_t s, bool &done);
cudaError_t sub_adjoint_sparse(const caxsi_plan *p, const TablePath *T, int subset, const float *w, float *f,
                               cudaStream_t s);
// out_kind: 0 = FP32 rows in tab, 1 = bf16 rows in v16, 2 = fp16 rows in v16
cudaError_t records_adjoint(const caxsi_plan *p, const TablePath *T, int subset, const float *w,
                            int out_kind, cudaStream_t s);

// tc_gemm.cu
// kband / nband (device, or null): B is zero outside bands; see tc_gemm.cu.
cudaError_t tc_gemm(int kind, int bn, int M, int N, int K, const void *A, const void *A2, int64_t lda,
                    const void *B, const void *B2, int64_t ldb, float *C, int64_t ldc, int *err,
                    int num_sms, cudaStream_t s, const int2 *kband = nullptr, const int2 *nband = nullptr,
                    uint16_t *C16 = nullptr, int b_blocked = 0);
// Band tables from the nonzero range of each row of B[N][K] along K (kband: per
// n-tile of bn rows, the k-blocks to keep) or of each column along N (nband: per
// K-chunk, the 32-column quarters to keep); eb = operand element bytes.
std::vector<int2> tc_kband(const std::vector<int2> &row_nz, int N, int bn, int K, int eb);
std::vector<int2> tc_nband(const std::vector<int2> &col_nz, int N, int bn, int K, int eb);

// TF32 split: hi = x rounded to TF32 (nearest), lo = x - hi (exact in FP32)
static __device__ __forceinline__ void tf32_split(float x, float &hi, float &lo) {
    uint32_t h;
    asm("cvt.rna.tf32.f32 %0, %1;" : "=r"(h) : "f"(x));
    hi = __uint_as_float(h);
    lo = x - hi;
}
// The split of an A operand of the 3xTF32 contractions: hi = x with its low 13
// mantissa bits cleared (what the tensor core reads from an FP32 operand, so x
// itself can stand for hi) and the exact remainder.
static __device__ __forceinline__ void tf32_split_trunc(float x, float &hi, float &lo) {
    hi = __uint_as_float(__float_as_uint(x) & 0xffffe000u);
    lo = x - hi;
}
void records_free(TablePath *T);
cudaError_t records_forward_items(const caxsi_plan *p, const TablePath *T, const int4 *items, int n_items,
                                  const float *Wtab, float *part, cudaStream_t s);
cudaError_t records_adjoint_items(const caxsi_plan *p, const TablePath *T, const int4 *items, int n_items,
                                  const float *w, int64_t w_stride, float *Vtab, cudaStream_t s);
