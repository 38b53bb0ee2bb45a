// FP32 SIMT GEMM for the table paths' contractions over q:
//   C[M][N] (+)= sum_k A[M][K] B(k, n)
// A is row-major with K contiguous; B is either "K-major" (B(k, n) = Bm[n*ldb + k])
// or "N-major" (B(k, n) = Bm[k*ldb + n]).  128 x 128 block tile, 8-deep k slices,
// 256 threads with an 8 x 8 register tile each (split in two 4-wide halves so
// that shared-memory reads are conflict-free float4 loads).  blockIdx.z selects
// a k slice of length k_chunk whose result goes to its own output plane
// (C + z * plane) for a later fixed-order reduction.  An optional per-column-tile
// k band [kband.x, kband.y) skips k ranges where B is known to be zero.
#include "internal.cuh"

namespace {

constexpr int BM = 128, BN = 128, BK = 8, THREADS = 256;

template <bool B_KMAJOR>
__global__ void __launch_bounds__(THREADS)
k_sgemm(int M, int N, int K, const float *__restrict__ A, int64_t lda,
        const float *__restrict__ Bm, int64_t ldb, float *__restrict__ C, int64_t ldc,
        int64_t plane, int k_chunk, const int2 *__restrict__ kband) {
    __shared__ __align__(16) float As[BK][BM + 4];
    __shared__ __align__(16) float Bs[BK][BN + 4];
    const int tid = threadIdx.x;
    const int bm = blockIdx.y * BM, bn = blockIdx.x * BN;
    int k0 = blockIdx.z * k_chunk;
    int k1 = min(K, k0 + k_chunk);
    if (kband) {
        const int2 kb = kband[blockIdx.x];
        k0 = max(k0, kb.x);
        k1 = min(k1, kb.y);
    }
    const int ty = tid >> 4, tx = tid & 15;
    float acc[8][8];
#pragma unroll
    for (int a = 0; a < 8; ++a)
#pragma unroll
        for (int b = 0; b < 8; ++b) acc[a][b] = 0.f;

    // loader coordinates: 128 rows x 8 k = 1024 values, 4 per thread
    const int lr = tid >> 1, lk = (tid & 1) * 4;   // A / K-major B: row lr, k lk..lk+3
    const int nk = tid >> 5, nc = (tid & 31) * 4;  // N-major B: k nk, cols nc..nc+3
    for (int kt = k0; kt < k1; kt += BK) {
        float ra[4], rb[4];
#pragma unroll
        for (int q = 0; q < 4; ++q) {
            const int k = kt + lk + q;
            const int r = bm + lr;
            ra[q] = (r < M && k < k1) ? A[(int64_t)r * lda + k] : 0.f;
        }
        if (B_KMAJOR) {
#pragma unroll
            for (int q = 0; q < 4; ++q) {
                const int k = kt + lk + q;
                const int c = bn + lr;
                rb[q] = (c < N && k < k1) ? Bm[(int64_t)c * ldb + k] : 0.f;
            }
        } else {
#pragma unroll
            for (int q = 0; q < 4; ++q) {
                const int k = kt + nk;
                const int c = bn + nc + q;
                rb[q] = (c < N && k < k1) ? Bm[(int64_t)k * ldb + c] : 0.f;
            }
        }
        __syncthreads();
#pragma unroll
        for (int q = 0; q < 4; ++q) As[lk + q][lr] = ra[q];
        if (B_KMAJOR) {
#pragma unroll
            for (int q = 0; q < 4; ++q) Bs[lk + q][lr] = rb[q];
        } else {
            *reinterpret_cast<float4 *>(&Bs[nk][nc]) = make_float4(rb[0], rb[1], rb[2], rb[3]);
        }
        __syncthreads();
#pragma unroll
        for (int kk = 0; kk < BK; ++kk) {
            const float4 a0 = *reinterpret_cast<const float4 *>(&As[kk][ty * 4]);
            const float4 a1 = *reinterpret_cast<const float4 *>(&As[kk][64 + ty * 4]);
            const float4 b0 = *reinterpret_cast<const float4 *>(&Bs[kk][tx * 4]);
            const float4 b1 = *reinterpret_cast<const float4 *>(&Bs[kk][64 + tx * 4]);
            const float av[8] = {a0.x, a0.y, a0.z, a0.w, a1.x, a1.y, a1.z, a1.w};
            const float bv[8] = {b0.x, b0.y, b0.z, b0.w, b1.x, b1.y, b1.z, b1.w};
#pragma unroll
            for (int a = 0; a < 8; ++a)
#pragma unroll
                for (int b = 0; b < 8; ++b) acc[a][b] = fmaf(av[a], bv[b], acc[a][b]);
        }
    }
    float *Cz = C + (int64_t)blockIdx.z * plane;
#pragma unroll
    for (int a = 0; a < 8; ++a) {
        const int r = bm + (a < 4 ? ty * 4 + a : 64 + ty * 4 + (a - 4));
        if (r >= M) continue;
#pragma unroll
        for (int b = 0; b < 8; ++b) {
            const int c = bn + (b < 4 ? tx * 4 + b : 64 + tx * 4 + (b - 4));
            if (c < N) Cz[(int64_t)r * ldc + c] = acc[a][b];
        }
    }
}

}  // namespace

// C = A * B^T-layout (B K-major): used for W[R][B] = F[R][Q] * S~[B][Q]^T.
cudaError_t sgemm_kmajor(int M, int N, int K, const float *A, int64_t lda, const float *Bm,
                         int64_t ldb, float *C, int64_t ldc, const int2 *kband, cudaStream_t s) {
    dim3 grid((N + BN - 1) / BN, (M + BM - 1) / BM, 1);
    k_sgemm<true><<<grid, THREADS, 0, s>>>(M, N, K, A, lda, Bm, ldb, C, ldc, 0, K, kband);
    return cudaGetLastError();
}

// C_z = A[:, kz] * B[kz, :] per k slice z (B N-major): used for F = V * S~ with
// split-k partial planes.
cudaError_t sgemm_nmajor_splitk(int M, int N, int K, const float *A, int64_t lda, const float *Bm,
                                int64_t ldb, float *C, int64_t ldc, int64_t plane, int splits,
                                cudaStream_t s) {
    const int k_chunk = ((K + splits - 1) / splits + BK - 1) / BK * BK;
    dim3 grid((N + BN - 1) / BN, (M + BM - 1) / BM, splits);
    k_sgemm<false><<<grid, THREADS, 0, s>>>(M, N, K, A, lda, Bm, ldb, C, ldc, plane, k_chunk, nullptr);
    return cudaGetLastError();
}
