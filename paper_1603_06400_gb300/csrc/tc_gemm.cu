// Tensor-core GEMM for the table paths' contractions over q (sm_103a, tcgen05).
//
//   C[M][N] = sum_k A[M][K] B[N][K]      (A, B row-major with K contiguous; C FP32)
//
// Forward:  Wtab = F S~^T   (A = f [R][Q], B = S~ [B][Q])
// Adjoint:  f = V S~        (A = V [R][Bp], B = S~^T [Q][Bt])
//
// Variants: KIND 0 = "3xTF32": A and B are each given as a TF32-rounded high
// part and an FP32 remainder (x = hi + lo, both read as TF32 by the tensor
// core); the product is accumulated as hi*hi + hi*lo + lo*hi in FP32, an error
// of about 2^-21 relative per product (FP32-level accuracy).  KIND 3 = the same
// with A given once in FP32: the tile as loaded is its own high part (the tensor
// core reads an FP32 operand as TF32 by dropping the low 13 mantissa bits) and
// four converter warps write the exact remainder x - hi(x) next to it (half the
// A traffic; the products with A_hi start before the remainder is written), and
// B_hi, B_lo side by side so that A_hi [B_hi | B_lo] is one instruction (bn = 128).
// KIND 4 = the on-chip A split with the three products of KIND 0 in KIND 0's
// order (bn = 256, two converter warps; the MMAs of a stage wait for its
// remainder), so that no separate pass splits A and the sums are those of KIND 0.  KIND 1 / 2 = single-pass
// bf16 / fp16 operands with FP32 accumulation.
//
// Structure (one CTA per SM, persistent over 128 x BN output tiles):
//   warp 0      TMA producer: 2-D tensor loads (128-byte swizzle) of the A and B
//               k-slices (128 bytes of K per row) into an NS-stage ring;
//   warp 1      MMA issuer: one thread issues tcgen05.mma (M = 128, N = BN,
//               K = 32 bytes per instruction) into a TMEM accumulator, commits
//               each stage back to the producer and each finished tile to the
//               epilogue; the accumulator is double-buffered in TMEM so the
//               epilogue of one tile overlaps the MMAs of the next;
//   warps 2..9  epilogue: tcgen05.ld of the warp's 32 TMEM lanes (two warps per
//               lane quarter, each taking half of the columns), FP32 stores.
// Long contractions are split into K-chunks of 4 stages: the tensor core
// accumulates one chunk into a TMEM buffer and the epilogue adds the chunk
// into running FP32 sums held in registers ("promotion"), so no chain of
// tensor-core accumulation is longer than one chunk; the accumulation inside
// the tensor core is not IEEE FP32 round-to-nearest and its error grows with
// the chain length.
// Band-limited B: the contractions' B operand (the spectral basis S~) is zero
// outside a band, so a product block that meets only zeros of B is skipped.
// kband (per n-tile): the k-blocks outside [x, y] are neither loaded nor
// multiplied.  nband (per K-chunk): the chunk's MMAs cover only the 32-column
// quarters [x, y] of the tile (N set in the instruction descriptor, the TMEM and
// B operand addresses offset), and the epilogue adds only those quarters; an
// empty chunk (x > y) issues no MMA.  The skipped products are exact zeros, so
// the results are those of the full products.
// Every mbarrier wait is bounded; on timeout the kernel records an error in
// err[0] and every role stops.
#include <cuda.h>
#include <cuda_bf16.h>
#include <cuda_fp16.h>
#include <stdint.h>

#include <algorithm>
#include <vector>

#include "internal.cuh"

namespace {

constexpr int TCG_THREADS = 320;   // producer, MMA, 8 epilogue warps
constexpr int TCG_EPI = 256;       // epilogue threads
constexpr int KCHUNK = 4;  // k-stages (128 bytes of K each) per tensor-core accumulation chain
constexpr int A_PF = 8;    // k-blocks of A prefetched into L2 ahead of its stage loads (long K)
constexpr uint32_t TCG_WAIT_LIMIT = 1u << 22;

__device__ __forceinline__ uint32_t s_addr(const void *p) {
    return (uint32_t)__cvta_generic_to_shared(p);
}
__device__ __forceinline__ void mb_init(uint64_t *bar, uint32_t count) {
    asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(s_addr(bar)), "r"(count) : "memory");
}
__device__ __forceinline__ void mb_expect_tx(uint64_t *bar, uint32_t bytes) {
    asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(s_addr(bar)), "r"(bytes)
                 : "memory");
}
__device__ __forceinline__ void mb_arrive(uint64_t *bar) {
    asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];" ::"r"(s_addr(bar)) : "memory");
}
__device__ __forceinline__ bool mb_try(uint64_t *bar, uint32_t parity) {
    uint32_t ok;
    asm volatile(
        "{\n .reg .pred p;\n mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n selp.u32 %0, 1, 0, p;\n}\n"
        : "=r"(ok)
        : "r"(s_addr(bar)), "r"(parity)
        : "memory");
    return ok != 0;
}
__device__ __forceinline__ bool mb_wait(uint64_t *bar, uint32_t parity, volatile int *abort) {
    for (uint32_t k = 0; k < TCG_WAIT_LIMIT; ++k) {
        if (mb_try(bar, parity)) return true;
        if ((k & 1023u) == 1023u && *abort) return false;
    }
    return false;
}
__device__ __forceinline__ void tma_load_2d(void *dst, const CUtensorMap *map, int x, int y, uint64_t *bar) {
    asm volatile(
        "cp.async.bulk.tensor.2d.shared::cluster.global.tile.mbarrier::complete_tx::bytes [%0], [%1, {%2, %3}], [%4];" ::"r"(
            s_addr(dst)),
        "l"((uint64_t)map), "r"(x), "r"(y), "r"(s_addr(bar))
        : "memory");
}
// L2 prefetch of the tile a tma_load_2d at (x, y) would read (no completion to wait for).
__device__ __forceinline__ void tma_prefetch_2d(const CUtensorMap *map, int x, int y) {
    asm volatile("cp.async.bulk.prefetch.tensor.2d.L2.global.tile [%0, {%1, %2}];" ::"l"((uint64_t)map), "r"(x),
                 "r"(y)
                 : "memory");
}
// Tile store from shared memory (bulk async group); rows / columns outside the
// tensor are not written.
__device__ __forceinline__ void tma_store_2d(const CUtensorMap *map, uint32_t src, int x, int y) {
    asm volatile("cp.async.bulk.tensor.2d.global.shared::cta.bulk_group [%0, {%2, %3}], [%1];" ::"l"(
                     (uint64_t)map),
                 "r"(src), "r"(x), "r"(y)
                 : "memory");
    asm volatile("cp.async.bulk.commit_group;" ::: "memory");
}
// K-major operand, 128-byte swizzle: rows of 128 bytes, 8-row groups 1024 bytes apart.
__device__ __forceinline__ uint64_t sw128_desc(const void *p) {
    const uint32_t a = s_addr(p);
    uint64_t d = (uint64_t)((a >> 4) & 0x3FFFu);
    d |= (uint64_t)1u << 16;            // leading byte offset (unused for swizzled K-major)
    d |= (uint64_t)(1024u >> 4) << 32;  // stride byte offset: next 8-row group
    d |= (uint64_t)1u << 46;            // descriptor version (sm_100 family)
    d |= (uint64_t)2u << 61;            // 128-byte swizzle
    return d;
}
template <int KIND>
__device__ __forceinline__ void mma(uint32_t d_tmem, uint64_t a, uint64_t b, uint32_t idesc, uint32_t acc) {
    if (KIND == 0 || KIND == 3 || KIND == 4) {   // TF32 operands
        asm volatile(
            "{\n .reg .pred p;\n setp.ne.b32 p, %4, 0;\n tcgen05.mma.cta_group::1.kind::tf32 [%0], %1, %2, %3, p;\n}\n" ::"r"(
                d_tmem),
            "l"(a), "l"(b), "r"(idesc), "r"(acc));
    } else {
        asm volatile(
            "{\n .reg .pred p;\n setp.ne.b32 p, %4, 0;\n tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n}\n" ::"r"(
                d_tmem),
            "l"(a), "l"(b), "r"(idesc), "r"(acc));
    }
}
__device__ __forceinline__ void mma_commit(uint64_t *bar) {
    asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(s_addr(bar))
                 : "memory");
}
__device__ __forceinline__ void fence_before() { asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory"); }
__device__ __forceinline__ void fence_after() { asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory"); }

__device__ __forceinline__ void tmem_ld32(uint32_t taddr, float (&r)[32]) {
    uint32_t u[32];
    asm volatile(
        "tcgen05.ld.sync.aligned.32x32b.x32.b32 {%0, %1, %2, %3, %4, %5, %6, %7, %8, %9, %10, %11, %12, %13, "
        "%14, %15, %16, %17, %18, %19, %20, %21, %22, %23, %24, %25, %26, %27, %28, %29, %30, %31}, [%32];"
        : "=r"(u[0]), "=r"(u[1]), "=r"(u[2]), "=r"(u[3]), "=r"(u[4]), "=r"(u[5]), "=r"(u[6]), "=r"(u[7]),
          "=r"(u[8]), "=r"(u[9]), "=r"(u[10]), "=r"(u[11]), "=r"(u[12]), "=r"(u[13]), "=r"(u[14]),
          "=r"(u[15]), "=r"(u[16]), "=r"(u[17]), "=r"(u[18]), "=r"(u[19]), "=r"(u[20]), "=r"(u[21]),
          "=r"(u[22]), "=r"(u[23]), "=r"(u[24]), "=r"(u[25]), "=r"(u[26]), "=r"(u[27]), "=r"(u[28]),
          "=r"(u[29]), "=r"(u[30]), "=r"(u[31])
        : "r"(taddr));
    asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
#pragma unroll
    for (int i = 0; i < 32; ++i) r[i] = __uint_as_float(u[i]);
}

struct TcArgs {
    int M, N, K;
    float *C;
    int64_t ldc;
    int *err;
    int ntn, ntiles, nk;
    const int2 *kband;   // [ntn] k-block range of each n-tile, or null (all)
    const int2 *nband;   // [chunks] column-quarter range of each K-chunk, or null (all)
    int vec_ok;     // rows of C start on 16-byte boundaries (vector stores allowed)
    int tma_store;  // C is written by TMA tensor stores through shared memory
    uint16_t *C16;  // non-null: C is written as bf16 (round to nearest) here instead of FP32 to C
    int b_blocked;  // B (and B2) in k-block order: tile (n-tile j, k-block k) at rows (j nk + k) BN of a [.][KE] map
};

constexpr uint32_t TCG_STG = 4096;   // per epilogue warp: one 32 x 32 FP32 chunk, 128-byte swizzled

template <int BN, int KIND, int NS, int NT>
__global__ void __launch_bounds__(NT, 1)
k_tc_gemm(const __grid_constant__ CUtensorMap tA, const __grid_constant__ CUtensorMap tA2,
          const __grid_constant__ CUtensorMap tB, const __grid_constant__ CUtensorMap tB2,
          const __grid_constant__ CUtensorMap tC, TcArgs a) {
    constexpr bool X3 = KIND == 0 || KIND == 3 || KIND == 4;
    constexpr bool SPLIT_A = KIND == 3 || KIND == 4;   // converter warps 10.. split A in shared memory
    constexpr int NCONV = KIND == 3 ? 128 : 64;        // converter threads (kind 4: within 168 registers)
    constexpr uint32_t A_BYTES = 128 * 128;
    constexpr uint32_t B_BYTES = BN * 128;
    constexpr uint32_t STAGE = X3 ? 2 * (A_BYTES + B_BYTES) : (A_BYTES + B_BYTES);
    constexpr int KE = X3 ? 32 : 64;  // K elements per 128-byte row slice
    // kind 3 keeps B_hi and B_lo side by side in a stage, so that one N = 2 BN
    // instruction forms A_hi [B_hi | B_lo]: its accumulator is 2 BN columns wide
    constexpr bool CAT = KIND == 3;
    constexpr uint32_t ACC_COLS = CAT ? 2 * BN : BN;
    constexpr uint32_t TMEM_COLS = 2 * ACC_COLS;
    constexpr uint32_t B2_OFF = CAT ? A_BYTES + B_BYTES : 2 * A_BYTES + B_BYTES;   // B_lo in a stage
    constexpr uint32_t A2_OFF = CAT ? A_BYTES + 2 * B_BYTES : A_BYTES + B_BYTES;   // A_lo in a stage
    // idesc: D = F32, A/B = TF32 (2) or BF16 (1) or F16 (0), both K-major, N >> 3, M >> 4
    constexpr uint32_t AB = X3 ? 2u : (KIND == 1 ? 1u : 0u);
    constexpr uint32_t IDESC0 = (1u << 4) | (AB << 7) | (AB << 10) | ((uint32_t)(128 >> 4) << 24);
    constexpr int NQ = BN / 32;   // 32-column quarters of a tile

    extern __shared__ unsigned char smem_raw[];
    // operand tiles need 1024-byte alignment of their shared-memory address (swizzle atoms)
    unsigned char *base = smem_raw + ((1024u - (s_addr(smem_raw) & 1023u)) & 1023u);
    unsigned char *stg_base = base + NS * STAGE;   // [8 epilogue warps][TCG_STG]
    uint64_t *full = reinterpret_cast<uint64_t *>(stg_base + 8 * TCG_STG);
    uint64_t *empty = full + NS;
    uint64_t *accf = empty + NS;
    uint64_t *acce = accf + 2;
    uint64_t *conv = acce + 2;   // [NS] A split done (SPLIT_A)
    uint32_t *tmem_slot = reinterpret_cast<uint32_t *>(conv + NS);
    volatile int *abort = reinterpret_cast<volatile int *>(tmem_slot + 1);

    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    if (threadIdx.x == 0) {
        for (int s = 0; s < NS; ++s) {
            mb_init(&full[s], 1);
            mb_init(&empty[s], 1);
            mb_init(&conv[s], NCONV);
        }
        for (int b = 0; b < 2; ++b) {
            mb_init(&accf[b], 1);
            mb_init(&acce[b], TCG_EPI);
        }
        *abort = 0;
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    }
    if (warp == 1) {
        asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(s_addr(tmem_slot)),
                     "r"(TMEM_COLS)
                     : "memory");
        asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
    }
    fence_before();
    __syncthreads();
    fence_after();
    const uint32_t tmem = *tmem_slot;

    if (warp == 0) {
        if (lane == 0) {
            uint32_t it = 0;
            for (int tile = blockIdx.x; tile < a.ntiles && !*abort; tile += gridDim.x) {
                const int m0 = (tile / a.ntn) * 128, n0 = (tile % a.ntn) * BN;
                const int2 kr = a.kband ? a.kband[tile % a.ntn] : make_int2(0, a.nk - 1);
                // a long contraction streams A from DRAM with only NS stages in flight:
                // A's k-blocks A_PF ahead go to L2 first (the next tile's at the end)
                const bool pf = a.nk > 2 * A_PF;
                const int nxt = tile + (int)gridDim.x;
                if (pf && tile == (int)blockIdx.x)   // later tiles were prefetched at the end of the previous one
                    for (int kt = kr.x; kt < kr.x + A_PF && kt <= kr.y; ++kt) tma_prefetch_2d(&tA, kt * KE, m0);
                for (int kt = kr.x; kt <= kr.y; ++kt, ++it) {
                    if (pf) {
                        const int kp = kt + A_PF;
                        if (kp <= kr.y) tma_prefetch_2d(&tA, kp * KE, m0);
                        else if (nxt < a.ntiles && !a.kband) tma_prefetch_2d(&tA, (kp - kr.y - 1) * KE, (nxt / a.ntn) * 128);
                    }
                    const uint32_t s = it % NS, ph = (it / NS) & 1u;
                    if (!mb_wait(&empty[s], ph ^ 1u, abort)) { *abort = 1; break; }
                    unsigned char *st = base + s * STAGE;
                    mb_expect_tx(&full[s], SPLIT_A ? STAGE - A_BYTES : STAGE);
                    const int x = kt * KE;
                    const int xb = a.b_blocked ? 0 : x;
                    const int yb = a.b_blocked ? ((n0 / BN) * a.nk + kt) * BN : n0;
                    tma_load_2d(st, &tA, x, m0, &full[s]);
                    tma_load_2d(st + A_BYTES, &tB, xb, yb, &full[s]);
                    if (X3) {
                        if (!SPLIT_A) tma_load_2d(st + A2_OFF, &tA2, x, m0, &full[s]);
                        tma_load_2d(st + B2_OFF, &tB2, xb, yb, &full[s]);
                    }
                }
            }
        }
    } else if (warp == 1) {
        if (lane == 0) {
            uint32_t it = 0, cc = 0;
            bool ok = true;
            for (int tile = blockIdx.x; tile < a.ntiles && ok && !*abort; tile += gridDim.x) {
                const int2 kr = a.kband ? a.kband[tile % a.ntn] : make_int2(0, a.nk - 1);
                const int nch = (kr.y - kr.x + KCHUNK) / KCHUNK;
                for (int c = 0; c < nch && ok; ++c, ++cc) {
                    const uint32_t b = cc & 1u, aph = (cc >> 1) & 1u;
                    if (!mb_wait(&acce[b], aph ^ 1u, abort)) { *abort = 1; ok = false; break; }
                    fence_after();
                    // the chunk's column quarters [qr.x, qr.y]: N and the TMEM / B offsets
                    // (kind 3: always all of them, the two halves in one instruction)
                    const int2 qr = a.nband && !CAT ? a.nband[c] : make_int2(0, NQ - 1);
                    const uint32_t idesc = IDESC0 | ((uint32_t)(((qr.y - qr.x + 1) * 32) >> 3) << 17);
                    const uint32_t idesc_cat = IDESC0 | ((uint32_t)((2 * BN) >> 3) << 17);
                    const uint32_t d = tmem + b * ACC_COLS + (uint32_t)(qr.x * 32);
                    const uint64_t boff = (uint64_t)(qr.x * 32 * 128 / 16);   // 32 rows of 128 bytes, 16-byte units
                    const int k0 = kr.x + c * KCHUNK, k1 = min(kr.y + 1, k0 + KCHUNK);
                    for (int kt = k0; kt < k1; ++kt, ++it) {
                        const uint32_t s = it % NS, ph = (it / NS) & 1u;
                        if (!mb_wait(&full[s], ph, abort)) { *abort = 1; ok = false; break; }
                        fence_after();
                        unsigned char *st = base + s * STAGE;
                        const uint64_t da = sw128_desc(st), db = sw128_desc(st + A_BYTES) + boff;
                        const uint64_t dal = sw128_desc(st + A2_OFF);
                        const uint64_t dbl = sw128_desc(st + B2_OFF) + boff;
                        if (SPLIT_A && !CAT) {
                            // kind 4: A_lo first, so that the three products go in kind 0's
                            // order (hi hi, hi lo, lo hi per K-step) and give its sums exactly
                            if (!mb_wait(&conv[s], ph, abort)) { *abort = 1; ok = false; break; }
                            fence_after();
                        }
                        if (CAT) {
                            // A_hi x [B_hi | B_lo]: columns [0, BN) get A_hi B_hi, [BN, 2 BN) A_hi B_lo
#pragma unroll
                            for (int ks = 0; ks < 4; ++ks) {
                                const uint64_t adv = (uint64_t)(ks * 2);  // 32 bytes per instruction, 16-byte units
                                const uint32_t acc = (kt > k0 || ks > 0) ? 1u : 0u;
                                mma<KIND>(d, da + adv, db + adv, idesc_cat, acc);
                            }
                        } else if (qr.x <= qr.y) {
#pragma unroll
                            for (int ks = 0; ks < 4; ++ks) {
                                const uint64_t adv = (uint64_t)(ks * 2);  // 32 bytes per instruction, 16-byte units
                                const uint32_t acc = (kt > k0 || ks > 0) ? 1u : 0u;
                                mma<KIND>(d, da + adv, db + adv, idesc, acc);
                                if (X3) {
                                    mma<KIND>(d, da + adv, dbl + adv, idesc, 1u);
                                    mma<KIND>(d, dal + adv, db + adv, idesc, 1u);
                                }
                            }
                        }
                        if (CAT) {
                            // the A_lo x B_hi products once the converters have written A_lo
                            if (!mb_wait(&conv[s], ph, abort)) { *abort = 1; ok = false; break; }
                            fence_after();
                            if (qr.x <= qr.y) {
#pragma unroll
                                for (int ks = 0; ks < 4; ++ks) {
                                    const uint64_t adv = (uint64_t)(ks * 2);
                                    mma<KIND>(d, dal + adv, db + adv, idesc, 1u);
                                }
                            }
                        }
                        mma_commit(&empty[s]);
                    }
                    if (!ok) break;
                    mma_commit(&accf[b]);
                }
            }
        }
    } else if (SPLIT_A && warp >= 10) {
        // converters: for each landed A tile write the remainder A_lo = x - hi(x)
        // into the A_lo slot, hi(x) = x with its low 13 mantissa bits cleared, the
        // TF32 value the tensor core reads from an FP32 operand (so the tile itself
        // serves as A_hi unchanged, and the A_hi products need not wait for this);
        // element-wise, so the 128-byte swizzle of the tile is kept as is
        const int ct = threadIdx.x - 320;
        uint32_t it = 0;
        bool ok = true;
        for (int tile = blockIdx.x; tile < a.ntiles && ok && !*abort; tile += gridDim.x) {
            const int2 kr = a.kband ? a.kband[tile % a.ntn] : make_int2(0, a.nk - 1);
            for (int kt = kr.x; kt <= kr.y; ++kt, ++it) {
                const uint32_t s = it % NS, ph = (it / NS) & 1u;
                if (!mb_wait(&full[s], ph, abort)) { *abort = 1; ok = false; break; }
                unsigned char *st = base + s * STAGE;
                const float4 *hi = reinterpret_cast<const float4 *>(st);
                float4 *lo = reinterpret_cast<float4 *>(st + A2_OFF);
#pragma unroll
                for (int e = ct; e < (int)(A_BYTES / 16); e += NCONV) {
                    const float4 x = hi[e];
                    float4 l;
                    l.x = x.x - __uint_as_float(__float_as_uint(x.x) & 0xffffe000u);
                    l.y = x.y - __uint_as_float(__float_as_uint(x.y) & 0xffffe000u);
                    l.z = x.z - __uint_as_float(__float_as_uint(x.z) & 0xffffe000u);
                    l.w = x.w - __uint_as_float(__float_as_uint(x.w) & 0xffffe000u);
                    lo[e] = l;
                }
                // make the generic-proxy writes visible to the tensor core (async proxy)
                asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
                mb_arrive(&conv[s]);
            }
        }
    } else {
        // epilogue: warps 2..9; warp % 4 selects the TMEM lane quarter, (warp - 2) / 4 the
        // column half of the tile
        constexpr int CW = BN / 2;   // columns per epilogue warp
        const int q = warp & 3, h = (warp - 2) >> 2;
        uint32_t cc = 0;
        bool ok = true;
        for (int tile = blockIdx.x; tile < a.ntiles && ok; tile += gridDim.x) {
            const int2 kr = a.kband ? a.kband[tile % a.ntn] : make_int2(0, a.nk - 1);
            const int nch = (kr.y - kr.x + KCHUNK) / KCHUNK;
            const int m0 = (tile / a.ntn) * 128, n0 = (tile % a.ntn) * BN + h * CW;
            const int row = m0 + q * 32 + lane;
            float *crow = a.C + (int64_t)row * a.ldc;
            float run[CW];
#pragma unroll
            for (int i = 0; i < CW; ++i) run[i] = 0.f;
            for (int c = 0; c < nch; ++c, ++cc) {
                const uint32_t b = cc & 1u, aph = (cc >> 1) & 1u;
                if (!mb_wait(&accf[b], aph, abort)) { *abort = 1; ok = false; break; }
                fence_after();
                const int2 qr = a.nband && !CAT ? a.nband[c] : make_int2(0, NQ - 1);
#pragma unroll
                for (int c0 = 0; c0 < CW; c0 += 32) {
                    const int qq = (h * CW + c0) >> 5;   // warp-uniform
                    if (qq < qr.x || qq > qr.y) continue;   // columns the chunk did not touch: zero
                    float r[32];
                    const uint32_t ta = tmem + ((uint32_t)(q * 32) << 16) + b * ACC_COLS + h * CW + c0;
                    tmem_ld32(ta, r);
#pragma unroll
                    for (int i = 0; i < 32; ++i) run[c0 + i] += r[i];
                    if (CAT) {   // the A_hi B_lo half of the accumulator
                        tmem_ld32(ta + BN, r);
#pragma unroll
                        for (int i = 0; i < 32; ++i) run[c0 + i] += r[i];
                    }
                }
                fence_before();
                mb_arrive(&acce[b]);
            }
            if (!ok) break;
            if (a.C16 && a.tma_store) {
                // bf16 tiles by TMA tensor stores: chunk c0 of 64 columns, lane = row, its
                // 64 columns as 8 words of 8 bf16 at 16-byte slot j ^ (row & 7)
                uint4 *stg = reinterpret_cast<uint4 *>(stg_base + (warp - 2) * TCG_STG);
#pragma unroll
                for (int c0 = 0; c0 < CW; c0 += 64) {
                    const int col = n0 + c0;
                    if (col >= a.N) break;   // warp-uniform
                    if (lane == 0) asm volatile("cp.async.bulk.wait_group.read 0;" ::: "memory");
                    __syncwarp();
#pragma unroll
                    for (int j = 0; j < 8; ++j) {
                        uint32_t wd[4];
#pragma unroll
                        for (int h2 = 0; h2 < 4; ++h2) {
                            const __nv_bfloat162 b2 = __floats2bfloat162_rn(run[c0 + 8 * j + 2 * h2],
                                                                           run[c0 + 8 * j + 2 * h2 + 1]);
                            wd[h2] = *reinterpret_cast<const uint32_t *>(&b2);
                        }
                        stg[lane * 8 + (j ^ (lane & 7))] = make_uint4(wd[0], wd[1], wd[2], wd[3]);
                    }
                    asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
                    __syncwarp();
                    if (lane == 0) tma_store_2d(&tC, s_addr(stg), col, m0 + q * 32);
                }
            } else if (a.C16) {
                // bf16 rows: each lane stores its row's 32 columns as four 16-byte words
                if (row < a.M) {
                    uint16_t *crow16 = a.C16 + (int64_t)row * a.ldc;
#pragma unroll
                    for (int c0 = 0; c0 < CW; c0 += 32) {
                        const int col = n0 + c0;
                        if (col >= a.N) break;
                        if (a.vec_ok && col + 32 <= a.N) {
                            uint4 *dst = reinterpret_cast<uint4 *>(crow16 + col);
#pragma unroll
                            for (int v4 = 0; v4 < 4; ++v4) {
                                uint32_t wd[4];
#pragma unroll
                                for (int h2 = 0; h2 < 4; ++h2) {
                                    const __nv_bfloat162 b2 = __floats2bfloat162_rn(run[c0 + 8 * v4 + 2 * h2],
                                                                                   run[c0 + 8 * v4 + 2 * h2 + 1]);
                                    wd[h2] = *reinterpret_cast<const uint32_t *>(&b2);
                                }
                                dst[v4] = make_uint4(wd[0], wd[1], wd[2], wd[3]);
                            }
                        } else {
#pragma unroll
                            for (int i = 0; i < 32; ++i)
                                if (col + i < a.N) {
                                    const __nv_bfloat16 b = __float2bfloat16_rn(run[c0 + i]);
                                    crow16[col + i] = *reinterpret_cast<const uint16_t *>(&b);
                                }
                        }
                    }
                }
            } else if (a.tma_store) {
                // chunk c0: lane = row, its 32 columns as 8 float4 at 16-byte slot j ^ (row & 7)
                float4 *stg = reinterpret_cast<float4 *>(stg_base + (warp - 2) * TCG_STG);
#pragma unroll
                for (int c0 = 0; c0 < CW; c0 += 32) {
                    const int col = n0 + c0;
                    if (col >= a.N) break;   // warp-uniform
                    if (lane == 0) asm volatile("cp.async.bulk.wait_group.read 0;" ::: "memory");
                    __syncwarp();
#pragma unroll
                    for (int j = 0; j < 8; ++j)
                        stg[lane * 8 + (j ^ (lane & 7))] = make_float4(run[c0 + 4 * j], run[c0 + 4 * j + 1],
                                                                       run[c0 + 4 * j + 2], run[c0 + 4 * j + 3]);
                    asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
                    __syncwarp();
                    if (lane == 0) tma_store_2d(&tC, s_addr(stg), col, m0 + q * 32);
                }
            } else if (row < a.M) {
#pragma unroll
                for (int c0 = 0; c0 < CW; c0 += 32) {
                    const int col = n0 + c0;
                    if (col >= a.N) break;
                    if (a.vec_ok && col + 32 <= a.N) {
                        float4 *dst = reinterpret_cast<float4 *>(crow + col);
#pragma unroll
                        for (int v4 = 0; v4 < 8; ++v4)
                            dst[v4] = make_float4(run[c0 + 4 * v4], run[c0 + 4 * v4 + 1], run[c0 + 4 * v4 + 2],
                                                  run[c0 + 4 * v4 + 3]);
                    } else {
#pragma unroll
                        for (int i = 0; i < 32; ++i)
                            if (col + i < a.N) crow[col + i] = run[c0 + i];
                    }
                }
            }
        }
    }
    // the tile stores must have completed before the block exits
    if (warp >= 2 && lane == 0 && a.tma_store) asm volatile("cp.async.bulk.wait_group 0;" ::: "memory");
    fence_before();
    __syncthreads();
    fence_after();
    if (*abort && threadIdx.x == 0) atomicExch(a.err, 1);
    if (warp == 1) {
        __syncwarp();
        asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(TMEM_COLS) : "memory");
    }
}

// ---- host side ------------------------------------------------------------------

using EncodeFn = CUresult (*)(CUtensorMap *, CUtensorMapDataType, cuuint32_t, void *, const cuuint64_t *,
                              const cuuint64_t *, const cuuint32_t *, const cuuint32_t *, CUtensorMapInterleave,
                              CUtensorMapSwizzle, CUtensorMapL2promotion, CUtensorMapFloatOOBfill);

EncodeFn encode_fn() {
    static EncodeFn fn = nullptr;
    if (!fn) {
        void *p = nullptr;
        cudaDriverEntryPointQueryResult q;
        if (cudaGetDriverEntryPoint("cuTensorMapEncodeTiled", &p, cudaEnableDefault, &q) == cudaSuccess &&
            q == cudaDriverEntryPointSuccess)
            fn = reinterpret_cast<EncodeFn>(p);
    }
    return fn;
}

// 2-D map over a row-major [rows][cols] matrix (cols contiguous, row stride in
// elements), box = 128 bytes of cols x box_rows rows, 128-byte swizzle, zero fill.
bool make_map(CUtensorMap *m, const void *ptr, int elem_bytes, int64_t rows, int64_t cols,
              int64_t row_stride, int box_rows) {
    EncodeFn enc = encode_fn();
    if (!enc) return false;
    const CUtensorMapDataType dt = elem_bytes == 4 ? CU_TENSOR_MAP_DATA_TYPE_FLOAT32 : CU_TENSOR_MAP_DATA_TYPE_UINT16;
    cuuint64_t dims[2] = {(cuuint64_t)cols, (cuuint64_t)rows};
    cuuint64_t strides[1] = {(cuuint64_t)(row_stride * elem_bytes)};
    cuuint32_t box[2] = {(cuuint32_t)(128 / elem_bytes), (cuuint32_t)box_rows};
    cuuint32_t es[2] = {1, 1};
    return enc(m, dt, 2, const_cast<void *>(ptr), dims, strides, box, es, CU_TENSOR_MAP_INTERLEAVE_NONE,
               CU_TENSOR_MAP_SWIZZLE_128B, CU_TENSOR_MAP_L2_PROMOTION_L2_256B,
               CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE) == CUDA_SUCCESS;
}

template <int BN, int KIND, int NS>
cudaError_t launch_tc(const CUtensorMap &tA, const CUtensorMap &tA2, const CUtensorMap &tB,
                      const CUtensorMap &tB2, const CUtensorMap &tC, TcArgs a, int num_sms, cudaStream_t s) {
    constexpr uint32_t STAGE = (KIND == 0 || KIND == 3 || KIND == 4 ? 2 : 1) * (128 * 128 + BN * 128);
    constexpr int NT = KIND == 3 ? TCG_THREADS + 128 : (KIND == 4 ? TCG_THREADS + 64 : TCG_THREADS);
    const size_t smem = 1024 + (size_t)NS * STAGE + 8 * TCG_STG + (3 * NS + 4) * 8 + 16;
    static_assert(1024 + NS * STAGE + 8 * TCG_STG + (3 * NS + 4) * 8 + 16 <= 232448, "shared memory");
    auto kfn = k_tc_gemm<BN, KIND, NS, NT>;
    cudaError_t e = cudaFuncSetAttribute(kfn, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return e;
    const int grid = a.ntiles < num_sms ? a.ntiles : num_sms;
    kfn<<<grid, NT, smem, s>>>(tA, tA2, tB, tB2, tC, a);
    return cudaGetLastError();
}

}  // namespace

// C[M][N] (row stride ldc) = A[M][K] (row stride lda) * B[N][K]^T (row stride ldb).
// kind 0: A = (A_hi, A_lo), B = (B_hi, B_lo) FP32 arrays (3xTF32); kind 3 (bn =
// 128) and kind 4 (bn = 256): A in FP32 (split on chip, A2 ignored), B = (B_hi,
// B_lo); kind 1 / 2: A, B bf16 / fp16 (A2, B2 ignored).  bn = 256 or 128.  Row strides in
// elements must make 16-byte multiples; base pointers 16-byte aligned.  With C16
// non-null the result is written there as bf16 (round to nearest), row stride
// ldc elements, and C is not used.
cudaError_t tc_gemm(int kind, int bn, int M, int N, int K, const void *A, const void *A2, int64_t lda,
                    const void *B, const void *B2, int64_t ldb, float *C, int64_t ldc, int *err,
                    int num_sms, cudaStream_t s, const int2 *kband, const int2 *nband, uint16_t *C16,
                    int b_blocked) {
    const int eb = (kind == 0 || kind == 3 || kind == 4) ? 4 : 2;
    if (kband && nband) return cudaErrorInvalidValue;              // one kind of band at a time
    if (nband && (N + bn - 1) / bn != 1) return cudaErrorInvalidValue;   // quarters of the only n-tile
    const int ke = 128 / eb, nk = (K * eb + 127) / 128;
    // B in k-block order: a [ntn * nk * bn][ke] map whose (bn x ke) boxes are the tiles
    const int64_t brows = b_blocked ? (int64_t)((N + bn - 1) / bn) * nk * bn : N;
    const int64_t bcols = b_blocked ? ke : K, bld = b_blocked ? ke : ldb;
    CUtensorMap tA, tA2, tB, tB2;
    if (!make_map(&tA, A, eb, M, K, lda, 128) || !make_map(&tB, B, eb, brows, bcols, bld, bn))
        return cudaErrorInvalidValue;
    if (kind == 0) {
        if (!make_map(&tA2, A2, eb, M, K, lda, 128) || !make_map(&tB2, B2, eb, brows, bcols, bld, bn))
            return cudaErrorInvalidValue;
    } else if (kind == 3 || kind == 4) {
        tA2 = tA;
        if (!make_map(&tB2, B2, eb, brows, bcols, bld, bn)) return cudaErrorInvalidValue;
    } else {
        tA2 = tA;
        tB2 = tB;
    }
    TcArgs a;
    a.M = M;
    a.N = N;
    a.K = K;
    a.C = C;
    a.ldc = ldc;
    a.err = err;
    a.C16 = C16;
    a.b_blocked = b_blocked;
    CUtensorMap tC;
    if (C16) {
        // bf16 output: TMA tensor stores of 32 rows x 64 columns (128-byte rows), else
        // 16-byte vector stores of 8 columns
        a.vec_ok = ((ldc & 7) == 0) && (((uintptr_t)C16 & 15) == 0);
        a.tma_store = a.vec_ok && make_map(&tC, C16, 2, M, N, ldc, 32) ? 1 : 0;
        if (!a.tma_store) tC = tA;
    } else {
        a.vec_ok = ((ldc & 3) == 0) && (((uintptr_t)C & 15) == 0);
        // C by TMA tensor stores: 32 x 32 boxes with the 128-byte swizzle of the staging buffer
        a.tma_store = a.vec_ok && make_map(&tC, C, 4, M, N, ldc, 32) ? 1 : 0;
        if (!a.tma_store) tC = tA;
    }
    a.ntn = (N + bn - 1) / bn;
    a.ntiles = ((M + 127) / 128) * a.ntn;
    a.nk = (K * eb + 127) / 128;
    a.kband = kband;
    a.nband = nband;
    if (bn == 256) {
        if (kind == 3) return cudaErrorInvalidValue;   // the concatenated-B form is built for bn = 128
        if (kind == 0) return launch_tc<256, 0, 2>(tA, tA2, tB, tB2, tC, a, num_sms, s);
        if (kind == 4) return launch_tc<256, 4, 2>(tA, tA2, tB, tB2, tC, a, num_sms, s);
        if (kind == 1) return launch_tc<256, 1, 4>(tA, tA2, tB, tB2, tC, a, num_sms, s);
        return launch_tc<256, 2, 4>(tA, tA2, tB, tB2, tC, a, num_sms, s);
    }
    if (kind == 0) return launch_tc<128, 0, 3>(tA, tA2, tB, tB2, tC, a, num_sms, s);
    if (kind == 3) return launch_tc<128, 3, 3>(tA, tA2, tB, tB2, tC, a, num_sms, s);
    if (kind == 4) return cudaErrorInvalidValue;   // built for bn = 256
    if (kind == 1) return launch_tc<128, 1, 6>(tA, tA2, tB, tB2, tC, a, num_sms, s);
    return launch_tc<128, 2, 6>(tA, tA2, tB, tB2, tC, a, num_sms, s);
}

std::vector<int2> tc_kband(const std::vector<int2> &row_nz, int N, int bn, int K, int eb) {
    const int ntn = (N + bn - 1) / bn, ke = 128 / eb, nk = (K * eb + 127) / 128;
    std::vector<int2> out(ntn);
    for (int nt = 0; nt < ntn; ++nt) {
        int lo = K, hi = -1;
        for (int i = nt * bn; i < std::min(N, (nt + 1) * bn); ++i)
            if (row_nz[i].x <= row_nz[i].y) {
                lo = std::min(lo, row_nz[i].x);
                hi = std::max(hi, row_nz[i].y);
            }
        out[nt] = hi < 0 ? make_int2(0, 0) : make_int2(lo / ke, std::min(nk - 1, hi / ke));
    }
    return out;
}

std::vector<int2> tc_nband(const std::vector<int2> &col_nz, int N, int bn, int K, int eb) {
    const int ke = 128 / eb, nk = (K * eb + 127) / 128, nch = (nk + KCHUNK - 1) / KCHUNK;
    const int nq = std::min(bn, N + 31 - (N + 31) % 32) / 32;
    std::vector<int2> out(nch);
    for (int c = 0; c < nch; ++c) {
        int lo = N, hi = -1;
        for (int k = c * KCHUNK * ke; k < std::min(K, (c + 1) * KCHUNK * ke); ++k)
            if (col_nz[k].x <= col_nz[k].y) {
                lo = std::min(lo, col_nz[k].x);
                hi = std::max(hi, col_nz[k].y);
            }
        out[c] = hi < 0 ? make_int2(1, 0) : make_int2(lo / 32, std::min(nq - 1, hi / 32));
    }
    return out;
}
