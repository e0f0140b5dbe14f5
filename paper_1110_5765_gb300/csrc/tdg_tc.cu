// Tensor-core form of step (c): the companded blocks multiplied on the 5th
// generation tensor cores (tcgen05), the per-slab "promotion" of (d) in
// registers.
//
//   TDG_TC_INT  a~, b~ are the integers of eq. 3 (|a~| <= gamma <= 2047) held
//               exactly in fp16; kind::f16 products are exact and every
//               partial sum of one slab stays below 2^24, so the fp32
//               accumulator in tensor memory holds eq. 4's integer exactly.
//   TDG_TC_FP8  a~, b~ are E4M3 codes (kind::f8f6f4), fp32 accumulation.
//
// C = sum_l (s_A,il s_B,lj) * (A~_l B~_l^T), slabs l of L k-values.
//
// Output tiles of 256 x 256 are computed by pairs of SMs with the two-CTA
// form of tcgen05.mma (cta_group::2, M = 256, N = 256): the CTAs of a
// cluster of two each hold 128 rows of A~ and 128 rows (output columns) of
// B~ in shared memory, and the pair's MMA reads both halves of both
// operands, so each shared-memory byte loaded feeds both SMs' tensor cores.
// Per SM and k-step that is a third less shared-memory traffic (TMA writes
// and MMA reads) than a one-CTA 128 x 256 tile.  Each CTA's TMEM holds its
// own 128 rows x 256 columns of the accumulator.  Persistent clusters walk
// their share of the tile pairs, the pipeline running on across tiles.
//   warp 0      allocates 512 TMEM columns (both CTAs, collectively); lane 0
//               streams 256 k-bytes of this CTA's A~ and B~ halves per stage
//               (two 128-byte-wide boxes each, 2-D TMA with 128-byte
//               swizzle) into a 3-deep ring, both CTAs' copies completing on
//               the even CTA's mbarrier.  Eight MMAs per stage: the issuing
//               thread's barrier operations between MMAs cost tensor-pipe
//               time on GB300 (128 cycles per 256 x 256 x 16 MMA back to
//               back, ~175-210 with a wait every four, ~152 every eight);
//   warp 1      (even CTA) lane 0 issues the pair's tcgen05.mma into one of
//               two TMEM accumulators, a fresh accumulation per slab, and
//               commits to mbarriers in both CTAs that free ring stages and
//               hand a full slab to the epilogue;
//   warps 2..17 epilogue: each thread owns one output row and 64 columns;
//               per slab it reads its TMEM lane (tcgen05.ld), applies
//               C_acc = fma(r, s_A s_B, C_acc) in fp32 and releases the
//               accumulator to the even CTA's MMA issuer, so the
//               next-but-one slab's MMAs can reuse it while this one is
//               being promoted.  At a tile's end each warp writes its
//               32 x 64 block of C through a 2 KB staging tile: TMA stores
//               when beta = 0 and C is mappable, else coalesced stores.
// Every wait is bounded (2 s of global time); on expiry the CTA records
// TDG_ETIMEOUT, drains what it issued (bounded) and frees its TMEM.
#include <cuda_fp16.h>

#include <algorithm>

#include "tdg_common.cuh"
#include "tdg_internal.h"

namespace tdg {

namespace {

constexpr int BM = 128, BN = 256;                  // per CTA: rows of A~, columns of C
constexpr int BNH = BN / 2;                          // rows of B~ per CTA
constexpr int STAGES = 3;
constexpr int ROW_BYTES = 128;                       // k-bytes per TMA box (one swizzle row)
constexpr int BOXES = 2;                             // boxes per operand and stage
constexpr int BOX_A = BM * ROW_BYTES;                // 16 KB
constexpr int BOX_B = BNH * ROW_BYTES;               // 16 KB
constexpr int STAGE_A = BOXES * BOX_A;               // 32 KB
constexpr int STAGE_B = BOXES * BOX_B;               // 32 KB
constexpr int MMAS_PER_BOX = 4;                      // 32 k-bytes per MMA
constexpr uint32_t PAIR_TX = 2 * (STAGE_A + STAGE_B);   // bytes one stage brings into the pair
constexpr int EPI_COLS = 64;                         // output columns per epilogue thread
constexpr int EPI_WARPS = 4 * (BN / EPI_COLS);       // 4 TMEM lane quadrants x column groups
constexpr int NUM_THREADS = 32 * (2 + EPI_WARPS);
constexpr int TMEM_COLS = 512;                       // 2 accumulators x 256 fp32 columns
// per epilogue warp: a 32-row x 16-column fp32 staging tile for the C store
constexpr int STG_BYTES = 32 * 16 * 4;
constexpr size_t SMEM_BYTES =
    1024 /*alignment slack*/ + STAGES * (STAGE_A + STAGE_B) + EPI_WARPS * STG_BYTES + 256;

// UMMA shared-memory descriptor, K-major operand with 128-byte swizzle:
// 8-row x 128-byte atoms, 1024 bytes between 8-row groups.
__device__ inline uint64_t desc_sw128(uint32_t saddr) {
    uint64_t d = 0;
    d |= (uint64_t)((saddr & 0x3FFFF) >> 4);      // start address
    d |= (uint64_t)(16 >> 4) << 16;               // leading byte offset (unused here)
    d |= (uint64_t)(1024 >> 4) << 32;             // stride byte offset
    d |= (uint64_t)1 << 46;                       // descriptor version
    d |= (uint64_t)2 << 61;                       // 128-byte swizzle
    return d;
}

// instruction descriptor: D fp32, A/B fp16 (or E4M3 under kind::f8f6f4,
// whose format code is also 0), both K-major, N = 256, M = 256 (the pair)
constexpr uint32_t IDESC = (1u << 4) | (0u << 7) | (0u << 10) | ((uint32_t)(BN >> 3) << 17) |
                           ((uint32_t)((2 * BM) >> 4) << 24);

// the pair's MMA, issued by the even CTA: A rows 0..127 and B~ rows 0..127
// from its shared memory, rows 128..255 of both from the peer's (same offsets)
template <int FP8>
__device__ inline void mma2(uint32_t dtmem, uint64_t ad, uint64_t bd, int accumulate) {
    if constexpr (FP8) {
        asm volatile(
            "{\n\t.reg .pred p;\n\tsetp.ne.b32 p, %4, 0;\n\t"
            "tcgen05.mma.cta_group::2.kind::f8f6f4 [%0], %1, %2, %3, p;\n\t}" ::"r"(dtmem),
            "l"(ad), "l"(bd), "r"(IDESC), "r"(accumulate));
    } else {
        asm volatile(
            "{\n\t.reg .pred p;\n\tsetp.ne.b32 p, %4, 0;\n\t"
            "tcgen05.mma.cta_group::2.kind::f16 [%0], %1, %2, %3, p;\n\t}" ::"r"(dtmem),
            "l"(ad), "l"(bd), "r"(IDESC), "r"(accumulate));
    }
}

// arrive on the mbarrier at bar's offset in both CTAs of the pair once the
// pair's MMAs issued so far have completed
__device__ inline void mma_commit_pair(uint64_t *bar) {
    asm volatile(
        "tcgen05.commit.cta_group::2.mbarrier::arrive::one.shared::cluster.multicast::cluster.b64"
        " [%0], %1;" ::"r"(smem_u32(bar)),
        "h"((uint16_t)0x3)
        : "memory");
}

// 2-D TMA load into this CTA's shared memory, completing bytes on an
// mbarrier that may sit in the peer CTA (bar_cl: shared::cluster address)
__device__ inline void tma_load_2d_pair(void *dst, const CUtensorMap *map, uint32_t bar_cl, int x,
                                        int y) {
    asm volatile(
        "cp.async.bulk.tensor.2d.cta_group::2.shared::cluster.global.mbarrier::complete_tx::bytes"
        " [%0], [%1, {%3, %4}], [%2];" ::"r"(smem_u32(dst)),
        "l"(map), "r"(bar_cl), "r"(x), "r"(y)
        : "memory");
}

// 2-D TMA store of a shared-memory box to global memory (out-of-range rows
// and columns are not written), tracked in this thread's bulk group
__device__ inline void tma_store_2d(const CUtensorMap *map, const void *src, int x, int y) {
    asm volatile(
        "cp.async.bulk.tensor.2d.global.shared::cta.bulk_group [%0, {%2, %3}], [%1];" ::"l"(map),
        "r"(smem_u32(src)), "r"(x), "r"(y)
        : "memory");
    asm volatile("cp.async.bulk.commit_group;" ::: "memory");
}
__device__ inline void tma_store_wait_read() {
    asm volatile("cp.async.bulk.wait_group.read 0;" ::: "memory");
}
__device__ inline void tma_store_wait_all() {
    asm volatile("cp.async.bulk.wait_group 0;" ::: "memory");
}

// shared::cluster address of the variable at p's offset in CTA `rank`
__device__ inline uint32_t cluster_addr(const void *p, uint32_t rank) {
    uint32_t r;
    asm volatile("mapa.shared::cluster.u32 %0, %1, %2;" : "=r"(r) : "r"(smem_u32(p)), "r"(rank));
    return r;
}

// arrive on an mbarrier given by its shared::cluster address (this CTA's or
// the peer's).  The TMEM reads this releases are ordered by the tcgen05
// fences around the arrive and the MMA issuer's wait.
__device__ inline void mbar_arrive_cluster(uint32_t bar_cl) {
    asm volatile("mbarrier.arrive.shared::cluster.b64 _, [%0];" ::"r"(bar_cl) : "memory");
}

__device__ inline uint32_t cluster_rank() {
    uint32_t r;
    asm volatile("mov.u32 %0, %%cluster_ctarank;" : "=r"(r));
    return r;
}

// every thread of both CTAs of the cluster
__device__ inline void cluster_sync() {
    asm volatile("barrier.cluster.arrive.release.aligned;\n\t"
                 "barrier.cluster.wait.acquire.aligned;" ::: "memory");
}

__device__ inline void tc_fence_before() {
    asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
}
__device__ inline void tc_fence_after() {
    asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
}

// 32 lanes x 32 bits, 16 consecutive columns per thread (one load, then
// the wait for it)
__device__ inline void tmem_ld16(uint32_t taddr, float *v) {
    uint32_t r[16];
    asm volatile(
        "tcgen05.ld.sync.aligned.32x32b.x16.b32 "
        "{%0, %1, %2, %3, %4, %5, %6, %7, %8, %9, %10, %11, %12, %13, %14, %15}, [%16];"
        : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]), "=r"(r[7]), "=r"(r[8]), "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]), "=r"(r[13]), "=r"(r[14]), "=r"(r[15])
        : "r"(taddr));
    asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
#pragma unroll
    for (int i = 0; i < 16; ++i) v[i] = __uint_as_float(r[i]);
}

// Waits.  Measured on GB300: the epilogue warps' waits for a finished slab
// suspend between tests (spinning takes issue slots from the producer and
// MMA warps); with E4M3 operands (one ring stage per slab) every wait of the
// kernel suspending from its first test was faster still, with fp16 operands
// slower, so the others spin there.
template <int FP8>
__device__ inline bool tc_wait(uint64_t *bar, uint32_t parity) {
    return FP8 ? mbar_wait_bounded_suspend(bar, parity, true) : mbar_wait_bounded(bar, parity);
}
template <int FP8>
__device__ inline bool tc_wait_epilogue(uint64_t *bar, uint32_t parity) {
    return mbar_wait_bounded_suspend(bar, parity, FP8 != 0);
}

// The plain-store path of the epilogue (beta != 0, or C rows that cannot be
// mapped for TMA): 32 rows x 16 columns of C_acc from the warp's staging tile
// (16-byte unit u of row r at u ^ ((r >> 1) & 3)), each store instruction
// writing 8 rows x 64 contiguous bytes.  Kept out of line: inlined, its
// address arithmetic made the promotion loop spill registers.
__device__ __noinline__ void store_staged_plain(const TcArgs &g, const unsigned char *stg, int lane,
                                                long long rbase, long long cbase, bool vec) {
#pragma unroll
    for (int i = 0; i < 4; ++i) {
        const int r = 8 * i + (lane >> 2), u = lane & 3;
        const float4 a4 = *reinterpret_cast<const float4 *>(stg + r * 64 + ((u ^ ((r >> 1) & 3)) * 16));
        const long long grow = rbase + r;
        const long long col = cbase + 4 * u;
        if (grow >= g.M) continue;
        float *crow = g.C + grow * g.ldc;
        const float acc[4] = {a4.x, a4.y, a4.z, a4.w};
        float o[4];
        if (vec && col + 4 <= g.N) {
            if (g.beta_zero) {
#pragma unroll
                for (int q = 0; q < 4; ++q) o[q] = __fmul_rn(g.alpha, acc[q]);
            } else {
                const float4 in = *reinterpret_cast<const float4 *>(crow + col);
                const float iv[4] = {in.x, in.y, in.z, in.w};
#pragma unroll
                for (int q = 0; q < 4; ++q) o[q] = __fmaf_rn(g.alpha, acc[q], __fmul_rn(g.beta, iv[q]));
            }
            *reinterpret_cast<float4 *>(crow + col) = make_float4(o[0], o[1], o[2], o[3]);
        } else {
#pragma unroll
            for (int q = 0; q < 4; ++q)
                if (col + q < g.N)
                    crow[col + q] = g.beta_zero ? __fmul_rn(g.alpha, acc[q])
                                                : __fmaf_rn(g.alpha, acc[q], __fmul_rn(g.beta, crow[col + q]));
        }
    }
}

template <int FP8>
__global__ void __launch_bounds__(NUM_THREADS, 1)
    tc_gemm_kernel(const __grid_constant__ CUtensorMap mapA,
                   const __grid_constant__ CUtensorMap mapB,
                   const __grid_constant__ CUtensorMap mapC, const TcArgs g) {
    pdl_entry();
    constexpr int KB = FP8 ? 128 : 64;          // k elements per box (four MMAs of 32 bytes)

    extern __shared__ unsigned char smem_raw[];
    // 1024-byte alignment for the swizzled operand tiles
    unsigned char *smem = (unsigned char *)(((uintptr_t)smem_raw + 1023) & ~(uintptr_t)1023);
    unsigned char *sA = smem;
    unsigned char *sB = smem + STAGES * STAGE_A;
    // C staging tiles (1024-byte aligned for the 64-byte swizzle of the C map), then barriers
    unsigned char *stg_base = sB + STAGES * STAGE_B;
    uint64_t *bars = reinterpret_cast<uint64_t *>(stg_base + EPI_WARPS * STG_BYTES);
    uint64_t *full = bars;                       // [STAGES]  TMA -> MMA
    uint64_t *empty = bars + STAGES;             // [STAGES]  MMA -> TMA
    uint64_t *acc_full = bars + 2 * STAGES;      // [2]       MMA -> epilogue
    uint64_t *acc_empty = bars + 2 * STAGES + 2; // [2]       epilogue -> MMA
    uint32_t *tmem_slot = reinterpret_cast<uint32_t *>(bars + 2 * STAGES + 4);
    int *abort_flag = reinterpret_cast<int *>(tmem_slot + 1);

    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    // persistent clusters of two: pair k of cluster c is c + k * (clusters),
    // row-major over 256 x 256 output tile pairs; this CTA holds the upper
    // (rank 0) or lower (rank 1) 128 rows of each and the left or right half
    // of its B~ rows
    const uint32_t rank = cluster_rank();
    const bool leader = rank == 0;
    const int cid = (int)blockIdx.x >> 1, ncl = (int)gridDim.x >> 1;
    const int tiles_n = (int)((g.N + BN - 1) / BN), tiles_m = (int)((g.M + BM - 1) / BM);
    const int npairs = tiles_n * ((tiles_m + 1) / 2);
    const int my_tiles = npairs > cid ? (npairs - 1 - cid) / ncl + 1 : 0;
    // a slab is L / 16 (fp16) or L / 32 (E4M3) MMAs, a multiple of four (one
    // box, since L % 64 == 0 or L % 128 == 0 respectively); a stage is two
    // boxes, so slabs and stages share boundaries in boxes; a tile whose
    // slabs span an odd number of boxes ends on a half-used stage (its
    // second boxes read past the codes, which TMA fills with zeros)
    const int nslab = g.nK;
    const int boxes_slab = g.L / KB;
    const int per_tile = (nslab * boxes_slab + BOXES - 1) / BOXES;   // stages per tile
    const int total = my_tiles * per_tile;
    auto tile_origin = [&](int k, long long &m0, long long &n0) {
        const int t = cid + k * ncl;
        m0 = (long long)(2 * (t / tiles_n) + (int)rank) * BM;   // may pass M: zero rows
        n0 = (long long)(t % tiles_n) * BN;
    };

    // full[] and acc_empty[] are used in the even CTA only (arrivals from both
    // CTAs); empty[] and acc_full[] in both (commits multicast to the pair)
    if (threadIdx.x == 0) {
        for (int s = 0; s < STAGES; ++s) {
            mbar_init(&full[s], 1);          // the even CTA's expect_tx arrival
            mbar_init(&empty[s], 1);         // the pair's MMA commit
        }
        for (int b = 0; b < 2; ++b) {
            mbar_init(&acc_full[b], 1);
            mbar_init(&acc_empty[b], 2 * EPI_WARPS);   // epilogue warps of both CTAs
        }
        *abort_flag = 0;
        fence_barrier_init();
    }
    if (warp == 0) {
        // one warp of each CTA allocates collectively: the same columns in both
        asm volatile("tcgen05.alloc.cta_group::2.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(
                         smem_u32(tmem_slot)),
                     "r"(TMEM_COLS)
                     : "memory");
        asm volatile("tcgen05.relinquish_alloc_permit.cta_group::2.sync.aligned;" ::: "memory");
    }
    tc_fence_before();
    // both CTAs' barriers exist before either copies, commits or arrives into them
    cluster_sync();
    tc_fence_after();
    const uint32_t tmem = *tmem_slot;

    if (warp == 0) {
        // ------------------------------------------------------------ TMA producer
        if (lane == 0) {
            tma_prefetch_desc(&mapA);
            tma_prefetch_desc(&mapB);
            int it = 0;
            for (; it < total; ++it) {
                const int stage = it % STAGES;
                if (it >= STAGES && !tc_wait<FP8>(&empty[stage], ((it / STAGES) + 1) & 1)) {
                    raise_status(const_cast<DevPlan *>(g.plan), TDG_ETIMEOUT);
                    *abort_flag = 1;
                    break;
                }
                if (*(volatile int *)abort_flag) break;
                const int kt = it / per_tile, j = it % per_tile;
                const int kx = j * BOXES * KB;
                long long m0, n0;
                tile_origin(kt, m0, n0);
                // this CTA's 128 rows of A~ and of B~; both CTAs' copies
                // complete on the even CTA's full barrier, which expects them all
                const uint32_t bar = cluster_addr(&full[stage], 0);
                if (leader) mbar_arrive_expect_tx(&full[stage], PAIR_TX);
#pragma unroll
                for (int x = 0; x < BOXES; ++x) {
                    tma_load_2d_pair(sA + stage * STAGE_A + x * BOX_A, &mapA, bar, kx + x * KB, (int)m0);
                    tma_load_2d_pair(sB + stage * STAGE_B + x * BOX_B, &mapB, bar, kx + x * KB,
                                     (int)(n0 + rank * BNH));
                }
            }
            // every copy issued must land before the CTA can exit: the pair's
            // MMA released each of the last stages only after reading them
            for (int k = max(0, it - STAGES); k < it; ++k)
                tc_wait<FP8>(&empty[k % STAGES], (k / STAGES) & 1);
        }
    } else if (warp == 1) {
        // ------------------------------------------------------------ MMA issuer
        if (lane == 0 && leader) {
            int it = 0;              // stages consumed
            int stage = 0, box = 0;  // ring position; next box within the stage
            uint32_t phase = 0;
            uint64_t ad0 = 0, bd0 = 0;
            bool ok = true;
            const int quads = boxes_slab;                 // 4-MMA groups per slab
            for (int kt = 0; kt < my_tiles && ok; ++kt) {
                for (int l = 0; l < nslab; ++l) {
                    const int gs = kt * nslab + l;        // global slab count
                    const int b = gs & 1;
                    if (gs >= 2 && !tc_wait<FP8>(&acc_empty[b], ((gs >> 1) + 1) & 1)) {
                        ok = false;
                        break;
                    }
                    tc_fence_after();
                    const uint32_t d = tmem + (uint32_t)(b * BN);
                    for (int q = 0; q < quads; ++q) {
                        if (box == 0) {
                            if (!tc_wait<FP8>(&full[stage], phase)) {
                                ok = false;
                                break;
                            }
                            tc_fence_after();
                            ad0 = desc_sw128(smem_u32(sA + stage * STAGE_A));
                            bd0 = desc_sw128(smem_u32(sB + stage * STAGE_B));
                        }
                        const uint64_t ad = ad0 + (uint64_t)((box * BOX_A) >> 4);
                        const uint64_t bd = bd0 + (uint64_t)((box * BOX_B) >> 4);
#pragma unroll
                        for (int kk = 0; kk < MMAS_PER_BOX; ++kk) {
                            const uint64_t adv = (uint64_t)((kk * 32) >> 4);
                            mma2<FP8>(d, ad + adv, bd + adv, (q | kk) != 0);
                        }
                        if (++box == BOXES) {
                            mma_commit_pair(&empty[stage]);     // frees the stage in both CTAs
                            box = 0;
                            ++it;
                            if (++stage == STAGES) { stage = 0; phase ^= 1; }
                        }
                    }
                    if (!ok) break;
                    mma_commit_pair(&acc_full[b]);          // the slab is complete in both TMEMs
                }
                if (ok && box != 0) {
                    // the tile ended inside a stage: release its unused half too
                    mma_commit_pair(&empty[stage]);
                    box = 0;
                    ++it;
                    if (++stage == STAGES) { stage = 0; phase ^= 1; }
                }
            }
            if (!ok) {
                raise_status(const_cast<DevPlan *>(g.plan), TDG_ETIMEOUT);
                *abort_flag = 1;
            }
            // the last use of every stage released: the pair's MMAs are done
            // (TMEM can be freed in both CTAs)
            for (int k = max(0, it - STAGES); k < it; ++k)
                tc_wait<FP8>(&empty[k % STAGES], (k / STAGES) & 1);
        }
    } else {
        // ------------------------------------------------------------ epilogue
        const int ew = warp - 2;
        const int quad = warp & 3;                     // TMEM lanes 32*quad .. +31
        const int cgrp = ew >> 2;                      // columns [EPI_COLS*cgrp, +EPI_COLS)
        const long long lstride = (long long)g.nM * g.nN;
        const uint32_t acc_empty_cl[2] = {cluster_addr(&acc_empty[0], 0),
                                          cluster_addr(&acc_empty[1], 0)};
        bool ok = true;
        // the thread's EPI_COLS columns lie in one column block (L % 64 == 0,
        // column groups 64-aligned), so one factor per slab, fetched a slab
        // ahead -- across tiles too: the next tile's first factor is fetched
        // during this tile's last slab, so the tile change costs the MMA
        // issuer as little as possible
        auto factor_row = [&](int k) -> const float * {
            long long m0, n0;
            tile_origin(k, m0, n0);
            const long long row = m0 + quad * 32 + lane;
            const long long col0 = n0 + cgrp * EPI_COLS;
            const int iblk = (int)min((long long)((unsigned long long)row / (unsigned)g.L),
                                      (long long)g.nM - 1);
            const int jblk = (int)min((long long)((unsigned long long)col0 / (unsigned)g.L),
                                      (long long)g.nN - 1);
            return g.pair + (long long)iblk * g.nN + jblk;
        };
        const float *prow = my_tiles > 0 ? factor_row(0) : g.pair;
        float pr_next = my_tiles > 0 ? __ldg(prow) : 0.f;
        for (int kt = 0; kt < my_tiles && ok; ++kt) {
            const float *prow_n = prow;
            float cacc[EPI_COLS];
#pragma unroll
            for (int c = 0; c < EPI_COLS; ++c) cacc[c] = 0.f;
            for (int l = 0; l < nslab; ++l) {
                const int gs = kt * nslab + l;
                const int b = gs & 1;
                const float pr = pr_next;
                if (l + 1 < nslab) {
                    pr_next = __ldg(prow + (long long)(l + 1) * lstride);
                } else if (kt + 1 < my_tiles) {
                    prow_n = factor_row(kt + 1);
                    pr_next = __ldg(prow_n);
                }
                if (!tc_wait_epilogue<FP8>(&acc_full[b], (gs >> 1) & 1)) { ok = false; break; }
                tc_fence_after();
                const uint32_t base =
                    tmem + ((uint32_t)(quad * 32) << 16) + (uint32_t)(b * BN + cgrp * EPI_COLS);
#pragma unroll
                for (int ch = 0; ch < EPI_COLS / 16; ++ch) {
                    float v[16];
                    tmem_ld16(base + ch * 16, v);
                    if (ch == EPI_COLS / 16 - 1) {
                        // the accumulator is read: hand it back before the last fmas
                        tc_fence_before();
                        __syncwarp();
                        if (lane == 0) mbar_arrive_cluster(acc_empty_cl[b]);
                    }
                    // C_acc = fma(r, s_A s_B, C_acc) on column pairs: each lane
                    // of fma.rn.f32x2 rounds once, as fmaf does
                    uint64_t pr2;
                    asm("mov.b64 %0, {%1, %1};" : "=l"(pr2) : "f"(pr));
#pragma unroll
                    for (int e = 0; e < 16; e += 2) {
                        uint64_t v2, c2;
                        asm("mov.b64 %0, {%1, %2};" : "=l"(v2) : "f"(v[e]), "f"(v[e + 1]));
                        asm("mov.b64 %0, {%1, %2};" : "=l"(c2) : "f"(cacc[ch * 16 + e]), "f"(cacc[ch * 16 + e + 1]));
                        asm("fma.rn.f32x2 %0, %1, %2, %0;" : "+l"(c2) : "l"(v2), "l"(pr2));
                        asm("mov.b64 {%0, %1}, %2;" : "=f"(cacc[ch * 16 + e]), "=f"(cacc[ch * 16 + e + 1]) : "l"(c2));
                    }
                }
            }
            if (!ok) break;
            // C out through this warp's staging tile, 16 columns at a time: the
            // thread of row r writes its 16 values as row r (16-byte units
            // XOR-swizzled by row, conflict-free), then each store instruction
            // of the warp writes 8 rows x 64 contiguous bytes (a thread per
            // 16 bytes) instead of 32 rows x 16 bytes
            unsigned char *stg = stg_base + ew * STG_BYTES;
            const bool vec = ((g.ldc & 3) == 0) && (((uintptr_t)g.C & 15) == 0);
            long long m0, n0;
            tile_origin(kt, m0, n0);
            const long long rbase = m0 + quad * 32;
            const long long col0 = n0 + cgrp * EPI_COLS;
            prow = prow_n;
            if (g.c_tma) {
                // beta = 0: alpha C_acc staged in the C map's 64-byte swizzle
                // (16-byte unit u of row r at u ^ ((r >> 1) & 3)), written by
                // one TMA store per 32 x 16 box, which clips rows and columns
                // outside C
#pragma unroll
                for (int ch = 0; ch < EPI_COLS / 16; ++ch) {
                    if (ch > 0 && lane == 0) tma_store_wait_read();   // the box before is read
                    __syncwarp();
#pragma unroll
                    for (int u = 0; u < 4; ++u) {
                        const int us = u ^ ((lane >> 1) & 3);
                        const float *cu = cacc + ch * 16 + 4 * u;
                        *reinterpret_cast<float4 *>(stg + lane * 64 + us * 16) =
                            make_float4(__fmul_rn(g.alpha, cu[0]), __fmul_rn(g.alpha, cu[1]),
                                        __fmul_rn(g.alpha, cu[2]), __fmul_rn(g.alpha, cu[3]));
                    }
                    fence_proxy_async();
                    __syncwarp();
                    if (lane == 0) tma_store_2d(&mapC, stg, (int)(col0 + ch * 16), (int)rbase);
                }
                if (lane == 0) tma_store_wait_read();
                __syncwarp();
                continue;
            }
#pragma unroll
            for (int ch = 0; ch < EPI_COLS / 16; ++ch) {
#pragma unroll
                for (int u = 0; u < 4; ++u) {
                    const int us = u ^ ((lane >> 1) & 3);
                    *reinterpret_cast<float4 *>(stg + lane * 64 + us * 16) =
                        make_float4(cacc[ch * 16 + 4 * u], cacc[ch * 16 + 4 * u + 1],
                                    cacc[ch * 16 + 4 * u + 2], cacc[ch * 16 + 4 * u + 3]);
                }
                __syncwarp();
                store_staged_plain(g, stg, lane, rbase, col0 + ch * 16, vec);
                __syncwarp();
            }
        }
        if (lane == 0) tma_store_wait_all();
        if (!ok) {
            raise_status(const_cast<DevPlan *>(g.plan), TDG_ETIMEOUT);
            *abort_flag = 1;
        }
    }

    tc_fence_before();
    // neither CTA leaves while the other may still write into it
    cluster_sync();
    if (warp == 0) {
        tc_fence_after();
        asm volatile("tcgen05.dealloc.cta_group::2.sync.aligned.b32 %0, %1;" ::"r"(tmem),
                     "r"(TMEM_COLS)
                     : "memory");
    }
}

}  // namespace

template <int FP8>
static cudaError_t launch_tc(const TcArgs &a, const CUtensorMap &mapA, const CUtensorMap &mapB,
                             const CUtensorMap &mapC, cudaStream_t st) {
    auto kern = tc_gemm_kernel<FP8>;
    static int max_clusters = 0;
    cudaLaunchConfig_t cfg = {};
    cudaLaunchAttribute attr[2];
    attr[0].id = cudaLaunchAttributeClusterDimension;
    attr[0].val.clusterDim.x = 2;
    attr[0].val.clusterDim.y = 1;
    attr[0].val.clusterDim.z = 1;
    attr[1].id = cudaLaunchAttributeProgrammaticStreamSerialization;
    attr[1].val.programmaticStreamSerializationAllowed = 1;
    cfg.blockDim = dim3(NUM_THREADS);
    cfg.dynamicSmemBytes = SMEM_BYTES;
    cfg.stream = st;
    cfg.attrs = attr;
    cfg.numAttrs = 1;                    // the occupancy query: cluster shape only
    if (!max_clusters) {
        cudaError_t e =
            cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)SMEM_BYTES);
        if (e != cudaSuccess) return e;
        int dev = 0, sms = 0;
        cudaGetDevice(&dev);
        cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
        cfg.gridDim = dim3((unsigned)max(2, sms & ~1));
        int n = 0;
        e = cudaOccupancyMaxActiveClusters(&n, (void *)kern, &cfg);
        if (e != cudaSuccess) return e;
        max_clusters = max(1, n);
    }
    const long long pairs = ((a.N + BN - 1) / BN) * (((a.M + BM - 1) / BM + 1) / 2);
    cfg.gridDim = dim3((unsigned)(2 * std::min<long long>(pairs, max_clusters)));
    // the launch: cluster shape, and programmatic serialisation unless the grid
    // leaves SMs idle
    cfg.numAttrs = pdl_for_grid(cfg.gridDim.x) ? 2 : 1;
    return cudaLaunchKernelEx(&cfg, kern, mapA, mapB, mapC, a);
}

cudaError_t launch_tc_gemm(int fp8, const TcArgs &a, const CUtensorMap &mapA,
                           const CUtensorMap &mapB, const CUtensorMap &mapC, cudaStream_t st) {
    return fp8 ? launch_tc<1>(a, mapA, mapB, mapC, st) : launch_tc<0>(a, mapA, mapB, mapC, st);
}

void tc_gemm_c_box(int *box_cols, int *box_rows) {
    *box_cols = 16;            // one epilogue warp's staging tile
    *box_rows = 32;
}

void tc_gemm_boxes(int fp8, int *box_rows_a, int *box_rows_b, int *box_k) {
    *box_rows_a = BM;
    *box_rows_b = BNH;         // each CTA of a pair loads half of the B~ tile
    *box_k = fp8 ? 128 : 64;   // two boxes per operand and stage
}

}  // namespace tdg
