// Steps (c) and (d): the packed multiply-accumulate on CUDA cores with the
// unpacking, de-companding and the sum over slabs fused into the kernel.
//
// Packing puts several integer products into one FP mantissa, so step (c)
// must run on the FP32 / FP64 FMA pipes (a tensor core would round the
// operands).  Layout: both operands k-major in HBM,
//     A operand  [k][x]  (sym: a_bar^T, x = m;  asym: a_bar^T, x = packed row;
//                         plain: op(A)^T),
//     B operand  [k][n]  (sym: b_bar;  asym / plain: b~ or op(B)),
// so a warp reads each k-row of a tile as consecutive 16-byte vectors.
//
// Per CTA: 256 threads each hold a TM x TN register tile of packed
// accumulators; thread 0 streams (BK x BM) and (BK x BN) boxes into a
// STAGES-deep shared-memory ring with 2-D TMA (cp.async.bulk.tensor, no
// multicast) completing on mbarriers, keeping STAGES - 1 tiles in flight.  (A
// separate producer warp would put three warps on one SM sub-partition and cap
// registers at 168 per thread.)  For every output the packed product of a slab
// is an fma chain in ascending k starting at +0 (eqs. 8 / 12); at the slab's
// end the accumulator is unpacked (eqs. 9-10 or 13-14), scaled by the slab's
// factor (T)(s_A s_B) and added into the running de-companded sum in ascending
// slab order (eqs. 5, 2), then reset.  That order is the oracle's, so results
// are bit-identical to it even beyond the error-free packing region.
//
// Where the running sums live: fp64 kernels keep them in registers.  The fp32
// kernels keep them in tensor memory (TMEM, 256 KB per SM, otherwise unused by
// CUDA-core work): at each slab end a thread reads 16 columns of its TMEM lane
// with tcgen05.ld, adds the unpacked values and writes them back with
// tcgen05.st.  That halves the registers per thread, so two CTAs share an SM.
//
// All waits are bounded (2 s of global time); on expiry the kernel records
// TDG_ETIMEOUT in the plan, waits (bounded) for its outstanding copies, frees
// its TMEM and returns without storing.
#pragma once

#include "tdg_common.cuh"
#include "tdg_internal.h"

namespace tdg {

template <typename T>
struct Vec4;
template <>
struct Vec4<float> {
    __device__ static inline void load(const float *p, float *o) {
        float4 v = *reinterpret_cast<const float4 *>(p);
        o[0] = v.x; o[1] = v.y; o[2] = v.z; o[3] = v.w;
    }
};
template <>
struct Vec4<double> {
    __device__ static inline void load(const double *p, double *o) {
        double2 v0 = *reinterpret_cast<const double2 *>(p);
        double2 v1 = *reinterpret_cast<const double2 *>(p + 2);
        o[0] = v0.x; o[1] = v0.y; o[2] = v1.x; o[3] = v1.y;
    }
};

__device__ inline float fma_rn(float a, float b, float c) { return __fmaf_rn(a, b, c); }

__device__ inline double fma_rn(double a, double b, double c) { return __fma_rn(a, b, c); }
__device__ inline float mul_rn(float a, float b) { return __fmul_rn(a, b); }
__device__ inline double mul_rn(double a, double b) { return __dmul_rn(a, b); }
__device__ inline float sub_rn(float a, float b) { return __fsub_rn(a, b); }
__device__ inline double sub_rn(double a, double b) { return __dsub_rn(a, b); }
__device__ inline float rint_t(float a) { return rintf(a); }
__device__ inline double rint_t(double a) { return rint(a); }

// acc[i][j] = fma(a[i], b[j], acc[i][j]) for a TM x TN register tile.  For
// fp32, adjacent columns go through one packed fma.rn.f32x2 (two IEEE fused
// multiply-adds, each rounded like fma.rn.f32: the same bits as the scalar
// form), which halves the FMA instructions the SM sub-partitions must issue.
template <typename T, int TM, int TN>
__device__ inline void outer_fma(T (&acc)[TM][TN], const T (&a)[TM], const T (&b)[TN]) {
    if constexpr (sizeof(T) == 4 && TN % 2 == 0) {
        uint64_t b2[TN / 2];
#pragma unroll
        for (int jp = 0; jp < TN / 2; ++jp)
            asm("mov.b64 %0, {%1, %2};" : "=l"(b2[jp]) : "f"(b[2 * jp]), "f"(b[2 * jp + 1]));
#pragma unroll
        for (int i = 0; i < TM; ++i) {
            uint64_t a2;
            asm("mov.b64 %0, {%1, %1};" : "=l"(a2) : "f"(a[i]));
#pragma unroll
            for (int jp = 0; jp < TN / 2; ++jp) {
                uint64_t c2;
                asm("mov.b64 %0, {%1, %2};" : "=l"(c2) : "f"(acc[i][2 * jp]), "f"(acc[i][2 * jp + 1]));
                asm("fma.rn.f32x2 %0, %1, %2, %0;" : "+l"(c2) : "l"(a2), "l"(b2[jp]));
                asm("mov.b64 {%0, %1}, %2;" : "=f"(acc[i][2 * jp]), "=f"(acc[i][2 * jp + 1]) : "l"(c2));
            }
        }
    } else {
#pragma unroll
        for (int i = 0; i < TM; ++i)
#pragma unroll
            for (int j = 0; j < TN; ++j) acc[i][j] = fma_rn(a[i], b[j], acc[i][j]);
    }
}
__device__ inline float pow2_t(float, int e) { return scalbnf(1.0f, e); }

// Round to nearest, ties to even, on the FMA/ALU pipes: for |x| < 2^23,
// (x + s) - s with s = copysign(2^23, x) rounds x to an integer (the sum has
// unit spacing and 2^23 is even), and copysign restores the sign of a zero
// result; larger floats are integers already.  Bit-identical to rintf for
// every non-NaN float (checked exhaustively over all 2^32 patterns).  Kept as
// an option: on GB300 the native rint measured faster in the slab epilogue.
#ifndef TDG_EPILOGUE_RINT_ALU
#define TDG_EPILOGUE_RINT_ALU 0   // measured slower than the native rint on GB300
#endif
__device__ inline float rint_epi(float x) {
#if TDG_EPILOGUE_RINT_ALU
    const float s = copysignf(8388608.0f, x);
    const float r = copysignf(__fsub_rn(__fadd_rn(x, s), s), x);
    return fabsf(x) < 8388608.0f ? r : x;
#else
    return rintf(x);
#endif
}
__device__ inline double rint_epi(double x) { return rint(x); }

// Round to nearest, ties to even, for |x| < 2^22 (small_round_ok):
// (x + 1.5 2^23) - 1.5 2^23 on
// the FMA pipe (the sum lies in (2^23, 2^24), where the spacing is 1).  Equal
// to rintf there up to the sign of a zero result, which the digit and the
// running sum it feeds do not carry (they start at +0 and only add).  Measured
// on GB300 in the slab epilogue: the kernel holds fewer values in flight
// (spills 16 bytes instead of 220) and runs about 8 % faster at 4096^3.
__device__ inline float rint_small(float x) {
    return __fsub_rn(__fadd_rn(x, 12582912.0f), 12582912.0f);
}

__device__ inline double pow2_t(double, int e) { return scalbn(1.0, e); }

// ---- tensor-memory helpers (CUDA-core use of TMEM: alloc, 16-column ld/st)
__device__ inline void tmem_alloc(uint32_t *slot, uint32_t ncols) {
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(
                     smem_u32(slot)),
                 "r"(ncols)
                 : "memory");
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
}
__device__ inline void tmem_dealloc(uint32_t base, uint32_t ncols) {
    asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(base), "r"(ncols)
                 : "memory");
}
__device__ inline void tmem_fence_before() {
    asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
}
__device__ inline void tmem_fence_after() {
    asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
}
__device__ inline void tmem_ld16(uint32_t taddr, float *v) {
    uint32_t r[16];
    asm volatile(
        "tcgen05.ld.sync.aligned.32x32b.x16.b32 "
        "{%0, %1, %2, %3, %4, %5, %6, %7, %8, %9, %10, %11, %12, %13, %14, %15}, [%16];"
        : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]),
          "=r"(r[7]), "=r"(r[8]), "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]),
          "=r"(r[13]), "=r"(r[14]), "=r"(r[15])
        : "r"(taddr));
    asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
#pragma unroll
    for (int i = 0; i < 16; ++i) v[i] = __uint_as_float(r[i]);
}
__device__ inline void tmem_st16(uint32_t taddr, const float *v) {
    asm volatile(
        "tcgen05.st.sync.aligned.32x32b.x16.b32 [%0], "
        "{%1, %2, %3, %4, %5, %6, %7, %8, %9, %10, %11, %12, %13, %14, %15, %16};" ::"r"(taddr),
        "r"(__float_as_uint(v[0])), "r"(__float_as_uint(v[1])), "r"(__float_as_uint(v[2])),
        "r"(__float_as_uint(v[3])), "r"(__float_as_uint(v[4])), "r"(__float_as_uint(v[5])),
        "r"(__float_as_uint(v[6])), "r"(__float_as_uint(v[7])), "r"(__float_as_uint(v[8])),
        "r"(__float_as_uint(v[9])), "r"(__float_as_uint(v[10])), "r"(__float_as_uint(v[11])),
        "r"(__float_as_uint(v[12])), "r"(__float_as_uint(v[13])), "r"(__float_as_uint(v[14])),
        "r"(__float_as_uint(v[15]))
        : "memory");
}
__device__ inline void tmem_wait_st() { asm volatile("tcgen05.wait::st.sync.aligned;" ::: "memory"); }

__host__ __device__ constexpr int pow2_at_least(int v) {
    int p = 32;
    while (p < v) p <<= 1;
    return p;
}

template <typename T, int FORM, int W, int BM, int BN, int TM, int TN, int BK, int STAGES>
struct GemmCfg {
    static constexpr int NT = (BM / TM) * (BN / TN);   // threads (16 x 16)
    static constexpr int RG = TM / 4, CG = TN / 4;     // 4-wide fragment groups
    static constexpr int NCACC = FORM == G_ASYM ? W : 1;
    // running de-companded sums in TMEM (fp32 packed forms) or registers
    static constexpr bool TMEMC = FORM != G_PLAIN && sizeof(T) == 4;
    static constexpr int NC = NCACC * TM * TN;         // sums per thread
    static constexpr int TMEM_COLS = pow2_at_least(2 * NC);
    static constexpr int MIN_CTAS = TMEMC ? 2 : 1;
    static constexpr size_t STAGE_A = (size_t)BK * BM * sizeof(T);
    static constexpr size_t STAGE_B = (size_t)BK * BN * sizeof(T);
    static constexpr size_t RING = STAGES * (STAGE_A + STAGE_B) + STAGES * sizeof(uint64_t) + 16;
    // with 256 TMEM columns per CTA at most two CTAs may share an SM's 512:
    // reserve enough shared memory that a third never fits
    static constexpr size_t SMEM = (TMEMC && TMEM_COLS > 128 && RING < 80 * 1024) ? 80 * 1024 : RING;
    static_assert(BM / TM == 16 && BN / TN == 16, "16 x 16 thread grid");
    static_assert(!TMEMC || NC % 16 == 0, "TMEM sums move in 16-column chunks");
    static_assert(!TMEMC || 2 * NC <= 256, "TMEM columns per CTA");
};

// Tile sequence shared by the loads and the math: slab l is split into
// ceil(slab_len / BK) stages of BK k-rows starting at k-row slab_row0(l).
template <typename T, int FORM>
struct SlabWalk {
    const GemmArgs<T> &g;
    __device__ inline int nslab() const { return FORM == G_PLAIN ? 1 : g.nK; }
    __device__ inline int len(int l) const {
        if (FORM == G_SYM) return g.P;
        if (FORM == G_ASYM) return (int)min((long long)g.L, g.K - (long long)l * g.L);
        return (int)g.K;
    }
    __device__ inline long long row0(int l) const {
        if (FORM == G_SYM) return (long long)l * g.P;
        if (FORM == G_ASYM) return (long long)l * g.L;
        return 0;
    }
};

// MIX (symmetric form, Sec. 6 control): each CTA tile reads its inner
// kernel's mask; where it is 0 the tile runs the conventional product (one fma
// chain over all of K from the plain operands, no slab epilogue) instead of
// the packed one.  Tiles never straddle inner kernels (L is a multiple of the
// tile), and the block scheduler balances the two kinds of tile.
template <typename T, int FORM, int W, int BM, int BN, int TM, int TN, int BK, int STAGES,
          bool KEEP, bool MIX, bool SMALL_T = false>
__global__ void __launch_bounds__(GemmCfg<T, FORM, W, BM, BN, TM, TN, BK, STAGES>::NT,
                                  GemmCfg<T, FORM, W, BM, BN, TM, TN, BK, STAGES>::MIN_CTAS)
    packed_gemm_kernel(const __grid_constant__ CUtensorMap mapA,
                       const __grid_constant__ CUtensorMap mapB,
                       const __grid_constant__ CUtensorMap mapPA,
                       const __grid_constant__ CUtensorMap mapPB, const GemmArgs<T> g) {
    pdl_entry();
    using Cfg = GemmCfg<T, FORM, W, BM, BN, TM, TN, BK, STAGES>;
    constexpr int RG = Cfg::RG, CG = Cfg::CG, NCACC = Cfg::NCACC;
    constexpr bool TMEMC = Cfg::TMEMC;
    static_assert(!MIX || (FORM == G_SYM && !KEEP), "mixed tiles: symmetric form only");

    // the device planner chose another packing
    if (g.plan->W != W) return;
    // both rounding variants queued: the one the plan does not select exits
    if constexpr (sizeof(T) == 4 && ((FORM == G_SYM && W == 2) || FORM == G_ASYM) && !KEEP) {
        if (g.small_t < 0 && small_round_ok(FORM, W, g.plan->q, g.plan->gA) != SMALL_T) return;
    }
    // this CTA's tile, row-major over ntn tiles per row; with slab splitting
    // (KEEP instantiation, groups > 1) CTA b takes tile b % ntiles and the
    // slabs of group b / ntiles
    const bool split = KEEP && g.groups > 1;
    long long tix = split ? (long long)blockIdx.x % g.ntiles : (long long)blockIdx.x;
    if constexpr (MIX) {
        if (g.tile_order) tix = g.tile_order[blockIdx.x];
    }
    const long long tmi = tix / g.ntn;
    const long long x0 = tmi * BM;                      // first A-operand column (m or packed row)
    const long long n0 = (tix - tmi * g.ntn) * BN;
    bool plain_tile = false;
    if constexpr (MIX) plain_tile = g.kmask[(x0 / g.L) * g.nN + n0 / g.L] == 0;
    const CUtensorMap *mA = plain_tile ? &mapPA : &mapA;
    const CUtensorMap *mB = plain_tile ? &mapPB : &mapB;

    extern __shared__ __align__(128) unsigned char smem[];
    T *sA = reinterpret_cast<T *>(smem);
    T *sB = reinterpret_cast<T *>(smem + STAGES * Cfg::STAGE_A);
    uint64_t *full = reinterpret_cast<uint64_t *>(smem + STAGES * (Cfg::STAGE_A + Cfg::STAGE_B));
    uint32_t *tmem_slot = reinterpret_cast<uint32_t *>(full + STAGES);
    // the test of the waits' expiry path waits on this barrier, which nothing
    // completes (the second 8 bytes after the ring's barriers)
    uint64_t *never = full + STAGES + 1;

    const int tid = threadIdx.x;
    const int warp = tid >> 5;
    const SlabWalk<T, FORM> walk{g};
    const SlabWalk<T, G_PLAIN> pwalk{g};
    const int nslab_all = plain_tile ? 1 : walk.nslab();
    const int l_begin = split ? (int)((long long)blockIdx.x / g.ntiles) * g.spg : 0;
    const int nslab = split ? min(nslab_all, l_begin + g.spg) : nslab_all;   // end of this CTA's slabs
    auto slab_len = [&](int l) { return plain_tile ? pwalk.len(l) : walk.len(l); };
    auto slab_row0 = [&](int l) { return plain_tile ? 0LL : walk.row0(l); };

    // ---- loads: thread 0 keeps STAGES - 1 tiles in flight ahead of the math
    int pl = l_begin, ps = 0, issued = 0;    // next tile to load: slab pl, stage ps
    auto issue_next = [&]() {
        if (pl >= nslab) return;
        const int stage = issued % STAGES;
        mbar_arrive_expect_tx(&full[stage], (uint32_t)(Cfg::STAGE_A + Cfg::STAGE_B));
        const int y = (int)(slab_row0(pl) + (long long)ps * BK);
        tma_load_2d(sA + (size_t)stage * BK * BM, mA, &full[stage], (int)x0, y);
        tma_load_2d(sB + (size_t)stage * BK * BN, mB, &full[stage], (int)n0, y);
        ++issued;
        if ((++ps) * BK >= slab_len(pl)) { ps = 0; ++pl; }
    };
    if (TMEMC && warp == 0) tmem_alloc(tmem_slot, Cfg::TMEM_COLS);
    if (tid == 0) {
        for (int s = 0; s < STAGES; ++s) mbar_init(&full[s], 1);
        if (g.stall_ns > 0) mbar_init(never, 1);
        fence_barrier_init();
        tma_prefetch_desc(mA);
        tma_prefetch_desc(mB);
        for (int s = 0; s < STAGES; ++s) issue_next();
    }
    if (TMEMC) tmem_fence_before();
    __syncthreads();
    if (TMEMC) tmem_fence_after();
    // this thread's TMEM lane (warps w and w+4 share lanes 32*(w%4) .. +31)
    // and its NC columns
    const uint32_t tcol = TMEMC ? *tmem_slot + ((uint32_t)(32 * (warp & 3)) << 16) +
                                      (uint32_t)((warp >> 2) * Cfg::NC)
                                : 0u;

    const int tx = tid % (BN / TN), ty = tid / (BN / TN);
    T acc[TM][TN];
    T cacc[TMEMC ? 1 : NCACC][TMEMC ? 1 : TM][TMEMC ? 1 : TN];
#pragma unroll
    for (int i = 0; i < TM; ++i)
#pragma unroll
        for (int j = 0; j < TN; ++j) acc[i][j] = T(0);
    if constexpr (!TMEMC) {
#pragma unroll
        for (int d = 0; d < NCACC; ++d)
#pragma unroll
            for (int i = 0; i < TM; ++i)
#pragma unroll
                for (int j = 0; j < TN; ++j) cacc[d][i][j] = T(0);
    }

    T z = T(1), Q = T(1);
    if (FORM != G_PLAIN) {
        z = pow2_t(T(0), -g.plan->q);
        Q = pow2_t(T(0), g.plan->q);
    }

    // row-block index of every fragment row (clamped inside the grid): rows
    // are m (a 4-row group never straddles a block since L % 16 == 0) or, for
    // the asymmetric form, packed rows with P = ceil(L / W) per block, which
    // can straddle when P % 4 != 0 (W = 3)
    int iblk[TM], jblk[CG];
#pragma unroll
    for (int gi = 0; gi < RG; ++gi)
#pragma unroll
        for (int e = 0; e < 4; ++e) {
            long long xr = x0 + gi * (BM / RG) + ty * 4 + e;
            long long ib = FORM == G_ASYM ? xr / g.P : xr / g.L;
            iblk[gi * 4 + e] = (int)min(ib, (long long)g.nM - 1);
        }
#pragma unroll
    for (int hj = 0; hj < CG; ++hj) {
        long long nc = n0 + hj * (BN / CG) + tx * 4;
        jblk[hj] = (int)min(nc / g.L, (long long)g.nN - 1);
    }

    // global coordinates of fragment element (i, j), digit d
    auto out_row = [&](int i, int d) -> long long {
        const long long xr = x0 + (i / 4) * (BM / RG) + ty * 4 + (i % 4);
        if (FORM == G_ASYM) {
            const long long ib = xr / g.P, jr = xr % g.P;
            const long long inblk = jr * W + d;
            if (inblk >= g.L) return -1;
            return ib * g.L + inblk;
        }
        return xr;
    };
    auto out_col = [&](int j) -> long long { return n0 + (j / 4) * (BN / CG) + tx * 4 + (j % 4); };
    auto store_c = [&](long long row, long long col, T v) {
        if (row < 0 || row >= g.M || col >= g.N) return;
        T *p = g.C + row * g.ldc + col;
        *p = g.beta_zero ? mul_rn(g.alpha, v) : fma_rn(g.alpha, v, mul_rn(g.beta, *p));
    };
    // four adjacent columns (col % 4 == 0) as one 16- or 32-byte store where
    // C allows it (beta = 0, aligned rows, all four inside): a warp then writes
    // whole 256-byte row segments, which also keeps C written to host memory
    // over the CPU link in full lines
    auto store_c4 = [&](long long row, long long col, const T *v) {
        const bool c_vec = g.beta_zero && (g.ldc % 4 == 0) &&
                           ((reinterpret_cast<uintptr_t>(g.C) & (4 * sizeof(T) - 1)) == 0);
        if (c_vec && row >= 0 && row < g.M && col + 4 <= g.N) {
            T *p = g.C + row * g.ldc + col;
            if constexpr (sizeof(T) == 4) {
                *reinterpret_cast<float4 *>(p) =
                    make_float4(mul_rn(g.alpha, v[0]), mul_rn(g.alpha, v[1]), mul_rn(g.alpha, v[2]),
                                mul_rn(g.alpha, v[3]));
            } else {
                reinterpret_cast<double2 *>(p)[0] = make_double2(mul_rn(g.alpha, v[0]), mul_rn(g.alpha, v[1]));
                reinterpret_cast<double2 *>(p)[1] = make_double2(mul_rn(g.alpha, v[2]), mul_rn(g.alpha, v[3]));
            }
            return;
        }
#pragma unroll
        for (int q = 0; q < 4; ++q) store_c(row, col + q, v[q]);
    };

    int it = 0;
    bool ok = true;
    for (int l = l_begin; l < nslab && ok; ++l) {
        const int slen = slab_len(l);
        for (int s = 0; s * BK < slen; ++s, ++it) {
            const int stage = it % STAGES;
            const bool got = (g.stall_ns > 0 && it == 0)
                                 ? mbar_wait_ns(never, 0, (uint64_t)g.stall_ns)
                                 : mbar_wait_bounded(&full[stage], (it / STAGES) & 1);
            // every thread is past tile it-1 here, so its stage can be refilled
            if (!__syncthreads_and(got)) {
                if (tid == 0) raise_status(const_cast<DevPlan *>(g.plan), TDG_ETIMEOUT);
                ok = false;
                break;
            }
            if (tid == 0 && it >= 1) issue_next();
            const T *As = sA + (size_t)stage * BK * BM;
            const T *Bs = sB + (size_t)stage * BK * BN;
            const int kcount = min(BK, slen - s * BK);
            if (kcount == BK) {
#pragma unroll
                for (int kk = 0; kk < BK; ++kk) {
                    T a[TM], b[TN];
#pragma unroll
                    for (int gi = 0; gi < RG; ++gi)
                        Vec4<T>::load(As + kk * BM + gi * (BM / RG) + ty * 4, a + 4 * gi);
#pragma unroll
                    for (int hj = 0; hj < CG; ++hj)
                        Vec4<T>::load(Bs + kk * BN + hj * (BN / CG) + tx * 4, b + 4 * hj);
                    outer_fma(acc, a, b);
                }
            } else {
                for (int kk = 0; kk < kcount; ++kk) {
                    T a[TM], b[TN];
#pragma unroll
                    for (int gi = 0; gi < RG; ++gi)
                        Vec4<T>::load(As + kk * BM + gi * (BM / RG) + ty * 4, a + 4 * gi);
#pragma unroll
                    for (int hj = 0; hj < CG; ++hj)
                        Vec4<T>::load(Bs + kk * BN + hj * (BN / CG) + tx * 4, b + 4 * hj);
                    outer_fma(acc, a, b);
                }
            }
        }
        if (!ok) break;
        if (FORM == G_PLAIN || plain_tile) continue;

        // ---- slab end: keep (optionally), unpack, de-compand, accumulate.
        // The unpacked values stream through in the order f = e * NCACC + d
        // (e = i * TN + j the fragment element, d the asymmetric digit).
        const bool first = l == 0;
        // this slab's de-companding factors, all loads issued before any use:
        // one per 4-row group (sym: a group never straddles a block) or per
        // packed row (asym), times one per 4-column group
        constexpr int PR = FORM == G_ASYM ? TM : RG;
        T prs[PR][CG];
        const T *pl_tab = g.pair + (long long)l * g.nM * g.nN;
#pragma unroll
        for (int pi = 0; pi < PR; ++pi)
#pragma unroll
            for (int hj = 0; hj < CG; ++hj)
                prs[pi][hj] = __ldg(pl_tab + (long long)iblk[FORM == G_ASYM ? pi : 4 * pi] * g.nN + jblk[hj]);
        float v[16];
        if constexpr (KEEP) {
            if (split) {
                // slab splitting: only the packed slab results leave the CTA;
                // the ordered sum over slabs runs in the unpack kernel
#pragma unroll
                for (int i = 0; i < TM; ++i) {
                    const long long xr = x0 + (i / 4) * (BM / RG) + ty * 4 + (i % 4);
#pragma unroll
                    for (int j = 0; j < TN; ++j) {
                        const long long nc = out_col(j);
                        if (xr < g.Mrows && nc < g.N)
                            g.Rbar[((long long)l * g.Mrows + xr) * g.N + nc] = acc[i][j];
                        acc[i][j] = T(0);
                    }
                }
                continue;
            }
        }
        if constexpr (FORM == G_SYM && TMEMC && !KEEP && TN % 2 == 0) {
            // eqs. 9-10 and the fma into the running sum on adjacent column
            // pairs (same factor, adjacent TMEM columns): the products and
            // fmas as packed f32x2 operations, each lane rounded as the
            // scalar form
            uint64_t z2, nq2;
            asm("mov.b64 %0, {%1, %1};" : "=l"(z2) : "f"((float)z));
            asm("mov.b64 %0, {%1, %1};" : "=l"(nq2) : "f"(-(float)Q));
#pragma unroll
            for (int e = 0; e < TM * TN; e += 2) {
                const int i = e / TN, j = e % TN, slot = e % 16;
                uint64_t pr2, u2, t2, d2, v2;
                asm("mov.b64 %0, {%1, %1};" : "=l"(pr2) : "f"((float)prs[i / 4][j / 4]));
                const float u0 = rint_epi((float)acc[i][j]), u1 = rint_epi((float)acc[i][j + 1]);
                acc[i][j] = T(0);
                acc[i][j + 1] = T(0);
                asm("mov.b64 %0, {%1, %2};" : "=l"(u2) : "f"(u0), "f"(u1));       // eq. 9
                asm("mul.rn.f32x2 %0, %1, %2;" : "=l"(t2) : "l"(z2), "l"(u2));
                float t0, t1;
                asm("mov.b64 {%0, %1}, %2;" : "=f"(t0), "=f"(t1) : "l"(t2));
                if constexpr (SMALL_T) {
                    t0 = rint_small(t0);
                    t1 = rint_small(t1);
                } else {
                    t0 = rint_epi(t0);
                    t1 = rint_epi(t1);
                }
                asm("mov.b64 %0, {%1, %2};" : "=l"(t2) : "f"(t0), "f"(t1));
                asm("fma.rn.f32x2 %0, %1, %2, %3;" : "=l"(d2) : "l"(nq2), "l"(t2), "l"(u2));  // eq. 10
                if (slot == 0) {
                    if (first) {
#pragma unroll
                        for (int q = 0; q < 16; ++q) v[q] = 0.f;
                    } else {
                        tmem_ld16(tcol + (uint32_t)e, v);
                    }
                }
                asm("mov.b64 %0, {%1, %2};" : "=l"(v2) : "f"(v[slot]), "f"(v[slot + 1]));
                asm("fma.rn.f32x2 %0, %1, %2, %0;" : "+l"(v2) : "l"(d2), "l"(pr2));
                asm("mov.b64 {%0, %1}, %2;" : "=f"(v[slot]), "=f"(v[slot + 1]) : "l"(v2));
                if (slot == 14) tmem_st16(tcol + (uint32_t)(e - 14), v);
            }
            tmem_wait_st();
            continue;
        }
#pragma unroll
        for (int e = 0; e < TM * TN; ++e) {
            const int i = e / TN, j = e % TN;
            const T pr = prs[FORM == G_ASYM ? i : i / 4][j / 4];
            const T r = acc[i][j];
            acc[i][j] = T(0);
            if constexpr (KEEP) {
                const long long xr = x0 + (i / 4) * (BM / RG) + ty * 4 + (i % 4);
                const long long nc = out_col(j);
                if (xr < g.Mrows && nc < g.N) g.Rbar[((long long)l * g.Mrows + xr) * g.N + nc] = r;
            }
            T digit[NCACC];
            if (FORM == G_SYM) {
                const T u = rint_epi(r);                        // eq. 9
                const T t = rint_epi(mul_rn(z, u));
                digit[0] = fma_rn(-Q, t, u);                    // eq. 10
            } else {
                T x = r;
#pragma unroll
                for (int d = 0; d < NCACC; ++d) {               // eqs. 13-14
                    if constexpr (SMALL_T) digit[d] = rint_small(x);
                    else digit[d] = rint_epi(x);
                    if (d + 1 < NCACC) x = mul_rn(Q, sub_rn(x, digit[d]));
                }
            }
#pragma unroll
            for (int d = 0; d < NCACC; ++d) {
                if constexpr (TMEMC) {
                    const int f = e * NCACC + d, slot = f % 16;
                    if (slot == 0) {
                        if (first) {
#pragma unroll
                            for (int q = 0; q < 16; ++q) v[q] = 0.f;
                        } else {
                            tmem_ld16(tcol + (uint32_t)f, v);
                        }
                    }
                    v[slot] = fma_rn((float)digit[d], (float)pr, v[slot]);
                    if (slot == 15) tmem_st16(tcol + (uint32_t)(f - 15), v);
                } else {
                    cacc[d][i][j] = fma_rn(digit[d], pr, cacc[d][i][j]);
                }
            }
        }
        if constexpr (TMEMC) tmem_wait_st();
    }

    if (!ok) {
        // let every copy this CTA issued land before it exits
        if (tid == 0)
            for (int k = it; k < issued; ++k) mbar_wait_bounded(&full[k % STAGES], (k / STAGES) & 1);
    } else if (split) {
        // C is written by the unpack kernel
    } else if (MIX && plain_tile) {
        // ------------------------------------------------------------ store C
        // of a conventional-product tile, straight from the fma chains
#pragma unroll
        for (int i = 0; i < TM; ++i) {
            const long long row = out_row(i, 0);
#pragma unroll
            for (int j = 0; j < TN; j += 4) store_c4(row, out_col(j), &acc[i][j]);
        }
    } else if constexpr (TMEMC) {
        // ------------------------------------------------------------ store C
        // from the running sums in TMEM, 16 columns at a time (kept out of
        // the slab loop so its code stays small)
#pragma unroll
        for (int f0 = 0; f0 < Cfg::NC; f0 += 16) {
            float v[16];
            tmem_ld16(tcol + (uint32_t)f0, v);
            if constexpr (NCACC == 1 && TN % 4 == 0) {
                // 16 consecutive sums = four groups of four adjacent columns
#pragma unroll
                for (int q = 0; q < 16; q += 4) {
                    T w[4];
#pragma unroll
                    for (int r = 0; r < 4; ++r) w[r] = (T)v[q + r];
                    store_c4(out_row((f0 + q) / TN, 0), out_col((f0 + q) % TN), w);
                }
            } else {
#pragma unroll
                for (int q = 0; q < 16; ++q) {
                    const int eq = (f0 + q) / NCACC, dq = (f0 + q) % NCACC;
                    store_c(out_row(eq / TN, dq), out_col(eq % TN), (T)v[q]);
                }
            }
        }
    } else {
        // ------------------------------------------------------------ store C
#pragma unroll
        for (int i = 0; i < TM; ++i)
#pragma unroll
            for (int d = 0; d < NCACC; ++d) {
                const long long row = out_row(i, d);
#pragma unroll
                for (int j = 0; j < TN; j += 4)
                    store_c4(row, out_col(j), FORM == G_PLAIN ? &acc[i][j] : &cacc[d][i][j]);
            }
    }
    if constexpr (TMEMC) {
        tmem_fence_before();
        __syncthreads();
        if (warp == 0) {
            tmem_fence_after();
            tmem_dealloc(*tmem_slot, Cfg::TMEM_COLS);
        }
    }
}

// One launch over the whole tile grid of shape C.
template <typename T, int FORM, int W, typename C, bool KEEP, bool MIX, bool SMALL_T = false>
cudaError_t launch_grid(const GemmArgs<T> &g0, const GemmOperands &ops, cudaStream_t st) {
    using Cfg = GemmCfg<T, FORM, W, C::BM, C::BN, C::TM, C::TN, C::BK, C::STAGES>;
    auto kern = packed_gemm_kernel<T, FORM, W, C::BM, C::BN, C::TM, C::TN, C::BK, C::STAGES, KEEP,
                                   MIX, SMALL_T>;
    static bool attr_set = false;
    if (!attr_set) {
        cudaError_t e =
            cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)Cfg::SMEM);
        if (e != cudaSuccess) return e;
        attr_set = true;
    }
    const CUtensorMapDataType dt =
        sizeof(T) == 8 ? CU_TENSOR_MAP_DATA_TYPE_FLOAT64 : CU_TENSOR_MAP_DATA_TYPE_FLOAT32;
    auto map = [&](CUtensorMap *m, const GemmOperand &o, int box) {
        return encode_map_2d(m, dt, sizeof(T), o.base, o.cols, o.rows, o.ld, box, C::BK,
                             CU_TENSOR_MAP_SWIZZLE_NONE) == CUDA_SUCCESS;
    };
    CUtensorMap ma, mb, mpa, mpb;
    if (!map(&ma, ops.a, C::BM) || !map(&mb, ops.b, C::BN)) return cudaErrorInvalidValue;
    if (MIX) {
        if (!map(&mpa, ops.pa, C::BM) || !map(&mpb, ops.pb, C::BN)) return cudaErrorInvalidValue;
    } else {
        mpa = ma;
        mpb = mb;
    }
    GemmArgs<T> g = g0;
    g.ntn = (int)((g.N + C::BN - 1) / C::BN);
    const long long ntiles = ((g.Mrows + C::BM - 1) / C::BM) * g.ntn;
    g.ntiles = ntiles;
    long long nblocks = ntiles;
    if (KEEP && g.groups > 1) {
        // slab splitting: groups of spg consecutive slabs per CTA
        const int nsl = FORM == G_PLAIN ? 1 : g.nK;
        g.spg = (nsl + g.groups - 1) / g.groups;
        g.groups = (nsl + g.spg - 1) / g.spg;
        nblocks = ntiles * g.groups;
    } else {
        g.groups = 1;
    }
    if (nblocks > 0x7fffffffLL) return cudaErrorInvalidConfiguration;
    return launch_pdl_if(pdl_for_grid(nblocks), kern, dim3((unsigned)nblocks), dim3(Cfg::NT),
                         Cfg::SMEM, st, ma, mb, mpa, mpb, g);
}

// KEEP (store every packed slab result for tdgemm_unpack) and MIX (Sec. 6
// mixed tiles) are separate instantiations so the usual kernel carries none of
// that code.
template <typename T, int FORM, int W, typename C>
cudaError_t launch_cfg(const GemmArgs<T> &g, const GemmOperands &ops, cudaStream_t st) {
    if constexpr (FORM == G_SYM) {
        if (g.kmask) {
            if (g.Rbar || !ops.pa.base || !ops.pb.base) return cudaErrorInvalidValue;
            if constexpr (sizeof(T) == 4 && W == 2) {
                // the packed tiles' unpack rounding as for the unmixed kernel
                if (g.small_t > 0) return launch_grid<T, FORM, W, C, false, true, true>(g, ops, st);
                if (g.small_t < 0) {
                    cudaError_t e = launch_grid<T, FORM, W, C, false, true, true>(g, ops, st);
                    if (e != cudaSuccess) return e;
                }
            }
            return launch_grid<T, FORM, W, C, false, true>(g, ops, st);
        }
    }
    if (g.kmask) return cudaErrorInvalidValue;
    if (FORM != G_PLAIN && g.Rbar) return launch_grid<T, FORM, W, C, true, false>(g, ops, st);
    if (g.groups > 1) return cudaErrorInvalidValue;     // slab splitting stores r-bar
    if constexpr (sizeof(T) == 4 && ((FORM == G_SYM && W == 2) || (FORM == G_ASYM && W >= 2))) {
        // the unpack's roundings as a compile-time variant: known on the host
        // for fixed-bit plans, else both queued and the plan picks one
        if (g.small_t > 0) return launch_grid<T, FORM, W, C, false, false, true>(g, ops, st);
        if (g.small_t < 0) {
            cudaError_t e = launch_grid<T, FORM, W, C, false, false, true>(g, ops, st);
            if (e != cudaSuccess) return e;
        }
    }
    return launch_grid<T, FORM, W, C, false, false>(g, ops, st);
}

}  // namespace tdg
