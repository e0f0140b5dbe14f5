// Steps (c) and (d): the packed multiply-accumulate on CUDA cores with the
// unpacking, de-companding and the sum over slabs fused into registers.
//
// Packing puts several integer products into one FP mantissa, so step (c)
// must run on the FP32 / FP64 FMA pipes (a tensor core would round the
// operands).  Layout: both operands k-major in HBM,
//     A operand  [k][x]  (sym: a_bar^T, x = m;  asym: a_bar^T, x = packed row;
//                         plain: op(A)^T),
//     B operand  [k][n]  (sym: b_bar;  asym / plain: b~ or op(B)),
// so a warp reads each k-row of a tile as consecutive 16-byte vectors.
//
// Per CTA: 256 threads each hold a TM x TN register tile; thread 0 streams
// (BK x BM) and (BK x BN) boxes into a STAGES-deep shared-memory ring with 2-D
// TMA (cp.async.bulk.tensor, no multicast) completing on mbarriers, keeping
// STAGES - 1 tiles in flight.  (A separate producer warp would put three
// warps on one SM sub-partition and cap registers at 168 per thread; the
// unpacked accumulators need more.)  For every output the packed product of a slab is an fma
// chain in ascending k starting at +0 (eqs. 8 / 12); at the slab's end the
// accumulator is unpacked (eqs. 9-10 or 13-14), scaled by the slab's factor
// (T)(s_A s_B) and added into a second register tile in ascending slab order
// (eqs. 5, 2), then reset.  That order is the oracle's, so results are
// bit-identical to it even beyond the error-free packing region.
// All waits are bounded (2 s of global time); on expiry the kernel records
// TDG_ETIMEOUT in the plan, waits (bounded) for its outstanding copies and
// returns without storing.
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
__device__ inline float pow2_t(float, int e) { return scalbnf(1.0f, e); }
__device__ inline double pow2_t(double, int e) { return scalbn(1.0, e); }

template <typename T, int FORM, int W, int BM, int BN, int TM, int TN, int BK, int STAGES>
struct GemmCfg {
    static constexpr int NT = (BM / TM) * (BN / TN);   // threads (16 x 16)
    static constexpr int RG = TM / 4, CG = TN / 4;     // 4-wide fragment groups
    static constexpr int NCACC = FORM == G_ASYM ? W : 1;
    static constexpr size_t STAGE_A = (size_t)BK * BM * sizeof(T);
    static constexpr size_t STAGE_B = (size_t)BK * BN * sizeof(T);
    static constexpr size_t SMEM = STAGES * (STAGE_A + STAGE_B) + STAGES * sizeof(uint64_t);
    static_assert(BM / TM == 16 && BN / TN == 16, "16 x 16 thread grid");
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

template <typename T, int FORM, int W, int BM, int BN, int TM, int TN, int BK, int STAGES>
__global__ void __launch_bounds__(GemmCfg<T, FORM, W, BM, BN, TM, TN, BK, STAGES>::NT, 1)
    packed_gemm_kernel(const __grid_constant__ CUtensorMap mapA,
                       const __grid_constant__ CUtensorMap mapB, const GemmArgs<T> g) {
    using Cfg = GemmCfg<T, FORM, W, BM, BN, TM, TN, BK, STAGES>;
    constexpr int RG = Cfg::RG, CG = Cfg::CG;

    if (g.plan->W != W) return;   // the device planner chose another packing

    extern __shared__ __align__(128) unsigned char smem[];
    T *sA = reinterpret_cast<T *>(smem);
    T *sB = reinterpret_cast<T *>(smem + STAGES * Cfg::STAGE_A);
    uint64_t *full = reinterpret_cast<uint64_t *>(smem + STAGES * (Cfg::STAGE_A + Cfg::STAGE_B));

    const int tid = threadIdx.x;
    const long long x0 = (long long)blockIdx.y * BM;   // first A-operand column (m or packed row)
    const long long n0 = (long long)blockIdx.x * BN;
    const SlabWalk<T, FORM> walk{g};
    const int nslab = walk.nslab();

    // ---- loads: thread 0 keeps STAGES - 1 tiles in flight ahead of the math
    int pl = 0, ps = 0, issued = 0;    // next tile to load: slab pl, stage ps
    auto issue_next = [&]() {
        if (pl >= nslab) return;
        const int stage = issued % STAGES;
        mbar_arrive_expect_tx(&full[stage], (uint32_t)(Cfg::STAGE_A + Cfg::STAGE_B));
        const int y = (int)(walk.row0(pl) + (long long)ps * BK);
        tma_load_2d(sA + (size_t)stage * BK * BM, &mapA, &full[stage], (int)x0, y);
        tma_load_2d(sB + (size_t)stage * BK * BN, &mapB, &full[stage], (int)n0, y);
        ++issued;
        if ((++ps) * BK >= walk.len(pl)) { ps = 0; ++pl; }
    };
    if (tid == 0) {
        for (int s = 0; s < STAGES; ++s) mbar_init(&full[s], 1);
        fence_barrier_init();
        tma_prefetch_desc(&mapA);
        tma_prefetch_desc(&mapB);
        for (int s = 0; s < STAGES; ++s) issue_next();
    }
    __syncthreads();

    const int tx = tid % (BN / TN), ty = tid / (BN / TN);
    T acc[TM][TN];
    T cacc[Cfg::NCACC][TM][TN];
#pragma unroll
    for (int i = 0; i < TM; ++i)
#pragma unroll
        for (int j = 0; j < TN; ++j) {
            acc[i][j] = T(0);
#pragma unroll
            for (int d = 0; d < Cfg::NCACC; ++d) cacc[d][i][j] = T(0);
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

    int it = 0;
    bool ok = true;
    for (int l = 0; l < nslab && ok; ++l) {
        const int slen = walk.len(l);
        for (int s = 0; s * BK < slen; ++s, ++it) {
            const int stage = it % STAGES;
            const bool got = mbar_wait_bounded(&full[stage], (it / STAGES) & 1);
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
#pragma unroll
                    for (int i = 0; i < TM; ++i)
#pragma unroll
                        for (int j = 0; j < TN; ++j) acc[i][j] = fma_rn(a[i], b[j], acc[i][j]);
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
#pragma unroll
                    for (int i = 0; i < TM; ++i)
#pragma unroll
                        for (int j = 0; j < TN; ++j) acc[i][j] = fma_rn(a[i], b[j], acc[i][j]);
                }
            }
        }
        if (!ok) break;
        if (FORM != G_PLAIN) {
            // ---- slab end: keep (optionally), unpack, de-compand, accumulate
#pragma unroll
            for (int gi = 0; gi < RG; ++gi)
#pragma unroll
                for (int hj = 0; hj < CG; ++hj)
#pragma unroll
                    for (int e = 0; e < 4; ++e) {
                        const T pr = g.pair[((long long)l * g.nM + iblk[gi * 4 + e]) * g.nN +
                                            jblk[hj]];
#pragma unroll
                        for (int f = 0; f < 4; ++f) {
                            const int i = gi * 4 + e, j = hj * 4 + f;
                            T r = acc[i][j];
                            if (g.Rbar) {
                                long long xr = x0 + gi * (BM / RG) + ty * 4 + e;
                                long long nc = n0 + hj * (BN / CG) + tx * 4 + f;
                                if (xr < g.Mrows && nc < g.N)
                                    g.Rbar[((long long)l * g.Mrows + xr) * g.N + nc] = r;
                            }
                            if (FORM == G_SYM) {
                                const T u = rint_t(r);                      // eq. 9
                                const T t = rint_t(mul_rn(z, u));
                                const T rt = fma_rn(-Q, t, u);              // eq. 10
                                cacc[0][i][j] = fma_rn(rt, pr, cacc[0][i][j]);
                            } else {
                                T x = r;
#pragma unroll
                                for (int d = 0; d < W; ++d) {               // eqs. 13-14
                                    const T rt = rint_t(x);
                                    cacc[d][i][j] = fma_rn(rt, pr, cacc[d][i][j]);
                                    if (d + 1 < W) x = mul_rn(Q, sub_rn(x, rt));
                                }
                            }
                            acc[i][j] = T(0);
                        }
                }
        }
    }
    if (!ok) {
        // let every copy this CTA issued land before it exits
        if (tid == 0)
            for (int k = it; k < issued; ++k) mbar_wait_bounded(&full[k % STAGES], (k / STAGES) & 1);
        return;
    }

    // ---------------------------------------------------------------- store C
#pragma unroll
    for (int gi = 0; gi < RG; ++gi)
#pragma unroll
        for (int e = 0; e < 4; ++e) {
            const long long xr = x0 + gi * (BM / RG) + ty * 4 + e;
#pragma unroll
            for (int d = 0; d < Cfg::NCACC; ++d) {
                long long row;
                if (FORM == G_ASYM) {
                    const long long ib = xr / g.P, jr = xr % g.P;
                    const long long inblk = jr * W + d;
                    if (inblk >= g.L) continue;
                    row = ib * g.L + inblk;
                } else {
                    row = xr;
                }
                if (row >= g.M) continue;
                T *crow = g.C + row * g.ldc;
#pragma unroll
                for (int hj = 0; hj < CG; ++hj)
#pragma unroll
                    for (int f = 0; f < 4; ++f) {
                        const long long nc = n0 + hj * (BN / CG) + tx * 4 + f;
                        if (nc >= g.N) continue;
                        const T v = FORM == G_PLAIN ? acc[gi * 4 + e][hj * 4 + f]
                                                    : cacc[d][gi * 4 + e][hj * 4 + f];
                        crow[nc] = g.beta_zero ? mul_rn(g.alpha, v)
                                               : fma_rn(g.alpha, v, mul_rn(g.beta, crow[nc]));
                    }
            }
        }
}

template <typename T, int FORM, int W, int BM, int BN, int TM, int TN, int BK, int STAGES>
cudaError_t launch_cfg(const GemmArgs<T> &g, const CUtensorMap &mapA, const CUtensorMap &mapB,
                       cudaStream_t st) {
    using Cfg = GemmCfg<T, FORM, W, BM, BN, TM, TN, BK, STAGES>;
    auto kern = packed_gemm_kernel<T, FORM, W, BM, BN, TM, TN, BK, STAGES>;
    static bool attr_set = false;
    if (!attr_set) {
        cudaError_t e =
            cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)Cfg::SMEM);
        if (e != cudaSuccess) return e;
        attr_set = true;
    }
    dim3 grid((unsigned)((g.N + BN - 1) / BN), (unsigned)((g.Mrows + BM - 1) / BM));
    kern<<<grid, Cfg::NT, Cfg::SMEM, st>>>(mapA, mapB, g);
    return cudaGetLastError();
}

}  // namespace tdg
