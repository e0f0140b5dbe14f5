// Pair-exact companders (eq. 26 for every subblock product, Prop. 4): the
// symmetric product with companders chosen per (i, l, j) instead of the
// separable Gamma_A, Gamma_B of the default path.
//
// The quantized block A~_il then depends on the block B_lj it meets, so A (and
// B) cannot be packed once per call.  Each CTA computes one L x L output block
// (L equals the CTA tile) and quantizes and packs its operands itself: 2-D TMA
// brings raw k-slices of op(A) (row-major, box {BK W, L}) and op(B) ({L, BK W})
// into a ring, all threads compand them with the pair's scalars
// c_A,ilj and c_B,ilj and pack W digits per number (eqs. 3, 6, 7) into a
// packed tile in shared memory, then the packed multiply-accumulate, unpack
// and de-compand run as in the default kernel, with the pair's factor
// (T)(s_A,ilj s_B,ilj).  Every operation and its order are those of the
// default path for one block pair, so results equal the oracle bit for bit.
//
// All waits are bounded (2 s); on expiry the CTA records TDG_ETIMEOUT, waits
// (bounded) for its copies, frees its TMEM and returns.
#include "tdg_gemm.cuh"

namespace tdg {

namespace {

template <int BM_, int BN_, int TM_, int TN_, int BK_, int STAGES_>
struct PxTiles {
    static constexpr int BM = BM_, BN = BN_, TM = TM_, TN = TN_, BK = BK_, STAGES = STAGES_;
};
using PxF32 = PxTiles<128, 128, 8, 8, 16, 2>;
using PxF64 = PxTiles<64, 64, 4, 4, 16, 2>;

// c_A,ilj, c_B,ilj (in T) at [(i nK + l) nN + j] and (T)(s_A,ilj s_B,ilj) at
// [(l nM + i) nN + j], from the block statistics and the call's R_max
template <typename T>
__global__ void px_scales_kernel(PlanParams pp, const double *__restrict__ mA,
                                 const double *__restrict__ vA, const double *__restrict__ mB,
                                 const double *__restrict__ vB, const DevPlan *__restrict__ plan,
                                 T *cA, T *cB, T *pair) {
    pdl_entry();
    const long long R = plan->R;
    if (plan->W < 2) return;                       // conventional product chosen
    const long long n = (long long)pp.nM * pp.nK * pp.nN;
    for (long long e = (long long)blockIdx.x * blockDim.x + threadIdx.x; e < n;
         e += (long long)gridDim.x * blockDim.x) {
        const long long i = e / ((long long)pp.nK * pp.nN);
        const long long r = e - i * pp.nK * pp.nN;
        const long long l = r / pp.nN, j = r - l * pp.nN;
        const double ma = mA[i * pp.nK + l], va = vA[i * pp.nK + l];
        const double mb = mB[l * pp.nN + j], vb = vB[l * pp.nN + j];
        const double t1 = __dmul_rn(va, __dmul_rn(mb, mb));
        const double t2 = __dmul_rn(vb, __dmul_rn(ma, ma));
        const double rho = (t1 > 0.0 && t2 > 0.0) ? __dsqrt_rn(__ddiv_rn(t2, t1)) : 1.0;
        int gA, gB;
        split_gammas(R, pp.L, rho, gA, gB);
        double ca = 0.0, cb = 0.0, sa = 0.0, sb = 0.0;
        if (ma > 0.0) { ca = __ddiv_rn((double)gA, ma); sa = __ddiv_rn(1.0, ca); }
        if (mb > 0.0) { cb = __ddiv_rn((double)gB, mb); sb = __ddiv_rn(1.0, cb); }
        cA[e] = (T)ca;
        cB[e] = (T)cb;
        pair[(l * pp.nM + i) * pp.nN + j] = (T)__dmul_rn(sa, sb);
    }
}

template <typename T>
__device__ inline T quant_px(T v, T c) {
    if constexpr (sizeof(T) == 4) return rintf(__fmul_rn(v, c));
    else return rint(__dmul_rn(v, c));
}

template <typename T, int W, typename C>
struct PxCfg {
    static constexpr int BM = C::BM, BN = C::BN, TM = C::TM, TN = C::TN, BK = C::BK;
    static constexpr int STAGES = C::STAGES;
    static constexpr int NT = (BM / TM) * (BN / TN);
    static constexpr int RG = TM / 4, CG = TN / 4;
    static constexpr int KR = BK * W;                        // raw k per stage
    static constexpr size_t RAW_A = (size_t)BM * KR * sizeof(T);
    static constexpr size_t RAW_B = (size_t)KR * BN * sizeof(T);
    static constexpr int PITCH_A = BM + 4;                   // packed A rows, padded
    static constexpr size_t PK_A = (size_t)BK * PITCH_A * sizeof(T);
    static constexpr size_t PK_B = (size_t)BK * BN * sizeof(T);
    static constexpr bool TMEMC = sizeof(T) == 4;
    static constexpr int NC = TM * TN;
    static constexpr int TMEM_COLS = pow2_at_least(2 * NC);
    static constexpr size_t SMEM =
        STAGES * (RAW_A + RAW_B) + PK_A + PK_B + STAGES * sizeof(uint64_t) + 16;
    static_assert(BM / TM == 16 && BN / TN == 16, "16 x 16 thread grid");
};

template <typename T, int W, typename C>
__global__ void __launch_bounds__(PxCfg<T, W, C>::NT, sizeof(T) == 4 ? 2 : 1)
    px_gemm_kernel(const __grid_constant__ CUtensorMap mapA,
                   const __grid_constant__ CUtensorMap mapB, const GemmArgs<T> g) {
    pdl_entry();
    using Cfg = PxCfg<T, W, C>;
    constexpr int BM = Cfg::BM, BN = Cfg::BN, TM = Cfg::TM, TN = Cfg::TN, BK = Cfg::BK;
    constexpr int STAGES = Cfg::STAGES, NT = Cfg::NT, RG = Cfg::RG, CG = Cfg::CG, KR = Cfg::KR;
    constexpr int PA = Cfg::PITCH_A;
    constexpr bool TMEMC = Cfg::TMEMC;

    if (g.plan->W != W) return;                 // the planner chose another packing
    const long long tmi = (long long)(blockIdx.x / g.ntn);
    const long long tnj = (long long)blockIdx.x - tmi * g.ntn;
    const long long x0 = tmi * BM, n0 = tnj * BN;   // the block pair (i, j) = (tmi, tnj)

    extern __shared__ __align__(128) unsigned char smem[];
    T *rawA = reinterpret_cast<T *>(smem);
    T *rawB = reinterpret_cast<T *>(smem + STAGES * Cfg::RAW_A);
    T *pkA = reinterpret_cast<T *>(smem + STAGES * (Cfg::RAW_A + Cfg::RAW_B));
    T *pkB = reinterpret_cast<T *>(smem + STAGES * (Cfg::RAW_A + Cfg::RAW_B) + Cfg::PK_A);
    uint64_t *full = reinterpret_cast<uint64_t *>(smem + STAGES * (Cfg::RAW_A + Cfg::RAW_B) +
                                                  Cfg::PK_A + Cfg::PK_B);
    uint32_t *tmem_slot = reinterpret_cast<uint32_t *>(full + STAGES);

    const int tid = threadIdx.x, warp = tid >> 5;
    const int sps = g.P / BK;                    // stages per slab (P = L / W)
    const int total = g.nK * sps;

    int issued = 0;
    auto issue_next = [&]() {
        if (issued >= total) return;
        const int stage = issued % STAGES;
        const int l = issued / sps, s = issued % sps;
        const int k0 = l * g.L + s * KR;
        mbar_arrive_expect_tx(&full[stage], (uint32_t)(Cfg::RAW_A + Cfg::RAW_B));
        tma_load_2d(rawA + (size_t)stage * BM * KR, &mapA, &full[stage], k0, (int)x0);
        tma_load_2d(rawB + (size_t)stage * KR * BN, &mapB, &full[stage], (int)n0, k0);
        ++issued;
    };
    if (TMEMC && warp == 0) tmem_alloc(tmem_slot, Cfg::TMEM_COLS);
    if (tid == 0) {
        for (int s = 0; s < STAGES; ++s) mbar_init(&full[s], 1);
        fence_barrier_init();
        tma_prefetch_desc(&mapA);
        tma_prefetch_desc(&mapB);
        for (int s = 0; s < STAGES; ++s) issue_next();
    }
    if (TMEMC) tmem_fence_before();
    __syncthreads();
    if (TMEMC) tmem_fence_after();
    const uint32_t tcol = TMEMC ? *tmem_slot + ((uint32_t)(32 * (warp & 3)) << 16) +
                                      (uint32_t)((warp >> 2) * Cfg::NC)
                                : 0u;

    const int tx = tid % (BN / TN), ty = tid / (BN / TN);
    T acc[TM][TN];
    T cacc[TMEMC ? 1 : TM][TMEMC ? 1 : TN];
#pragma unroll
    for (int i = 0; i < TM; ++i)
#pragma unroll
        for (int j = 0; j < TN; ++j) acc[i][j] = T(0);
    if constexpr (!TMEMC) {
#pragma unroll
        for (int i = 0; i < TM; ++i)
#pragma unroll
            for (int j = 0; j < TN; ++j) cacc[i][j] = T(0);
    }
    const T z = pow2_t(T(0), -g.plan->q), Q = pow2_t(T(0), g.plan->q);

    bool ok = true;
    T ca = T(0), cb = T(0);
    for (int it = 0; it < total && ok; ++it) {
        const int stage = it % STAGES;
        const int l = it / sps, s = it % sps;
        if (s == 0) {
            const long long e = (tmi * g.nK + l) * g.nN + tnj;
            ca = g.cApx[e];
            cb = g.cBpx[e];
        }
        const bool got = mbar_wait_bounded(&full[stage], (it / STAGES) & 1);
        // every thread is past the MAC of stage it - 1: the packed tiles are free
        if (!__syncthreads_and(got)) {
            if (tid == 0) raise_status(const_cast<DevPlan *>(g.plan), TDG_ETIMEOUT);
            ok = false;
            break;
        }
        // ---- compand (eq. 3) and pack (eqs. 6, 7) this stage's raw slices
        const T *ra = rawA + (size_t)stage * BM * KR;
        const T *rb = rawB + (size_t)stage * KR * BN;
        for (int e = tid; e < BM * BK; e += NT) {
            const int m = e / BK, kk = e - m * BK;
            T v = quant_px(ra[m * KR + W * kk + (W - 1)], ca);
#pragma unroll
            for (int d = W - 2; d >= 0; --d) v = fma_rn(z, v, quant_px(ra[m * KR + W * kk + d], ca));
            pkA[kk * PA + m] = v;
        }
        for (int e = tid; e < BK * BN; e += NT) {
            const int kk = e / BN, n = e - kk * BN;
            T v = quant_px(rb[(W * kk + (W - 1)) * BN + n], cb);
#pragma unroll
            for (int d = W - 2; d >= 0; --d) v = fma_rn(Q, v, quant_px(rb[(W * kk + d) * BN + n], cb));
            pkB[kk * BN + n] = v;
        }
        __syncthreads();
        if (tid == 0) issue_next();              // the raw slot is consumed
        // ---- packed multiply-accumulate (eq. 8)
#pragma unroll
        for (int kk = 0; kk < BK; ++kk) {
            T a[TM], b[TN];
#pragma unroll
            for (int gi = 0; gi < RG; ++gi)
                Vec4<T>::load(pkA + kk * PA + gi * (BM / RG) + ty * 4, a + 4 * gi);
#pragma unroll
            for (int hj = 0; hj < CG; ++hj)
                Vec4<T>::load(pkB + kk * BN + hj * (BN / CG) + tx * 4, b + 4 * hj);
            outer_fma(acc, a, b);
        }
        if (s != sps - 1) continue;

        // ---- slab end: unpack (eqs. 9-10), de-compand with the pair's factor
        const T pr = g.pair[((long long)l * g.nM + tmi) * g.nN + tnj];
        const bool first = l == 0;
        float v[16];
#pragma unroll
        for (int e = 0; e < TM * TN; ++e) {
            const int i = e / TN, j = e % TN;
            const T r = acc[i][j];
            acc[i][j] = T(0);
            const T u = rint_epi(r);                        // eq. 9
            const T t = rint_epi(mul_rn(z, u));
            const T digit = fma_rn(-Q, t, u);               // eq. 10
            if constexpr (TMEMC) {
                const int slot = e % 16;
                if (slot == 0) {
                    if (first) {
#pragma unroll
                        for (int q = 0; q < 16; ++q) v[q] = 0.f;
                    } else {
                        tmem_ld16(tcol + (uint32_t)e, v);
                    }
                }
                v[slot] = fma_rn((float)digit, (float)pr, v[slot]);
                if (slot == 15) tmem_st16(tcol + (uint32_t)(e - 15), v);
            } else {
                cacc[i][j] = fma_rn(digit, pr, cacc[i][j]);
            }
        }
        if constexpr (TMEMC) tmem_wait_st();
    }

    auto store_c = [&](long long row, long long col, T val) {
        if (row >= g.M || col >= g.N) return;
        T *p = g.C + row * g.ldc + col;
        *p = g.beta_zero ? mul_rn(g.alpha, val) : fma_rn(g.alpha, val, mul_rn(g.beta, *p));
    };
    auto out_row = [&](int i) { return x0 + (i / 4) * (BM / RG) + ty * 4 + (i % 4); };
    auto out_col = [&](int j) { return n0 + (j / 4) * (BN / CG) + tx * 4 + (j % 4); };
    if (!ok) {
        if (tid == 0)
            for (int k = 0; k < issued; ++k) mbar_wait_bounded(&full[k % STAGES], (k / STAGES) & 1);
    } else if constexpr (TMEMC) {
#pragma unroll
        for (int f0 = 0; f0 < Cfg::NC; f0 += 16) {
            float vv[16];
            tmem_ld16(tcol + (uint32_t)f0, vv);
#pragma unroll
            for (int q = 0; q < 16; ++q) {
                const int e = f0 + q;
                store_c(out_row(e / TN), out_col(e % TN), (T)vv[q]);
            }
        }
    } else {
#pragma unroll
        for (int i = 0; i < TM; ++i)
#pragma unroll
            for (int j = 0; j < TN; ++j) store_c(out_row(i), out_col(j), cacc[i][j]);
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

template <typename T, int W, typename C>
cudaError_t launch_px_w(const GemmArgs<T> &g0, const GemmOperands &ops, cudaStream_t st) {
    using Cfg = PxCfg<T, W, C>;
    auto kern = px_gemm_kernel<T, W, C>;
    static bool attr_set = false;
    if (!attr_set) {
        cudaError_t e =
            cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)Cfg::SMEM);
        if (e != cudaSuccess) return e;
        attr_set = true;
    }
    const CUtensorMapDataType dt =
        sizeof(T) == 8 ? CU_TENSOR_MAP_DATA_TYPE_FLOAT64 : CU_TENSOR_MAP_DATA_TYPE_FLOAT32;
    CUtensorMap ma, mb;
    // op(A) row-major [M][K]: box {BK W (k), BM (m)}; op(B) row-major [K][N]: box {BN, BK W}
    if (encode_map_2d(&ma, dt, sizeof(T), ops.a.base, ops.a.cols, ops.a.rows, ops.a.ld, Cfg::KR,
                      C::BM, CU_TENSOR_MAP_SWIZZLE_NONE) != CUDA_SUCCESS ||
        encode_map_2d(&mb, dt, sizeof(T), ops.b.base, ops.b.cols, ops.b.rows, ops.b.ld, C::BN,
                      Cfg::KR, CU_TENSOR_MAP_SWIZZLE_NONE) != CUDA_SUCCESS)
        return cudaErrorInvalidValue;
    GemmArgs<T> g = g0;
    g.ntn = (int)((g.N + C::BN - 1) / C::BN);
    const long long ntiles = ((g.M + C::BM - 1) / C::BM) * g.ntn;
    if (ntiles > 0x7fffffffLL) return cudaErrorInvalidConfiguration;
    return launch_pdl_if(pdl_for_grid(ntiles), kern, dim3((unsigned)ntiles), dim3(Cfg::NT),
                         Cfg::SMEM, st, ma, mb, g);
}

}  // namespace

int pair_exact_tile(int dtype) { return dtype == TDG_F64 ? PxF64::BM : PxF32::BM; }
int pair_exact_bk() { return PxF32::BK; }

template <typename T>
cudaError_t launch_px_scales(const PlanParams &pp, const double *mA, const double *vA,
                             const double *mB, const double *vB, const DevPlan *plan, T *cA,
                             T *cB, T *pair, cudaStream_t st) {
    const long long n = (long long)pp.nM * pp.nK * pp.nN;
    const int grid = (int)std::min<long long>((n + 255) / 256, 152LL * 8);
    return launch_pdl(px_scales_kernel<T>, dim3(grid), dim3(256), 0, st, pp, mA, vA, mB, vB, plan,
                      cA, cB, pair);
}

template <typename T>
cudaError_t launch_px_gemm(int W, const GemmArgs<T> &g, const GemmOperands &ops, cudaStream_t st) {
    using C = std::conditional_t<sizeof(T) == 8, PxF64, PxF32>;
    switch (W) {
        case 2: return launch_px_w<T, 2, C>(g, ops, st);
        case 4: return launch_px_w<T, 4, C>(g, ops, st);
    }
    return cudaErrorNotSupported;
}

template cudaError_t launch_px_scales<float>(const PlanParams &, const double *, const double *,
                                             const double *, const double *, const DevPlan *,
                                             float *, float *, float *, cudaStream_t);
template cudaError_t launch_px_scales<double>(const PlanParams &, const double *, const double *,
                                              const double *, const double *, const DevPlan *,
                                              double *, double *, double *, cudaStream_t);
template cudaError_t launch_px_gemm<float>(int, const GemmArgs<float> &, const GemmOperands &,
                                           cudaStream_t);
template cudaError_t launch_px_gemm<double>(int, const GemmArgs<double> &, const GemmOperands &,
                                            cudaStream_t);

}  // namespace tdg
