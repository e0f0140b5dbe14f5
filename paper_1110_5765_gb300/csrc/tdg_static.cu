// tdgemm_run_static: the fixed-bit companded-and-packed product with every
// intermediate buffer in one file-scope device array instead of memory from
// cudaMalloc.
//
// Who needs it: callers that may not allocate device memory at the point of
// the call — frameworks whose allocator owns the whole device and forbids side
// allocations by libraries, plug-ins that are handed only the buffers they
// compute on, and services that must not take a first-use allocation (and the
// device-wide synchronisation cudaMalloc/cudaFree can imply) on a hot path.
// They pass A, B and C; the statistics, companders, de-companding factors and
// packed operands live in g_scratch below.
//
// Unlike the plan-based path, nothing reports device-side conditions back: a
// NaN or Inf in A or B is flagged in the plan record inside g_scratch, which
// no entry point reads, and C then holds non-finite values.
//
// Limits and sharing:
//   * g_scratch holds kStaticScratchBytes (32 MiB) on every GPU that loads the
//     library, for the life of the process.  A problem whose workspace is
//     larger is rejected with TDG_EINVAL before any device work.
//   * Every call uses the same array; it keeps the previous call's contents.
//     The per-call plan record is cleared at the start of every call; every
//     other byte a call reads it has written first.  Two calls whose device
//     work overlaps (different streams, or different host threads on one
//     device) race on the array: order them on one stream.
//   * The first call on a device looks up the array's device address
//     (cudaGetSymbolAddress, with that device current) and caches it.
// The paper has no counterpart to this entry point.
#include <cuda.h>
#include <cuda_runtime.h>
#include <math.h>
#include <stdarg.h>
#include <stdio.h>

#include <algorithm>
#include <mutex>

#include "tdg_common.cuh"
#include "tdg_internal.h"
#include "tdgemm.h"

namespace tdg {
namespace {

constexpr size_t kStaticScratchBytes = 32ull << 20;
static __device__ __align__(256) unsigned char g_scratch[kStaticScratchBytes];

constexpr int kMaxDevices = 64;
unsigned char *g_scratch_dev[kMaxDevices] = {};
std::mutex g_setup_mutex;

tdg_status err(tdg_status st, const char *fmt, ...) {
    char buf[512];
    va_list ap;
    va_start(ap, fmt);
    vsnprintf(buf, sizeof(buf), fmt, ap);
    va_end(ap);
    record_error(buf);
    return st;
}

// device address of g_scratch for the current device (host code must not use
// the symbol's host-side stand-in as a device pointer)
tdg_status scratch_for_current_device(unsigned char **out) {
    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) return err(TDG_ECUDA, "cudaGetDevice: %s", cudaGetErrorString(e));
    if (dev < 0 || dev >= kMaxDevices) return err(TDG_EUNSUPPORTED, "device ordinal %d", dev);
    std::lock_guard<std::mutex> lock(g_setup_mutex);
    if (!g_scratch_dev[dev]) {
        void *p = nullptr;
        e = cudaGetSymbolAddress(&p, g_scratch);
        if (e != cudaSuccess || !p)
            return err(TDG_ECUDA, "cudaGetSymbolAddress(g_scratch): %s", cudaGetErrorString(e));
        g_scratch_dev[dev] = (unsigned char *)p;
    }
    *out = g_scratch_dev[dev];
    return TDG_OK;
}

long long rup(long long v, long long m) { return (v + m - 1) / m * m; }

#define ST_TRY(expr)                                                                    \
    do {                                                                                \
        cudaError_t e_ = (expr);                                                        \
        if (e_ != cudaSuccess)                                                          \
            return err(TDG_ECUDA, "%s failed: %s", #expr, cudaGetErrorString(e_));      \
    } while (0)

template <typename T>
tdg_status run_static(bool nA, bool nB, long long M, long long N, long long K, long long lda,
                      long long ldb, long long ldc, int L, int W, int form, int bits,
                      const T *A, const T *B, T *C, double alpha, double beta,
                      cudaStream_t st) {
    const int nM = cdiv_i(M, L), nK = cdiv_i(K, L), nN = cdiv_i(N, L);
    const int P = (L + W - 1) / W;
    // operand shapes (k-major), as the plan-based entry points lay them out
    long long a_rows, a_cols, b_rows = 0, b_cols = N;
    if (form == TDG_SYM) { a_rows = (long long)nK * P; a_cols = M; b_rows = a_rows; }
    else { a_rows = K; a_cols = (long long)nM * P; b_rows = K; }
    const long long a_ld = rup(a_cols, 32), b_ld = rup(b_cols, 32);
    // carve the scratch (256-byte aligned pieces)
    const size_t nA_blk = (size_t)nM * nK, nB_blk = (size_t)nK * nN;
    size_t off = 0;
    auto take = [&](size_t bytes) { size_t o = off; off += (bytes + 255) / 256 * 256; return o; };
    const size_t o_plan = take(sizeof(DevPlan));
    const size_t o_agg =
        take(((size_t)4 * nK + (size_t)kLevelRecDoubles * (kMaxW - 1) * kMaxLevels) * 8);
    const size_t o_mA = take(nA_blk * 8), o_eA = take(nA_blk * 8);
    const size_t o_mB = take(nB_blk * 8), o_eB = take(nB_blk * 8);
    const size_t o_sA = take(nA_blk * 8), o_sB = take(nB_blk * 8);
    const size_t o_cA = take(nA_blk * sizeof(T)), o_cB = take(nB_blk * sizeof(T));
    const size_t o_pair = take((size_t)nK * nM * nN * sizeof(T));
    const size_t o_A = take((size_t)(a_rows * a_ld) * sizeof(T));
    const size_t o_B = take((size_t)(b_rows * b_ld) * sizeof(T));
    if (off > kStaticScratchBytes)
        return err(TDG_EINVAL,
                   "tdgemm_run_static: this product needs %zu bytes of scratch; the static "
                   "scratch holds %zu bytes (use tdgemm_plan for larger products)",
                   off, kStaticScratchBytes);
    unsigned char *ws = nullptr;
    tdg_status s = scratch_for_current_device(&ws);
    if (s != TDG_OK) return s;
    DevPlan *dplan = (DevPlan *)(ws + o_plan);
    double *agg = (double *)(ws + o_agg);
    double *mA = (double *)(ws + o_mA), *eA = (double *)(ws + o_eA);
    double *mB = (double *)(ws + o_mB), *eB = (double *)(ws + o_eB);
    double *sA = (double *)(ws + o_sA), *sB = (double *)(ws + o_sB);
    T *cA = (T *)(ws + o_cA), *cB = (T *)(ws + o_cB), *pair = (T *)(ws + o_pair);
    T *Abuf = (T *)(ws + o_A), *Bbuf = (T *)(ws + o_B);

    // the plan record carries the device status, the non-finite flag and the
    // planner's counter: start at zero
    ST_TRY(cudaMemsetAsync(dplan, 0, sizeof(DevPlan), st));
    ST_TRY(launch_block_stats<T>(A, nA ? M : K, nA ? K : M, lda, nA ? 0 : 1, nK, mA, eA, B,
                                 nB ? K : N, nB ? N : K, ldb, nB ? 0 : 1, nN, mB, eB, L, dplan,
                                 st));
    PlanParams pp{};
    pp.mode = MODE_FIXED; pp.form = form; pp.dtype = sizeof(T) == 8 ? TDG_F64 : TDG_F32;
    pp.L = L; pp.Wreq = W; pp.p = sizeof(T) == 8 ? 53 : 24; pp.bits = bits;
    pp.allow_fallback = 0; pp.noise_rms = 0; pp.target_db = NAN;
    pp.nM = nM; pp.nK = nK; pp.nN = nN; pp.M = M; pp.N = N; pp.K = K;
    pp.t0 = 0; pp.nt = 0;
    ST_TRY(launch_planner<T>(pp, mA, eA, mB, eB, nullptr, dplan, agg, cA, sA, cB, sB, pair, st));
    PackOperand<T> oa{}, ob{};
    oa.src = A; oa.X = M; oa.K = K; oa.L = L; oa.c = cA; oa.cx = nK; oa.cl = 1;
    if (nA) { oa.sx = lda; oa.sk = 1; } else { oa.sx = 1; oa.sk = lda; }
    ob.src = B; ob.X = N; ob.K = K; ob.L = L; ob.c = cB; ob.cx = 1; ob.cl = nN;
    if (nB) { ob.sx = 1; ob.sk = ldb; } else { ob.sx = ldb; ob.sk = 1; }
    if (form == TDG_SYM) {
        ST_TRY(launch_pack_k<T>(oa, W, dplan, W, -1, Abuf, a_ld, a_rows, st));
        ST_TRY(launch_pack_k<T>(ob, W, dplan, W, +1, Bbuf, b_ld, b_rows, st));
    } else {
        ST_TRY(launch_pack_x<T>(oa, W, dplan, W, -1, Abuf, a_ld, st));
        ST_TRY(launch_pack_k<T>(ob, 1, dplan, W, 0, Bbuf, b_ld, b_rows, st));
    }
    const int gform = form == TDG_SYM ? G_SYM : G_ASYM;
    GemmOperands ops{};
    ops.a = {Abuf, a_cols, a_rows, a_ld};
    ops.b = {Bbuf, b_cols, b_rows, b_ld};
    GemmArgs<T> g{};
    g.plan = dplan; g.M = M; g.N = N; g.K = K; g.Mrows = a_cols; g.Krows = a_rows;
    g.L = L; g.P = P; g.nM = nM; g.nK = nK; g.nN = nN; g.pair = pair;
    g.C = C; g.ldc = ldc; g.alpha = (T)alpha; g.beta = (T)beta; g.beta_zero = beta == 0.0;
    g.Rbar = nullptr;
    {
        const long long gam = (1LL << (bits - 1)) - 1;
        g.small_t = small_round_ok(gform, W, q_for((long long)L * gam * gam), (int)gam) ? 1 : 0;
    }
    ST_TRY(launch_packed_gemm<T>(gform, W, g, ops, st));
    return TDG_OK;
}

}  // namespace
}  // namespace tdg

extern "C" tdg_status tdgemm_run_static(char transA, char transB, int64_t M, int64_t N,
                                        int64_t K, int64_t lda, int64_t ldb, int64_t ldc,
                                        int L, int W, tdg_dtype dtype, tdg_form form, int bits,
                                        const void *A, const void *B, void *C, double alpha,
                                        double beta, void *stream) {
    using namespace tdg;
    auto okT = [](char t) { return t == 'N' || t == 'n' || t == 'T' || t == 't'; };
    if (!okT(transA) || !okT(transB)) return err(TDG_EINVAL, "trans must be 'N' or 'T'");
    if (M < 1 || N < 1 || K < 1) return err(TDG_EINVAL, "M, N, K must be >= 1");
    // the block counts and tile coordinates are 32-bit: sizes beyond 2^31 would
    // wrap them and with them the scratch layout
    if (M > (1LL << 31) || N > (1LL << 31) || K > (1LL << 31))
        return err(TDG_EINVAL, "M, N, K must be <= 2^31");
    const bool nA = transA == 'N' || transA == 'n', nB = transB == 'N' || transB == 'n';
    if (lda < (nA ? K : M) || ldb < (nB ? N : K) || ldc < N)
        return err(TDG_EINVAL, "leading dimension too small");
    if (dtype != TDG_F32 && dtype != TDG_F64) return err(TDG_EINVAL, "bad dtype");
    if (form != TDG_SYM && form != TDG_ASYM)
        return err(TDG_EINVAL, "tdgemm_run_static takes the SYM or ASYM form");
    if (L < 16 || L > 1024 || L % 16) return err(TDG_EINVAL, "L must be a multiple of 16 in [16, 1024]");
    if (W < 1 || W > kMaxW) return err(TDG_EINVAL, "W must be in 1..4");
    if (bits < 2 || bits > 20) return err(TDG_EINVAL, "bits must be in 2..20");
    if (!A || !B || !C) return err(TDG_EINVAL, "A, B and C must be device pointers");
    if (!isfinite(alpha) || !isfinite(beta)) return err(TDG_EINVAL, "alpha/beta not finite");
    cudaStream_t st = (cudaStream_t)stream;
    if (dtype == TDG_F64)
        return run_static<double>(nA, nB, M, N, K, lda, ldb, ldc, L, W, form, bits,
                                  (const double *)A, (const double *)B, (double *)C, alpha, beta,
                                  st);
    return run_static<float>(nA, nB, M, N, K, lda, ldb, ldc, L, W, form, bits,
                             (const float *)A, (const float *)B, (float *)C, alpha, beta, st);
}
