// The C ABI of include/tdgemm.h: plan objects, argument checks, workspace,
// and the stream-ordered launch sequence of steps (a)-(d).
#include <cuda.h>
#include <cuda_runtime.h>
#include <math.h>
#include <stdarg.h>
#include <stdio.h>
#include <string.h>

#include <algorithm>
#include <mutex>
#include <vector>

#include "tdg_common.cuh"
#include "tdg_internal.h"
#include "tdg_pack.h"
#include "tdgemm.h"

using namespace tdg;

// ---------------------------------------------------------------------------
// errors
// ---------------------------------------------------------------------------
static thread_local char g_err[512] = "";

static tdg_status fail(tdg_status st, const char *fmt, ...) {
    va_list ap;
    va_start(ap, fmt);
    vsnprintf(g_err, sizeof(g_err), fmt, ap);
    va_end(ap);
    return st;
}

// lets other translation units report through tdgemm_last_error()
void tdg::record_error(const char *msg) { snprintf(g_err, sizeof(g_err), "%s", msg); }

int tdg::device_sms() {
    static std::mutex mu;
    static int sms[64] = {};
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= 64) return 1;
    std::lock_guard<std::mutex> lock(mu);
    if (!sms[dev]) {
        int n = 0;
        if (cudaDeviceGetAttribute(&n, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess || n < 1)
            n = 1;
        sms[dev] = n;
    }
    return sms[dev];
}

#define CU_TRY(expr)                                                                  \
    do {                                                                              \
        cudaError_t e_ = (expr);                                                      \
        if (e_ != cudaSuccess)                                                        \
            return fail(e_ == cudaErrorMemoryAllocation ? TDG_ENOMEM : TDG_ECUDA,     \
                        "%s failed: %s (%s:%d)", #expr, cudaGetErrorString(e_),       \
                        __FILE__, __LINE__);                                          \
    } while (0)

// 2-D TMA map over a row-major [rows][cols] array with leading dimension ld.
static tdg_status make_map(CUtensorMap *m, CUtensorMapDataType dt, size_t esz, const void *base,
                           long long cols, long long rows, long long ld, int box_cols,
                           int box_rows, CUtensorMapSwizzle sw) {
    CUresult r = encode_map_2d(m, dt, esz, base, cols, rows, ld, box_cols, box_rows, sw);
    if (r == CUDA_ERROR_NOT_SUPPORTED) return fail(TDG_ECUDA, "cuTensorMapEncodeTiled is not available");
    if (r == CUDA_ERROR_INVALID_VALUE && (((uintptr_t)base & 15) || ((ld * (long long)esz) & 15)))
        return fail(TDG_EINVAL, "TMA operand not 16-byte aligned (ld=%lld)", ld);
    if (r != CUDA_SUCCESS) return fail(TDG_ECUDA, "cuTensorMapEncodeTiled failed (%d)", (int)r);
    return TDG_OK;
}

// ---------------------------------------------------------------------------
// plan object
// ---------------------------------------------------------------------------
static long long round_up(long long v, long long m) { return (v + m - 1) / m * m; }

struct tdgemm_plan_s {
    // problem
    char tA, tB;
    long long M, N, K, lda, ldb, ldc;
    int L, W, dtype, form, bits;
    double target;
    uint32_t flags;
    int mode, manual_q;
    double manual_cA, manual_cB;
    int nM, nK, nN;
    size_t esz;
    // device workspace (one allocation)
    unsigned char *ws = nullptr;
    size_t ws_bytes = 0;
    DevPlan *dplan = nullptr;
    double *mA, *eA, *mB, *eB, *sA, *sB, *stab, *agg;
    void *cA, *cB, *pair;
    void *Abuf, *Bbuf, *Rbar;
    void *cApx = nullptr, *cBpx = nullptr, *pairpx = nullptr;   // TDG_PAIR_EXACT
    size_t Abuf_bytes, Bbuf_bytes;
    std::vector<double> stab_host;
    bool stab_dirty = false;
    bool have_table = false;
    // host-buffer staging (tdgemm_run_host)
    void *hA = nullptr, *hB = nullptr, *hC = nullptr;
    // pipelined host-buffer staging (tdgemm_run_host_async): two sets, a copy
    // stream, per set an event after its copies and one after the computation
    // that read it
    struct HostSet {
        void *A = nullptr, *B = nullptr, *C = nullptr;
        cudaEvent_t copied = nullptr, done = nullptr;
        bool used = false;
    } hset[2];
    cudaStream_t copy_stream = nullptr;
    int next_set = 0;
    // Sec. 6 inner-kernel control (off: kctrl_mode == 0)
    int kctrl_mode = 0;
    double kctrl_value = 0.0, kctrl_thr = 0.0;
    long long kctrl_k = 0;
    Speedups speedup{};                       // F_W by W (Sec. 5.B), 0 = not given
    void *kA = nullptr, *kB = nullptr;        // plain k-major copies for unaccelerated kernels
    double *kratio = nullptr;
    unsigned char *kmask = nullptr;
    int *korder = nullptr;                    // launch order of the mixed GEMM's tiles
    long long ktiles_m = 0, ktiles_n = 0;
    // state
    const void *A_user = nullptr, *B_user = nullptr;
    bool packed = false, gemm_done = false, b_packed = false;
    int split_groups = 1;   // slab splitting of the packed GEMM (> 1: on)
    long long stall_ns = 0; // test of the bounded waits (tdgemm_set_wait_test)
    int last_pack_W = 0;
    cudaStream_t last_stream = nullptr;
    int device = 0;
};

static int Pof(int L, int W) { return (L + W - 1) / W; }

static bool is_packed_form(int f) { return f == TDG_SYM || f == TDG_ASYM; }
static bool is_tc_form(int f) { return f == TDG_TC_INT || f == TDG_TC_FP8; }

// candidate W values whose kernels are queued (each checks the device plan)
static std::vector<int> candidates(const tdgemm_plan_s *p) {
    std::vector<int> c;
    if (p->form == TDG_PLAIN || is_tc_form(p->form)) return {1};
    if (p->mode == MODE_TARGET) {
        for (int w = p->W; w >= 2; --w) c.push_back(w);
        if (p->flags & TDG_ALLOW_FALLBACK) c.push_back(0);   // 0: plain fallback
    } else {
        c.push_back(p->W);
    }
    return c;
}

// rows / cols / ld of the k-major operand buffers for candidate W (0 = plain)
struct OpShape {
    long long a_rows, a_cols, a_ld, b_rows, b_cols, b_ld;
};
static OpShape op_shape(const tdgemm_plan_s *p, int W) {
    OpShape s;
    const long long pad = 32;
    if (W == 0 || p->form == TDG_PLAIN) {
        s.a_rows = p->K; s.a_cols = p->M;
        s.b_rows = p->K; s.b_cols = p->N;
    } else if (p->form == TDG_SYM) {
        long long Kp = (long long)p->nK * Pof(p->L, W);
        s.a_rows = Kp; s.a_cols = p->M;
        s.b_rows = Kp; s.b_cols = p->N;
    } else {  // ASYM
        s.a_rows = p->K; s.a_cols = (long long)p->nM * Pof(p->L, W);
        s.b_rows = p->K; s.b_cols = p->N;
    }
    s.a_ld = round_up(s.a_cols, pad);
    s.b_ld = round_up(s.b_cols, pad);
    return s;
}

static tdg_status validate(char tA, char tB, long long M, long long N, long long K,
                           long long lda, long long ldb, long long ldc, int L, int W, int dtype,
                           int form, double target, int bits) {
    auto okT = [](char t) { return t == 'N' || t == 'n' || t == 'T' || t == 't'; };
    if (!okT(tA) || !okT(tB)) return fail(TDG_EINVAL, "trans must be 'N' or 'T'");
    if (M < 1 || N < 1 || K < 1) return fail(TDG_EINVAL, "M, N, K must be >= 1");
    if (M > (1LL << 31) || N > (1LL << 31) || K > (1LL << 31))
        return fail(TDG_EINVAL, "M, N, K must be <= 2^31");
    const bool nA = (tA == 'N' || tA == 'n'), nB = (tB == 'N' || tB == 'n');
    if (lda < (nA ? K : M)) return fail(TDG_EINVAL, "lda too small");
    if (ldb < (nB ? N : K)) return fail(TDG_EINVAL, "ldb too small");
    if (ldc < N) return fail(TDG_EINVAL, "ldc too small");
    if (dtype != TDG_F32 && dtype != TDG_F64) return fail(TDG_EINVAL, "bad dtype");
    if (form < TDG_PLAIN || form > TDG_TC_FP8) return fail(TDG_EINVAL, "bad form");
    if (L < 16 || L > 1024 || L % 16) return fail(TDG_EINVAL, "L must be a multiple of 16 in [16, 1024]");
    if (is_packed_form(form)) {
        if (W < 1 || W > kMaxW) return fail(TDG_EINVAL, "W must be in 1..4");
        if (bits > 0) {
            if (bits < 2 || bits > 20) return fail(TDG_EINVAL, "bits must be in 2..20");
        } else {
            if (!isfinite(target)) return fail(TDG_EINVAL, "target SNR must be finite when bits == 0");
            if (W < 2) return fail(TDG_EINVAL, "target mode needs W >= 2");
        }
    } else {
        if (W != 1) return fail(TDG_EINVAL, "W must be 1 for this form");
    }
    if (is_tc_form(form)) {
        if (dtype != TDG_F32) return fail(TDG_EUNSUPPORTED, "tensor-core forms take fp32 inputs");
        if (form == TDG_TC_INT && L % 64) return fail(TDG_EINVAL, "TC_INT needs L % 64 == 0");
        if (form == TDG_TC_FP8 && L % 128) return fail(TDG_EINVAL, "TC_FP8 needs L % 128 == 0");
        if (form == TDG_TC_INT) {
            if (bits > 0) {
                long long g = (1LL << (bits - 1)) - 1;
                if (bits > 12 || (double)L * g * g > kTcIntExact)
                    return fail(TDG_EINVAL, "TC_INT: L * gamma^2 must stay below 2^24 and gamma <= 2047");
            } else if (!isfinite(target)) {
                return fail(TDG_EINVAL, "target SNR must be finite when bits == 0");
            }
        }
    }
    return TDG_OK;
}

extern "C" tdg_status tdgemm_plan(tdgemm_plan_t *plan, char transA, char transB, int64_t M,
                                  int64_t N, int64_t K, int64_t lda, int64_t ldb, int64_t ldc,
                                  int L, int W, tdg_dtype dtype, tdg_form form,
                                  double target_snr_db, int bits, uint32_t flags) {
    if (!plan) return fail(TDG_EINVAL, "plan pointer is NULL");
    *plan = nullptr;
    tdg_status v = validate(transA, transB, M, N, K, lda, ldb, ldc, L, W, dtype, form,
                            target_snr_db, bits);
    if (v != TDG_OK) return v;
    if ((flags & TDG_NOISE_RMS) && (flags & TDG_NOISE_UNIFORM))
        return fail(TDG_EINVAL, "TDG_NOISE_RMS and TDG_NOISE_UNIFORM exclude each other");
    if (flags & TDG_PAIR_EXACT) {
        const bool tn = (transA == 'N' || transA == 'n') && (transB == 'N' || transB == 'n');
        if (form != TDG_SYM || !tn)
            return fail(TDG_EINVAL, "TDG_PAIR_EXACT needs the SYM form with transA = transB = 'N'");
        if (L != pair_exact_tile(dtype))
            return fail(TDG_EINVAL, "TDG_PAIR_EXACT needs L = %d for this dtype",
                        pair_exact_tile(dtype));
        const bool fixed = bits > 0;
        if (!(W == 2 || (fixed && W == 4)))
            return fail(TDG_EINVAL, "TDG_PAIR_EXACT packs W = 2, or W = 4 with fixed bits");
        if (flags & TDG_KEEP_PACKED)
            return fail(TDG_EINVAL, "TDG_PAIR_EXACT does not keep packed slab results");
    }
    tdgemm_plan_s *p = new tdgemm_plan_s();
    p->tA = (transA == 'T' || transA == 't') ? 'T' : 'N';
    p->tB = (transB == 'T' || transB == 't') ? 'T' : 'N';
    p->M = M; p->N = N; p->K = K; p->lda = lda; p->ldb = ldb; p->ldc = ldc;
    p->L = L; p->W = W; p->dtype = dtype; p->form = form; p->bits = bits;
    p->target = target_snr_db; p->flags = flags;
    p->mode = (form == TDG_PLAIN || form == TDG_TC_FP8) ? MODE_FIXED
              : (bits > 0 ? MODE_FIXED : MODE_TARGET);
    p->nM = cdiv_i(M, L); p->nK = cdiv_i(K, L); p->nN = cdiv_i(N, L);
    p->esz = dtype == TDG_F64 ? 8 : 4;
    cudaGetDevice(&p->device);

    // ---- workspace sizes
    const size_t al = 256;
    auto up = [&](size_t b) { return (b + al - 1) / al * al; };
    const size_t nAblk = (size_t)p->nM * p->nK, nBblk = (size_t)p->nK * p->nN;
    size_t off = 0;
    size_t o_plan = off; off += up(sizeof(DevPlan));
    size_t o_agg = off;
    off += up(((size_t)4 * p->nK + (size_t)kLevelRecDoubles * (kMaxW - 1) * kMaxLevels) * 8);
    size_t o_mA = off; off += up(nAblk * 8);
    size_t o_eA = off; off += up(nAblk * 8);
    size_t o_mB = off; off += up(nBblk * 8);
    size_t o_eB = off; off += up(nBblk * 8);
    size_t o_sA = off; off += up(nAblk * 8);
    size_t o_sB = off; off += up(nBblk * 8);
    size_t o_cA = off; off += up(nAblk * p->esz);
    size_t o_cB = off; off += up(nBblk * p->esz);
    size_t o_pair = off; off += up((size_t)p->nK * p->nM * p->nN * p->esz);
    size_t o_stab = off; off += up((size_t)(kMaxW - 1) * kMaxLevels * 8);
    const size_t npx = (flags & TDG_PAIR_EXACT) ? (size_t)p->nM * p->nK * p->nN : 0;
    size_t o_px = off; off += up(3 * npx * p->esz);      // c_A, c_B, pair factors per (i, l, j)
    size_t abytes = 0, bbytes = 0, rbytes = 0;
    if (is_tc_form(form)) {
        const long long ldk = round_up(K, 128);
        const size_t e1 = form == TDG_TC_FP8 ? 1 : 2;
        abytes = (size_t)M * ldk * e1;
        bbytes = (size_t)N * ldk * e1;
    } else {
        // slab splitting for few output tiles over many slabs (e.g. 288 x 288 x
        // 21600): the packed slab products of a tile run on several CTAs and
        // the ordered sum over slabs in the unpack kernel; needs the r-bar
        // buffer that TDG_KEEP_PACKED also uses
        if (is_packed_form(form) && !(flags & (TDG_KEEP_PACKED | TDG_PAIR_EXACT)) && p->nK >= 4) {
            int bxa, bxb, bk, dev = 0, sms = 0;
            packed_gemm_boxes(dtype, form == TDG_SYM ? G_SYM : G_ASYM, W, &bxa, &bxb, &bk);
            cudaGetDevice(&dev);
            cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
            const long long mrows = form == TDG_ASYM ? (long long)p->nM * Pof(L, W) : M;
            const long long ntiles = ((mrows + bxa - 1) / bxa) * ((N + bxb - 1) / bxb);
            if (sms > 0 && ntiles * 2 <= sms)
                p->split_groups = (int)std::min<long long>(p->nK, (2LL * sms + ntiles - 1) / ntiles);
        }
        for (int w : candidates(p)) {
            OpShape s = op_shape(p, w);
            abytes = std::max(abytes, (size_t)(s.a_rows * s.a_ld) * p->esz);
            bbytes = std::max(bbytes, (size_t)(s.b_rows * s.b_ld) * p->esz);
            if ((flags & TDG_KEEP_PACKED || p->split_groups > 1) && w >= 1 && is_packed_form(form)) {
                long long mrows = form == TDG_ASYM ? (long long)p->nM * Pof(L, w) : M;
                rbytes = std::max(rbytes, (size_t)((size_t)p->nK * (size_t)mrows * (size_t)N * p->esz));
            }
        }
    }
    if (p->split_groups > 1 && !(flags & TDG_KEEP_PACKED) && rbytes > ((size_t)1 << 30)) {
        p->split_groups = 1;       // the r-bar buffer would exceed 1 GiB
        rbytes = 0;
    }
    size_t o_A = off; off += up(abytes);
    size_t o_B = off; off += up(bbytes);
    size_t o_R = off; off += up(rbytes);
    p->ws_bytes = off;
    cudaError_t e = cudaMalloc(&p->ws, off);
    if (e != cudaSuccess) {
        delete p;
        return fail(e == cudaErrorMemoryAllocation ? TDG_ENOMEM : TDG_ECUDA,
                    "workspace of %zu bytes: %s", off, cudaGetErrorString(e));
    }
    e = cudaMemset(p->ws, 0, off);
    if (e != cudaSuccess) {
        cudaFree(p->ws);
        delete p;
        return fail(TDG_ECUDA, "cudaMemset: %s", cudaGetErrorString(e));
    }
    p->dplan = (DevPlan *)(p->ws + o_plan);
    p->agg = (double *)(p->ws + o_agg);
    p->mA = (double *)(p->ws + o_mA); p->eA = (double *)(p->ws + o_eA);
    p->mB = (double *)(p->ws + o_mB); p->eB = (double *)(p->ws + o_eB);
    p->sA = (double *)(p->ws + o_sA); p->sB = (double *)(p->ws + o_sB);
    p->cA = p->ws + o_cA; p->cB = p->ws + o_cB; p->pair = p->ws + o_pair;
    p->stab = (double *)(p->ws + o_stab);
    if (npx) {
        p->cApx = p->ws + o_px;
        p->cBpx = p->ws + o_px + npx * p->esz;
        p->pairpx = p->ws + o_px + 2 * npx * p->esz;
    }
    p->Abuf = p->ws + o_A; p->Bbuf = p->ws + o_B;
    p->Abuf_bytes = abytes; p->Bbuf_bytes = bbytes;
    p->Rbar = rbytes ? p->ws + o_R : nullptr;
    p->stab_host.assign((size_t)(kMaxW - 1) * kMaxLevels, -1.0);
    p->stab_dirty = true;
    *plan = p;
    return TDG_OK;
}

extern "C" tdg_status tdgemm_set_rep_noise(tdgemm_plan_t p, int W, const double *s, int t0,
                                           int n) {
    if (!p) return fail(TDG_EINVAL, "plan is NULL");
    if (W < 2 || W > kMaxW) return fail(TDG_EINVAL, "W must be in 2..4");
    if (!s || n < 0 || t0 < 0 || t0 + n > kMaxLevels)
        return fail(TDG_EINVAL, "levels must lie in [0, %d)", kMaxLevels);
    for (int i = 0; i < n; ++i) p->stab_host[(size_t)(W - 2) * kMaxLevels + t0 + i] = s[i];
    p->stab_dirty = true;
    p->have_table = true;
    return TDG_OK;
}

extern "C" tdg_status tdgemm_set_manual(tdgemm_plan_t p, int q, double c_a, double c_b) {
    if (!p) return fail(TDG_EINVAL, "plan is NULL");
    if (!is_packed_form(p->form)) return fail(TDG_EINVAL, "manual mode needs the SYM or ASYM form");
    if (q < 1 || q > 60) return fail(TDG_EINVAL, "q must be in 1..60");
    if (!(c_a > 0) || !(c_b > 0) || !isfinite(c_a) || !isfinite(c_b))
        return fail(TDG_EINVAL, "companders must be positive and finite");
    p->mode = MODE_MANUAL;
    p->manual_q = q;
    p->manual_cA = c_a;
    p->manual_cB = c_b;
    p->b_packed = false;   // B's companders changed
    return TDG_OK;
}

extern "C" tdg_status tdgemm_set_kernel_control(tdgemm_plan_t p, int mode, double value) {
    if (!p) return fail(TDG_EINVAL, "plan is NULL");
    if (mode == 0) { p->kctrl_mode = 0; p->packed = p->b_packed = false; return TDG_OK; }
    if (p->form != TDG_SYM) return fail(TDG_EINVAL, "inner-kernel control needs the SYM form");
    if (p->mode == MODE_MANUAL) return fail(TDG_EINVAL, "inner-kernel control needs a planned (not manual) plan");
    if (mode < 1 || mode > 3)
        return fail(TDG_EINVAL, "mode must be 0, 1 (SNR), 2 (fraction) or 3 (throughput)");
    if (p->flags & (TDG_KEEP_PACKED | TDG_PAIR_EXACT))
        return fail(TDG_EINVAL,
                    "inner-kernel control works without TDG_KEEP_PACKED and TDG_PAIR_EXACT");
    if (!isfinite(value)) return fail(TDG_EINVAL, "value must be finite");
    if (mode == 2 && (value < 0.0 || value > 1.0)) return fail(TDG_EINVAL, "fraction must be in [0, 1]");
    if (mode == 3) {
        if (value < 1.0) return fail(TDG_EINVAL, "throughput target must be >= 1 (x the conventional product)");
        // the device planner may choose any packing from W down to 2
        const int wlo = p->mode == MODE_TARGET ? 2 : p->W;
        for (int w = wlo; w <= p->W; ++w)
            if (!(p->speedup.fw[w] > 0.0))
                return fail(TDG_EINVAL, "throughput control needs F_W for W = %d (tdgemm_set_speedup)", w);
    }
    {
        // the mixed launch runs both kinds of tile with one box shape
        int sa, sb, sk, pa, pb, pk;
        packed_gemm_boxes(p->dtype, G_SYM, 2, &sa, &sb, &sk);
        packed_gemm_boxes(p->dtype, G_PLAIN, 1, &pa, &pb, &pk);
        if (sa != pa || sb != pb || sk != pk)
            return fail(TDG_EUNSUPPORTED, "packed and plain tiles differ for this dtype");
        if (p->L % sa || p->L % sb)
            return fail(TDG_EINVAL,
                        "inner-kernel control needs L to be a multiple of the %dx%d CTA tile",
                        sa, sb);
    }
    const long long T = (long long)p->nM * p->nN;
    if (T > 16384) return fail(TDG_EINVAL, "inner-kernel control supports up to 16384 inner kernels");
    if (!p->kratio) {
        int bm, bn, bk;
        packed_gemm_boxes(p->dtype, G_SYM, 2, &bm, &bn, &bk);
        p->ktiles_m = (p->M + bm - 1) / bm;
        p->ktiles_n = (p->N + bn - 1) / bn;
        CU_TRY(cudaMalloc(&p->kratio, (size_t)T * 8));
        CU_TRY(cudaMalloc(&p->kmask, (size_t)T));
        CU_TRY(cudaMemset(p->kmask, 0, (size_t)T));
        CU_TRY(cudaMalloc(&p->korder, (size_t)(p->ktiles_m * p->ktiles_n) * sizeof(int)));
    }
    if (!p->kA) {
        OpShape s = op_shape(p, 0);
        CU_TRY(cudaMalloc(&p->kA, (size_t)(s.a_rows * s.a_ld) * p->esz));
        CU_TRY(cudaMalloc(&p->kB, (size_t)(s.b_rows * s.b_ld) * p->esz));
    }
    p->kctrl_mode = mode;
    p->kctrl_value = value;
    p->kctrl_thr = mode == 1 ? pow(10.0, value / 10.0) : 0.0;
    p->kctrl_k = mode == 2 ? (long long)ceil(value * (double)T) : 0;
    p->packed = p->b_packed = false;   // the packed operands no longer match: pack again
    return TDG_OK;
}

extern "C" tdg_status tdgemm_set_speedup(tdgemm_plan_t p, int W, double speedup) {
    if (!p) return fail(TDG_EINVAL, "plan is NULL");
    if (W < 2 || W > kMaxW) return fail(TDG_EINVAL, "W must be in 2..4");
    if (!(speedup > 0.0) || !isfinite(speedup)) return fail(TDG_EINVAL, "F_W must be positive and finite");
    p->speedup.fw[W] = speedup;
    if (p->kctrl_mode == 3) p->packed = p->b_packed = false;   // the mask changes: pack again
    return TDG_OK;
}

extern "C" tdg_status tdgemm_set_wait_test(tdgemm_plan_t p, int64_t limit_ns) {
    if (!p) return fail(TDG_EINVAL, "plan is NULL");
    if (!(is_packed_form(p->form) || p->form == TDG_PLAIN) || (p->flags & TDG_PAIR_EXACT))
        return fail(TDG_EINVAL,
                    "the wait test covers the CUDA-core GEMM (PLAIN, SYM, ASYM without "
                    "TDG_PAIR_EXACT)");
    if (limit_ns < 0 || limit_ns > 1000000000LL)
        return fail(TDG_EINVAL, "limit_ns must be in [0, 1e9]");
    p->stall_ns = limit_ns;
    return TDG_OK;
}

extern "C" tdg_status tdgemm_kernel_mask(tdgemm_plan_t p, uint8_t *out, int64_t n) {
    if (!p || !out) return fail(TDG_EINVAL, "NULL argument");
    const long long T = (long long)p->nM * p->nN;
    if (!p->kctrl_mode || !p->kmask) return fail(TDG_ESTATE, "inner-kernel control is off");
    if (n < T) return fail(TDG_EINVAL, "output holds %lld bytes, need %lld", (long long)n, T);
    if (!p->packed) return fail(TDG_ESTATE, "kernel mask before tdgemm_quantize_pack");
    CU_TRY(cudaStreamSynchronize(p->last_stream));
    CU_TRY(cudaMemcpy(out, p->kmask, (size_t)T, cudaMemcpyDeviceToHost));
    return TDG_OK;
}

static PlanParams params_of(const tdgemm_plan_s *p) {
    PlanParams pp;
    pp.mode = p->mode; pp.form = p->form; pp.dtype = p->dtype;
    pp.L = p->L; pp.Wreq = p->W; pp.p = p->dtype == TDG_F64 ? 53 : 24;
    if (is_tc_form(p->form)) pp.p = 24;
    pp.bits = p->bits;
    pp.allow_fallback = (p->flags & TDG_ALLOW_FALLBACK) ? 1 : 0;
    pp.noise_rms = (p->flags & TDG_NOISE_UNIFORM) ? 0 : 1;
    pp.target_db = p->target;
    pp.manual_q = p->manual_q; pp.manual_cA = p->manual_cA; pp.manual_cB = p->manual_cB;
    pp.nM = p->nM; pp.nK = p->nK; pp.nN = p->nN;
    pp.M = p->M; pp.N = p->N; pp.K = p->K;
    pp.t0 = 0; pp.nt = kMaxLevels;
    return pp;
}

// op(A)[m][k] and op(B)[k][n] as (x, k) operands of the pack kernels
template <typename T>
static PackOperand<T> operand_A(const tdgemm_plan_s *p, const T *A, const T *c) {
    PackOperand<T> o;
    o.src = A; o.X = p->M; o.K = p->K; o.L = p->L;
    if (p->tA == 'N') { o.sx = p->lda; o.sk = 1; } else { o.sx = 1; o.sk = p->lda; }
    o.c = c; o.cx = p->nK; o.cl = 1;            // c_A[i][l]
    return o;
}
template <typename T>
static PackOperand<T> operand_B(const tdgemm_plan_s *p, const T *B, const T *c) {
    PackOperand<T> o;
    o.src = B; o.X = p->N; o.K = p->K; o.L = p->L;
    if (p->tB == 'N') { o.sx = 1; o.sk = p->ldb; } else { o.sx = p->ldb; o.sk = 1; }
    o.c = c; o.cx = 1; o.cl = p->nN;            // c_B[l][j]
    return o;
}

template <typename T>
static tdg_status pack_impl(tdgemm_plan_t p, const T *A, const T *B, cudaStream_t st,
                            bool reuse_b = false) {
    // reuse_b: B, its statistics, companders and packed copy are those of the
    // previous pack (the caller keeps B unchanged); only A is processed
    CU_TRY(cudaMemsetAsync(p->dplan, 0, sizeof(DevPlan), st));
    if (p->stab_dirty) {
        CU_TRY(cudaMemcpyAsync(p->stab, p->stab_host.data(), p->stab_host.size() * 8,
                               cudaMemcpyHostToDevice, st));
        p->stab_dirty = false;
    }
    const bool nA = p->tA == 'N', nB = p->tB == 'N';
    // tensor-core forms whose compander is gamma / max|x| of the block alone:
    // statistics, companders and codes in one pass over each input
    const bool tc_fused = is_tc_form(p->form) && p->mode == MODE_FIXED && p->L <= 128 &&
                          p->L % 64 == 0;
    if (tc_fused) {
        if constexpr (sizeof(T) == 4) {
            const long long ldk = round_up(p->K, 128);
            const int fp8 = p->form == TDG_TC_FP8;
            const double gamma = fp8 ? kFp8Max : (double)((1 << (p->bits - 1)) - 1);
            PackOperand<float> oa = operand_A<float>(p, A, nullptr);
            PackOperand<float> ob = operand_B<float>(p, B, nullptr);
            CU_TRY(launch_codes_stats(oa, p->mA, p->eA, (float *)p->cA, p->sA, p->Abuf,
                                      reuse_b ? nullptr : &ob, p->mB, p->eB, (float *)p->cB,
                                      p->sB, p->Bbuf, fp8, gamma, ldk, p->dplan, st));
        }
    } else if (p->form != TDG_PLAIN && p->mode != MODE_MANUAL) {
        // stats of op(A): stored rows x cols; op block grid nM x nK
        CU_TRY(launch_block_stats<T>(A, nA ? p->M : p->K, nA ? p->K : p->M, p->lda, nA ? 0 : 1,
                                     p->nK, p->mA, p->eA, B, reuse_b ? 0 : (nB ? p->K : p->N),
                                     nB ? p->N : p->K, p->ldb, nB ? 0 : 1, p->nN, p->mB, p->eB,
                                     p->L, p->dplan, st));
    }
    PlanParams pp = params_of(p);
    const double *stab = p->have_table ? p->stab : nullptr;
    CU_TRY(launch_planner<T>(pp, p->mA, p->eA, p->mB, p->eB, stab, p->dplan, p->agg, (T *)p->cA,
                             p->sA, (T *)p->cB, p->sB, (T *)p->pair, st, tc_fused));
    const bool px = (p->flags & TDG_PAIR_EXACT) != 0;
    if (px)
        CU_TRY(launch_px_scales<T>(pp, p->mA, p->eA, p->mB, p->eB, p->dplan, (T *)p->cApx,
                                   (T *)p->cBpx, (T *)p->pairpx, st));
    if (p->kctrl_mode) {
        CU_TRY(launch_kernel_control(pp, p->mA, p->eA, p->mB, p->eB, p->dplan, p->kctrl_mode,
                                     p->kctrl_thr, p->kctrl_k, p->kctrl_value, p->speedup,
                                     p->kratio, p->kmask, st));
        {
            int bm, bn, bk;
            packed_gemm_boxes(p->dtype, G_SYM, 2, &bm, &bn, &bk);
            CU_TRY(launch_tile_order(p->kmask, p->nN, p->L, bm, bn, p->ktiles_m, p->ktiles_n,
                                     p->korder, st));
        }
        OpShape s0 = op_shape(p, 0);
        const bool directA = !nA && (p->lda * (long long)sizeof(T)) % 16 == 0 && ((uintptr_t)A & 15) == 0;
        const bool directB = nB && (p->ldb * (long long)sizeof(T)) % 16 == 0 && ((uintptr_t)B & 15) == 0;
        if (!directA)
            CU_TRY(launch_pack_k<T>(operand_A<T>(p, A, nullptr), 1, p->dplan, 0, 0, (T *)p->kA,
                                    s0.a_ld, s0.a_rows, st));
        if (!directB && !reuse_b)
            CU_TRY(launch_pack_k<T>(operand_B<T>(p, B, nullptr), 1, p->dplan, 0, 0, (T *)p->kB,
                                    s0.b_ld, s0.b_rows, st));
    }
    if (is_tc_form(p->form)) {
        if constexpr (sizeof(T) == 4) {
            if (!tc_fused) {       // (the fused path wrote the codes with the statistics)
                const long long ldk = round_up(p->K, 128);
                const int fp8 = p->form == TDG_TC_FP8;
                // B first, as for the packs: its blocks were read last
                if (!reuse_b)
                    CU_TRY(launch_codes(operand_B<float>(p, B, (const float *)p->cB), fp8,
                                        p->Bbuf, ldk, st));
                CU_TRY(launch_codes(operand_A<float>(p, A, (const float *)p->cA), fp8, p->Abuf,
                                    ldk, st));
            }
        }
    } else {
        for (int w : candidates(p)) {
            OpShape s = op_shape(p, w);
            if (w == 0 || p->form == TDG_PLAIN) {
                // plain product: k-major copies unless the caller's layout already is
                const bool directA = !nA && (p->lda * (long long)sizeof(T)) % 16 == 0 &&
                                     ((uintptr_t)A & 15) == 0;
                const bool directB = nB && (p->ldb * (long long)sizeof(T)) % 16 == 0 &&
                                     ((uintptr_t)B & 15) == 0;
                if (!directA)
                    CU_TRY(launch_pack_k<T>(operand_A<T>(p, A, nullptr), 1, p->dplan, 1, 0,
                                            (T *)p->Abuf, s.a_ld, s.a_rows, st));
                if (!directB && !reuse_b)
                    CU_TRY(launch_pack_k<T>(operand_B<T>(p, B, nullptr), 1, p->dplan, 1, 0,
                                            (T *)p->Bbuf, s.b_ld, s.b_rows, st));
            } else if (px) {
                // each CTA compands and packs its own tiles from A and B
            } else if (p->form == TDG_SYM) {
                if (!reuse_b)
                    CU_TRY(launch_pack_k_pair<T>(operand_A<T>(p, A, (const T *)p->cA),
                                                 operand_B<T>(p, B, (const T *)p->cB), w,
                                                 p->dplan, w, (T *)p->Abuf, s.a_ld, s.a_rows,
                                                 (T *)p->Bbuf, s.b_ld, s.b_rows, st));   // eqs. 6, 7
                else
                    CU_TRY(launch_pack_k<T>(operand_A<T>(p, A, (const T *)p->cA), w, p->dplan, w,
                                            -1, (T *)p->Abuf, s.a_ld, s.a_rows, st));   // eq. 6
            } else {
                if (!reuse_b)
                    CU_TRY(launch_pack_k<T>(operand_B<T>(p, B, (const T *)p->cB), 1, p->dplan, w,
                                            0, (T *)p->Bbuf, s.b_ld, s.b_rows, st));       // b~ only
                CU_TRY(launch_pack_x<T>(operand_A<T>(p, A, (const T *)p->cA), w, p->dplan, w, -1,
                                        (T *)p->Abuf, s.a_ld, st));                   // eq. 11
            }
        }
    }
    p->A_user = A;
    p->B_user = B;
    p->packed = true;
    p->gemm_done = false;
    p->last_stream = st;
    return TDG_OK;
}

extern "C" tdg_status tdgemm_quantize_pack(tdgemm_plan_t p, const void *A, const void *B,
                                           void *stream) {
    if (!p) return fail(TDG_EINVAL, "plan is NULL");
    if (!A || !B) return fail(TDG_EINVAL, "A and B must be device pointers");
    cudaStream_t st = (cudaStream_t)stream;
    tdg_status r = p->dtype == TDG_F64
                       ? pack_impl<double>(p, (const double *)A, (const double *)B, st)
                       : pack_impl<float>(p, (const float *)A, (const float *)B, st);
    if (r == TDG_OK) p->b_packed = true;
    return r;
}

extern "C" tdg_status tdgemm_quantize_pack_a(tdgemm_plan_t p, const void *A, void *stream) {
    if (!p) return fail(TDG_EINVAL, "plan is NULL");
    if (!A) return fail(TDG_EINVAL, "A must be a device pointer");
    if (!(p->mode == MODE_FIXED || p->mode == MODE_MANUAL || p->form == TDG_PLAIN ||
          p->form == TDG_TC_FP8))
        return fail(TDG_EINVAL,
                    "B can be reused only when its companders do not depend on A (fixed bits, "
                    "manual parameters, the plain or the E4M3 form)");
    if (!p->b_packed || !p->B_user)
        return fail(TDG_ESTATE, "tdgemm_quantize_pack_a before a tdgemm_quantize_pack with B");
    cudaStream_t st = (cudaStream_t)stream;
    if (p->dtype == TDG_F64)
        return pack_impl<double>(p, (const double *)A, (const double *)p->B_user, st, true);
    return pack_impl<float>(p, (const float *)A, (const float *)p->B_user, st, true);
}

template <typename T>
static tdg_status gemm_impl(tdgemm_plan_t p, T *C, double alpha, double beta, cudaStream_t st) {
    // the plain k-major operands: the caller's buffers where their layout and
    // alignment already fit, else the copies the pack step made
    auto plain_ops = [&](const void *abuf, const void *bbuf, GemmOperand &a, GemmOperand &b) {
        OpShape s = op_shape(p, 0);
        a = {abuf, s.a_cols, s.a_rows, s.a_ld};
        b = {bbuf, s.b_cols, s.b_rows, s.b_ld};
        if (p->tA != 'N' && (p->lda * (long long)sizeof(T)) % 16 == 0 &&
            ((uintptr_t)p->A_user & 15) == 0)
            a = {p->A_user, s.a_cols, s.a_rows, p->lda};
        if (p->tB == 'N' && (p->ldb * (long long)sizeof(T)) % 16 == 0 &&
            ((uintptr_t)p->B_user & 15) == 0)
            b = {p->B_user, s.b_cols, s.b_rows, p->ldb};
    };
    for (int w : candidates(p)) {
        const bool plain = (w == 0 || p->form == TDG_PLAIN);
        const int gform = plain ? G_PLAIN : (p->form == TDG_SYM ? G_SYM : G_ASYM);
        const int Wk = plain ? 1 : w;
        OpShape s = op_shape(p, w);
        GemmOperands ops{};
        if (plain) {
            plain_ops(p->Abuf, p->Bbuf, ops.a, ops.b);
        } else {
            ops.a = {p->Abuf, s.a_cols, s.a_rows, s.a_ld};
            ops.b = {p->Bbuf, s.b_cols, s.b_rows, s.b_ld};
        }
        GemmArgs<T> g{};
        g.plan = p->dplan;
        g.M = p->M; g.N = p->N; g.K = p->K;
        g.Mrows = s.a_cols;
        g.Krows = s.a_rows;
        g.L = p->L; g.P = plain ? p->L : Pof(p->L, Wk);
        g.nM = p->nM; g.nK = p->nK; g.nN = p->nN;
        g.pair = (const T *)p->pair;
        g.C = C; g.ldc = p->ldc;
        g.alpha = (T)alpha; g.beta = (T)beta; g.beta_zero = beta == 0.0;
        g.Rbar = (!plain && (p->flags & TDG_KEEP_PACKED)) ? (T *)p->Rbar : nullptr;
        g.stall_ns = p->stall_ns;
        if (p->mode == MODE_FIXED) {
            const long long gam = (1LL << (p->bits - 1)) - 1;
            g.small_t = small_round_ok(gform, Wk, q_for((long long)p->L * gam * gam), (int)gam) ? 1 : 0;
        } else {
            g.small_t = p->mode == MODE_MANUAL ? 0 : -1;
        }
        const bool split = !plain && p->split_groups > 1 && !p->kctrl_mode && p->Rbar;
        if (split) {
            g.Rbar = (T *)p->Rbar;
            g.groups = p->split_groups;
        }
        if (p->kctrl_mode && !plain) {
            // Sec. 6: the tiles of inner kernels left unaccelerated compute the
            // conventional product from the plain operands, same launch
            plain_ops(p->kA, p->kB, ops.pa, ops.pb);
            g.kmask = p->kmask;
            g.tile_order = p->korder;
        }
        cudaError_t e;
        if (!plain && (p->flags & TDG_PAIR_EXACT)) {
            GemmOperands raw{};
            raw.a = {p->A_user, p->K, p->M, p->lda};      // op(A) row-major [M][K]
            raw.b = {p->B_user, p->N, p->K, p->ldb};      // op(B) row-major [K][N]
            g.pair = (const T *)p->pairpx;
            g.cApx = (const T *)p->cApx;
            g.cBpx = (const T *)p->cBpx;
            g.P = p->L / Wk;
            e = launch_px_gemm<T>(Wk, g, raw, st);
        } else {
            e = launch_packed_gemm<T>(gform, Wk, g, ops, st);
        }
        if (e == cudaErrorInvalidValue)
            return fail(TDG_ECUDA, "packed GEMM: an operand could not be mapped for TMA");
        if (e != cudaSuccess)
            return fail(TDG_ECUDA, "packed GEMM launch failed: %s", cudaGetErrorString(e));
        if (split) CU_TRY(launch_unpack<T>(gform, Wk, g, nullptr, st));   // sum over slabs, C
    }
    return TDG_OK;
}

extern "C" tdg_status tdgemm_gemm(tdgemm_plan_t p, void *C, double alpha, double beta,
                                  void *stream) {
    if (!p) return fail(TDG_EINVAL, "plan is NULL");
    if (!C) return fail(TDG_EINVAL, "C is NULL");
    if (!p->packed) return fail(TDG_ESTATE, "tdgemm_gemm before tdgemm_quantize_pack");
    if (!isfinite(alpha) || !isfinite(beta)) return fail(TDG_EINVAL, "alpha/beta not finite");
    cudaStream_t st = (cudaStream_t)stream;
    tdg_status r;
    if (is_tc_form(p->form)) {
        const int fp8 = p->form == TDG_TC_FP8;
        int bra, brb, bk;
        tc_gemm_boxes(fp8, &bra, &brb, &bk);
        const long long ldk = round_up(p->K, 128);
        const CUtensorMapDataType dt =
            fp8 ? CU_TENSOR_MAP_DATA_TYPE_UINT8 : CU_TENSOR_MAP_DATA_TYPE_FLOAT16;
        const size_t e1 = fp8 ? 1 : 2;
        CUtensorMap ma, mb;
        r = make_map(&ma, dt, e1, p->Abuf, p->K, p->M, ldk, bk, bra, CU_TENSOR_MAP_SWIZZLE_128B);
        if (r != TDG_OK) return r;
        r = make_map(&mb, dt, e1, p->Bbuf, p->K, p->N, ldk, bk, brb, CU_TENSOR_MAP_SWIZZLE_128B);
        if (r != TDG_OK) return r;
        TcArgs a;
        a.plan = p->dplan; a.M = p->M; a.N = p->N; a.K = p->K;
        a.L = p->L; a.nM = p->nM; a.nK = p->nK; a.nN = p->nN;
        a.pair = (const float *)p->pair; a.C = (float *)C; a.ldc = p->ldc;
        a.alpha = (float)alpha; a.beta = (float)beta; a.beta_zero = beta == 0.0;
        // C through TMA stores where it can be mapped (beta = 0 and 16-byte
        // aligned rows), else through plain stores
        CUtensorMap mc;
        memset(&mc, 0, sizeof(mc));
        a.c_tma = 0;
        if (beta == 0.0 && ((uintptr_t)C & 15) == 0 && ((p->ldc * 4) & 15) == 0) {
            int cbx, cby;
            tc_gemm_c_box(&cbx, &cby);
            a.c_tma = encode_map_2d(&mc, CU_TENSOR_MAP_DATA_TYPE_FLOAT32, 4, C, p->N, p->M, p->ldc,
                                    cbx, cby, CU_TENSOR_MAP_SWIZZLE_64B) == CUDA_SUCCESS;
        }
        cudaError_t e = launch_tc_gemm(fp8, a, ma, mb, mc, st);
        if (e == cudaErrorNotSupported) return fail(TDG_EUNSUPPORTED, "tensor-core GEMM not built");
        CU_TRY(e);
        r = TDG_OK;
    } else if (p->dtype == TDG_F64) {
        r = gemm_impl<double>(p, (double *)C, alpha, beta, st);
    } else {
        r = gemm_impl<float>(p, (float *)C, alpha, beta, st);
    }
    if (r == TDG_OK) { p->gemm_done = true; p->last_stream = st; }
    return r;
}

extern "C" tdg_status tdgemm_run(tdgemm_plan_t p, const void *A, const void *B, void *C,
                                 double alpha, double beta, void *stream) {
    tdg_status r = tdgemm_quantize_pack(p, A, B, stream);
    if (r != TDG_OK) return r;
    return tdgemm_gemm(p, C, alpha, beta, stream);
}

extern "C" tdg_status tdgemm_run_host(tdgemm_plan_t p, const void *A, const void *B, void *C,
                                      double alpha, double beta, void *stream) {
    if (!p) return fail(TDG_EINVAL, "plan is NULL");
    if (!A || !B || !C) return fail(TDG_EINVAL, "A, B and C must be host pointers");
    cudaStream_t st = (cudaStream_t)stream;
    const size_t esz = p->esz;
    const size_t abytes = (size_t)((p->tA == 'N') ? p->M : p->K) * p->lda * esz;
    const size_t bbytes = (size_t)((p->tB == 'N') ? p->K : p->N) * p->ldb * esz;
    const size_t cbytes = (size_t)p->M * p->ldc * esz;
    if (!p->hA) {
        CU_TRY(cudaMalloc(&p->hA, abytes));
        CU_TRY(cudaMalloc(&p->hB, bbytes));
        CU_TRY(cudaMalloc(&p->hC, cbytes));
    }
    // C written by the GEMM's epilogue straight into host memory the device
    // can address (pinned), in place of a copy back: where the CUDA-core
    // packed GEMM kernel writes C (whole row segments per warp) and does not
    // read it (beta = 0)
    void *c_direct = nullptr;
    if (beta == 0.0 && (is_packed_form(p->form) || p->form == TDG_PLAIN) &&
        p->split_groups <= 1 && !(p->flags & TDG_PAIR_EXACT)) {
        cudaPointerAttributes at{};
        if (cudaPointerGetAttributes(&at, C) == cudaSuccess) {
            if (at.type == cudaMemoryTypeHost && at.devicePointer) c_direct = at.devicePointer;
        } else {
            (void)cudaGetLastError();
        }
    }
    CU_TRY(cudaMemcpyAsync(p->hA, A, abytes, cudaMemcpyHostToDevice, st));
    CU_TRY(cudaMemcpyAsync(p->hB, B, bbytes, cudaMemcpyHostToDevice, st));
    if (beta != 0.0) CU_TRY(cudaMemcpyAsync(p->hC, C, cbytes, cudaMemcpyHostToDevice, st));
    tdg_status r = tdgemm_run(p, p->hA, p->hB, c_direct ? c_direct : p->hC, alpha, beta, stream);
    if (r != TDG_OK) {
        // the copies already queued read the caller's buffers: let them finish
        // before the caller may reuse them
        cudaStreamSynchronize(st);
        return r;
    }
    if (!c_direct) CU_TRY(cudaMemcpyAsync(C, p->hC, cbytes, cudaMemcpyDeviceToHost, st));
    CU_TRY(cudaStreamSynchronize(st));
    return TDG_OK;
}

// pinned host memory (registered or allocated page-locked): its device alias, else nullptr
static void *pinned_alias(const void *h) {
    cudaPointerAttributes at{};
    if (cudaPointerGetAttributes(&at, h) != cudaSuccess) {
        (void)cudaGetLastError();
        return nullptr;
    }
    return at.type == cudaMemoryTypeHost ? at.devicePointer : nullptr;
}

extern "C" tdg_status tdgemm_run_host_async(tdgemm_plan_t p, const void *A, const void *B, void *C,
                                            double alpha, double beta, void *stream) {
    if (!p) return fail(TDG_EINVAL, "plan is NULL");
    if (!A || !B || !C) return fail(TDG_EINVAL, "A, B and C must be host pointers");
    void *c_alias = pinned_alias(C);
    if (!pinned_alias(A) || !pinned_alias(B) || !c_alias)
        return fail(TDG_EINVAL, "tdgemm_run_host_async needs pinned host memory for A, B and C");
    cudaStream_t st = (cudaStream_t)stream;
    const size_t esz = p->esz;
    const size_t abytes = (size_t)((p->tA == 'N') ? p->M : p->K) * p->lda * esz;
    const size_t bbytes = (size_t)((p->tB == 'N') ? p->K : p->N) * p->ldb * esz;
    const size_t cbytes = (size_t)p->M * p->ldc * esz;
    if (!p->copy_stream) {
        CU_TRY(cudaStreamCreateWithFlags(&p->copy_stream, cudaStreamNonBlocking));
        for (auto &h : p->hset) {
            CU_TRY(cudaMalloc(&h.A, abytes));
            CU_TRY(cudaMalloc(&h.B, bbytes));
            CU_TRY(cudaMalloc(&h.C, cbytes));
            CU_TRY(cudaEventCreateWithFlags(&h.copied, cudaEventDisableTiming));
            CU_TRY(cudaEventCreateWithFlags(&h.done, cudaEventDisableTiming));
        }
    }
    // C in place over the CPU-GPU link where tdgemm_run_host writes it so
    const bool c_direct = beta == 0.0 && (is_packed_form(p->form) || p->form == TDG_PLAIN) &&
                          p->split_groups <= 1 && !(p->flags & TDG_PAIR_EXACT);
    auto &h = p->hset[p->next_set];
    p->next_set ^= 1;
    // the set is free once the computation queued on it before has run
    if (h.used) CU_TRY(cudaStreamWaitEvent(p->copy_stream, h.done, 0));
    CU_TRY(cudaMemcpyAsync(h.A, A, abytes, cudaMemcpyHostToDevice, p->copy_stream));
    CU_TRY(cudaMemcpyAsync(h.B, B, bbytes, cudaMemcpyHostToDevice, p->copy_stream));
    if (beta != 0.0) CU_TRY(cudaMemcpyAsync(h.C, C, cbytes, cudaMemcpyHostToDevice, p->copy_stream));
    CU_TRY(cudaEventRecord(h.copied, p->copy_stream));
    CU_TRY(cudaStreamWaitEvent(st, h.copied, 0));
    tdg_status r = tdgemm_run(p, h.A, h.B, c_direct ? c_alias : h.C, alpha, beta, stream);
    if (r != TDG_OK) {
        // the copies already queued read the caller's buffers: let them finish
        cudaStreamSynchronize(p->copy_stream);
        return r;
    }
    if (!c_direct) CU_TRY(cudaMemcpyAsync(C, h.C, cbytes, cudaMemcpyDeviceToHost, st));
    CU_TRY(cudaEventRecord(h.done, st));
    h.used = true;
    return TDG_OK;
}

extern "C" tdg_status tdgemm_unpack(tdgemm_plan_t p, int64_t *rint_out, void *C, void *stream) {
    if (!p) return fail(TDG_EINVAL, "plan is NULL");
    if (!is_packed_form(p->form)) return fail(TDG_EINVAL, "unpack needs the SYM or ASYM form");
    if (!(p->flags & TDG_KEEP_PACKED) || !p->Rbar)
        return fail(TDG_ESTATE, "unpack needs a plan made with TDG_KEEP_PACKED");
    if (!p->gemm_done) return fail(TDG_ESTATE, "unpack before tdgemm_gemm");
    if (p->mode == MODE_TARGET)
        return fail(TDG_EINVAL, "unpack supports fixed-bit and manual plans");
    cudaStream_t st = (cudaStream_t)stream;
    const int w = p->W;
    OpShape s = op_shape(p, w);
    const int gform = p->form == TDG_SYM ? G_SYM : G_ASYM;
    if (p->dtype == TDG_F64) {
        GemmArgs<double> g{};
        g.plan = p->dplan; g.M = p->M; g.N = p->N; g.K = p->K; g.Mrows = s.a_cols;
        g.Krows = s.a_rows; g.L = p->L; g.P = Pof(p->L, w); g.nM = p->nM; g.nK = p->nK;
        g.nN = p->nN; g.pair = (const double *)p->pair; g.C = (double *)C; g.ldc = p->ldc;
        g.Rbar = (double *)p->Rbar;
        g.alpha = 1.0; g.beta_zero = 1;           // C = sum over slabs, as it stands
        CU_TRY(launch_unpack<double>(gform, w, g, rint_out, st));
    } else {
        GemmArgs<float> g{};
        g.plan = p->dplan; g.M = p->M; g.N = p->N; g.K = p->K; g.Mrows = s.a_cols;
        g.Krows = s.a_rows; g.L = p->L; g.P = Pof(p->L, w); g.nM = p->nM; g.nK = p->nK;
        g.nN = p->nN; g.pair = (const float *)p->pair; g.C = (float *)C; g.ldc = p->ldc;
        g.Rbar = (float *)p->Rbar;
        g.alpha = 1.0f; g.beta_zero = 1;          // C = sum over slabs, as it stands
        CU_TRY(launch_unpack<float>(gform, w, g, rint_out, st));
    }
    return TDG_OK;
}

extern "C" tdg_status tdgemm_plan_info(tdgemm_plan_t p, tdgemm_info *out) {
    if (!p || !out) return fail(TDG_EINVAL, "NULL argument");
    if (!p->packed) return fail(TDG_ESTATE, "plan_info before tdgemm_quantize_pack");
    CU_TRY(cudaStreamSynchronize(p->last_stream));
    DevPlan a;
    CU_TRY(cudaMemcpy(&a, p->dplan, sizeof(DevPlan), cudaMemcpyDeviceToHost));
    out->W_used = a.W;
    out->q = a.q;
    out->gamma_a = a.gA;
    out->gamma_b = a.gB;
    out->r_max = a.R;
    out->w_ef = a.Wef;
    out->level = a.level;
    out->pred_snr_db = a.pred_snr;
    out->workspace_bytes = (int64_t)p->ws_bytes;
    out->device_status = a.status ? a.status : (a.nonfinite ? TDG_ENONFINITE : 0);
    out->carrier = p->form == TDG_TC_FP8 ? 8 : (p->form == TDG_TC_INT ? 16 : 0);
    return TDG_OK;
}

extern "C" tdg_status tdgemm_plan_destroy(tdgemm_plan_t p) {
    if (!p) return TDG_OK;
    cudaDeviceSynchronize();
    cudaFree(p->ws);
    if (p->hA) cudaFree(p->hA);
    if (p->hB) cudaFree(p->hB);
    if (p->hC) cudaFree(p->hC);
    for (auto &h : p->hset) {
        if (h.A) cudaFree(h.A);
        if (h.B) cudaFree(h.B);
        if (h.C) cudaFree(h.C);
        if (h.copied) cudaEventDestroy(h.copied);
        if (h.done) cudaEventDestroy(h.done);
    }
    if (p->copy_stream) cudaStreamDestroy(p->copy_stream);
    if (p->kA) cudaFree(p->kA);
    if (p->kB) cudaFree(p->kB);
    if (p->kratio) cudaFree(p->kratio);
    if (p->kmask) cudaFree(p->kmask);
    if (p->korder) cudaFree(p->korder);
    delete p;
    return TDG_OK;
}

extern "C" tdg_status tdgemm_snr(const void *C, int64_t ldc, tdg_dtype dtype, const double *ref,
                                 int64_t ldr, int64_t M, int64_t N, double *out3, void *stream) {
    if (!C || !ref || !out3) return fail(TDG_EINVAL, "NULL pointer");
    if (M < 1 || N < 1 || ldc < N || ldr < N) return fail(TDG_EINVAL, "bad shape");
    if (dtype != TDG_F32 && dtype != TDG_F64) return fail(TDG_EINVAL, "bad dtype");
    CU_TRY(launch_snr(C, ldc, dtype, ref, ldr, M, N, out3, (cudaStream_t)stream));
    return TDG_OK;
}

extern "C" const char *tdgemm_last_error(void) { return g_err; }

extern "C" const char *tdgemm_version(void) { return "tdgemm 0.1 (sm_103a)"; }
