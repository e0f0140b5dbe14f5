// Shared device-side definitions of the tdgemm CUDA library (sm_103a).
#pragma once

#include <cuda.h>
#include <cuda_runtime.h>
#include <stdint.h>

#include "tdgemm.h"

namespace tdg {

constexpr int kUSafe = 50;             // Prop. 1: u_safe = 50
constexpr int kMaxW = 4;               // packings built: W in 1..4
constexpr int kMaxLevels = 192;        // R_max candidate levels t in [0, 192)
constexpr int kLevelRecDoubles = 6;    // workspace per planner candidate (W, level)
constexpr double kTcIntExact = 16777215.0;  // per-slab |sum| that fp32 holds exactly
constexpr int kTcIntMaxGamma = 2048;        // integers exactly representable in fp16
constexpr double kFp8Max = 448.0;           // largest finite E4M3 value

enum Mode { MODE_FIXED = 0, MODE_TARGET = 1, MODE_MANUAL = 2 };

// What the planner decided; written by the planner kernel in device memory,
// read by every later kernel of the same plan (no host round trip).
struct DevPlan {
    int W;             // packing used (1 = plain product)
    int q;             // z = 2^-q
    int gA, gB;        // integer companders (gamma)
    long long R;       // L * gA * gB
    int Wef;           // eq. 16
    int level;         // chosen R_max level (target mode), -1 otherwise
    int status;        // tdg_status raised on the device (0 = ok)
    int nonfinite;     // set by the statistics kernel
    double pred_snr;   // model SNR (dB), NaN if not modelled
    double s_rep;      // representation-noise RMSE the model used (0 if none)
    double S, T1, T2, T3;  // noise-model aggregates
    unsigned int levels_done;  // candidate-level CTAs finished (the last one decides)
    // planner inputs, written by the last per-slab aggregate CTA before the
    // decision: the slab sums S, T1, T2, T3 (unscaled) and rho = sqrt(T2 / T1)
    unsigned int aggs_done;
    double tS, tT1, tT2, tT3, trho;
};

// Per-slab aggregates X_l = sum_i sigma_A,il^2, MA_l = sum_i m_A,il^2,
// Y_l = sum_j sigma_B,lj^2, MB_l = sum_j m_B,lj^2 of slab l, written to
// agg[4 l .. 4 l + 3] by one warp: lanes over i (j), then a fixed xor tree.
__device__ inline void slab_aggregate_warp(int l, int nM, int nK, int nN,
                                           const double *mA, const double *vA,
                                           const double *mB, const double *vB, double *agg) {
    const int lane = threadIdx.x & 31;
    double X = 0, MA = 0, Y = 0, MB = 0;
    for (int i = lane; i < nM; i += 32) {
        X += vA[(long long)i * nK + l];
        const double m = mA[(long long)i * nK + l];
        MA += m * m;
    }
    for (int j = lane; j < nN; j += 32) {
        Y += vB[(long long)l * nN + j];
        const double m = mB[(long long)l * nN + j];
        MB += m * m;
    }
#pragma unroll
    for (int off = 16; off > 0; off >>= 1) {
        X += __shfl_xor_sync(0xffffffffu, X, off);
        MA += __shfl_xor_sync(0xffffffffu, MA, off);
        Y += __shfl_xor_sync(0xffffffffu, Y, off);
        MB += __shfl_xor_sync(0xffffffffu, MB, off);
    }
    if (lane == 0) {
        agg[4 * (long long)l + 0] = X;
        agg[4 * (long long)l + 1] = MA;
        agg[4 * (long long)l + 2] = Y;
        agg[4 * (long long)l + 3] = MB;
    }
}


// Planner inputs that do not change between calls.
struct PlanParams {
    int mode;          // Mode
    int form;          // tdg_form
    int dtype;         // tdg_dtype
    int L, Wreq;
    int p;             // mantissa bits of T (24 / 53): u_sys = 2^-p
    int bits;          // fixed-bit mode
    int allow_fallback;
    int noise_rms;     // representation noise scaled by crest factors
    double target_db;
    int manual_q;
    double manual_cA, manual_cB;
    int nM, nK, nN;    // block counts
    long long M, N, K;
    int t0, nt;        // rep-noise table levels [t0, t0 + nt)
};

// ---------------------------------------------------------------------------
// small integer helpers shared by planner kernels
// ---------------------------------------------------------------------------
__host__ __device__ inline int cdiv_i(long long a, long long b) { return (int)((a + b - 1) / b); }

// R_max level t: floor(2^(t div 4) * (4 + t mod 4) / 4)
__host__ __device__ inline long long r_level(int t) {
    return ((long long)(4 + (t & 3)) << (t >> 2)) >> 2;
}

// number of bits of a positive integer
__host__ __device__ inline int bit_length(unsigned long long v) {
#ifdef __CUDA_ARCH__
    return v ? 64 - __clzll((long long)v) : 0;
#else
    return v ? 64 - __builtin_clzll(v) : 0;
#endif
}

// eq. 15: smallest q with 2^q >= 2 R + u_safe
__host__ __device__ inline int q_for(long long R) {
    return bit_length((unsigned long long)(2 * R + kUSafe - 1));
}

// eq. 16 in integers: W_ef = 1 + floor((p - bitlen(2R + 1)) / q); for R >= 1
// 2R + 1 is odd and above 1, so log2(2R + 1) lies strictly inside
// (bitlen - 1, bitlen) and the floor equals that of the logarithmic form.
__host__ __device__ inline int w_ef(long long R, int q, int p) {
    int b = bit_length((unsigned long long)(2 * R + 1));
    int num = p - b;
    int fl = num >= 0 ? num / q : -((-num + q - 1) / q);
    return 1 + fl;
}

// Roundings of the unpack that may use the add-subtract form, exact for
// |x| < 2^22, with planned companders (|a~| <= gamma_A, |b~| <= gamma_B; manual
// companders bound nothing and leave gamma 0 in the plan) and q <= 22, so
// R_max < Q / 2 <= 2^21:
//   symmetric, W = 2: the second rounding t = rint(z u) of eq. 10, since
//     z u = S_01 + (R + z S_10 + e) / Q with |S_01| <= R_max and the rest below
//     2 in magnitude (for W > 2, z u carries powers of Q);
//   asymmetric, any W: every rounding of eqs. 13-14, since r-bar =
//     sum_i z^i R_i with |R_i| <= R_max, and each peeled remainder
//     Q (r-bar_i - r~_i) is again such a sum (errors beyond the error-free
//     region stay below Q / 2).
__host__ __device__ inline bool small_round_ok(int form, int W, int q, int gA) {
    if (q > 22 || gA <= 0) return false;
    if (form == 1) return W == 2;       // symmetric (G_SYM)
    return form == 2;                   // asymmetric (G_ASYM)
}

// integer compander split of eq. 26 for a budget R: gA = floor(sqrt((R/L) rho))
__device__ inline void split_gammas(long long R, int L, double rho, int &gA, int &gB) {
    long long G = R / L;
    if (G < 1) { gA = gB = 0; return; }
    double v = __dsqrt_rn(__dmul_rn(__ddiv_rn((double)R, (double)L), rho));
    long long a = (long long)floor(v);
    if (a < 1) a = 1;
    if (a > G) a = G;
    long long b = R / ((long long)L * a);
    if (b < 1) b = 1;
    gA = (int)min(a, (long long)INT32_MAX);
    gB = (int)min(b, (long long)INT32_MAX);
}

// ---------------------------------------------------------------------------
// PTX helpers: shared-memory addresses, mbarriers, TMA
// ---------------------------------------------------------------------------
__device__ inline uint32_t smem_u32(const void *p) {
    return (uint32_t)__cvta_generic_to_shared(p);
}

__device__ inline void mbar_init(uint64_t *bar, uint32_t count) {
    asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_u32(bar)), "r"(count)
                 : "memory");
}

__device__ inline void fence_barrier_init() {
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
}

__device__ inline void fence_proxy_async() {
    asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
}

__device__ inline void mbar_arrive_expect_tx(uint64_t *bar, uint32_t bytes) {
    asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(smem_u32(bar)),
                 "r"(bytes)
                 : "memory");
}

__device__ inline void mbar_arrive(uint64_t *bar) {
    asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];" ::"r"(smem_u32(bar)) : "memory");
}

__device__ inline bool mbar_try_wait(uint64_t *bar, uint32_t parity) {
    uint32_t ok;
    asm volatile(
        "{\n\t.reg .pred p;\n\t"
        "mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n\t"
        "selp.u32 %0, 1, 0, p;\n\t}"
        : "=r"(ok)
        : "r"(smem_u32(bar)), "r"(parity)
        : "memory");
    return ok != 0;
}

// The same test, letting the hardware suspend the thread for up to hint_ns
// while the phase is incomplete (for warps whose waits are long and whose
// spinning would take issue slots from the warps they wait for)
__device__ inline bool mbar_try_wait_suspend(uint64_t *bar, uint32_t parity, uint32_t hint_ns) {
    uint32_t ok;
    asm volatile(
        "{\n\t.reg .pred p;\n\t"
        "mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2, %3;\n\t"
        "selp.u32 %0, 1, 0, p;\n\t}"
        : "=r"(ok)
        : "r"(smem_u32(bar)), "r"(parity), "r"(hint_ns)
        : "memory");
    return ok != 0;
}

// Bounded wait on an mbarrier phase: gives up after `budget_ns` nanoseconds
// of the global timer and returns false.
__device__ inline uint64_t global_ns() {
    uint64_t t;
    asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
    return t;
}

constexpr uint64_t kWaitBudgetNs = 2000000000ull;   // 2 s

__device__ inline bool mbar_wait_bounded(uint64_t *bar, uint32_t parity) {
    if (mbar_try_wait(bar, parity)) return true;
    uint64_t start = global_ns();
    while (true) {
        if (mbar_try_wait(bar, parity)) return true;
        if (global_ns() - start > kWaitBudgetNs) return false;
    }
}

// bounded wait with its own budget (the test of the waits' expiry path)
__device__ inline bool mbar_wait_ns(uint64_t *bar, uint32_t parity, uint64_t budget_ns) {
    if (mbar_try_wait(bar, parity)) return true;
    uint64_t start = global_ns();
    while (true) {
        if (mbar_try_wait(bar, parity)) return true;
        if (global_ns() - start > budget_ns) return false;
    }
}

// bounded wait whose retries (and, with first_too, its first test) may
// suspend the thread for up to 1 ms each
__device__ inline bool mbar_wait_bounded_suspend(uint64_t *bar, uint32_t parity,
                                                 bool first_too = false) {
    if (first_too ? mbar_try_wait_suspend(bar, parity, 1000000u) : mbar_try_wait(bar, parity))
        return true;
    uint64_t start = global_ns();
    while (true) {
        if (mbar_try_wait_suspend(bar, parity, 1000000u)) return true;
        if (global_ns() - start > kWaitBudgetNs) return false;
    }
}

// 2-D tiled TMA load of box (x, y) into shared memory, completing on `bar`.
__device__ inline void tma_load_2d(void *dst, const CUtensorMap *map, uint64_t *bar, int x,
                                   int y) {
    asm volatile(
        "cp.async.bulk.tensor.2d.shared::cluster.global.mbarrier::complete_tx::bytes"
        " [%0], [%1, {%3, %4}], [%2];" ::"r"(smem_u32(dst)),
        "l"(map), "r"(smem_u32(bar)), "r"(x), "r"(y)
        : "memory");
}

__device__ inline void tma_prefetch_desc(const CUtensorMap *map) {
    asm volatile("prefetch.tensormap [%0];" ::"l"(map) : "memory");
}

// Programmatic dependent launch.  Every kernel of the library starts by
// waiting for the kernel before it in the stream to finish (its writes then
// visible) and by letting the next kernel be scheduled, so a launch and the
// ramp-up of its CTAs overlap the predecessor's tail.  No global memory is
// touched before the wait; launched without the attribute both are no-ops.
__device__ inline void pdl_entry() {
    asm volatile("griddepcontrol.wait;" ::: "memory");
    asm volatile("griddepcontrol.launch_dependents;" ::: "memory");
}

// launch with the programmatic-stream-serialization attribute (pdl = false:
// a plain stream-ordered launch; the kernel's griddepcontrol steps are then
// no-ops)
template <typename... KArgs, typename... Args>
inline cudaError_t launch_pdl_if(bool pdl, void (*kern)(KArgs...), dim3 grid, dim3 block,
                                 size_t smem, cudaStream_t st, Args... args) {
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = grid;
    cfg.blockDim = block;
    cfg.dynamicSmemBytes = smem;
    cfg.stream = st;
    cudaLaunchAttribute at[1];
    at[0].id = cudaLaunchAttributeProgrammaticStreamSerialization;
    at[0].val.programmaticStreamSerializationAllowed = 1;
    cfg.attrs = at;
    cfg.numAttrs = pdl ? 1 : 0;
    return cudaLaunchKernelEx(&cfg, kern, args...);
}

template <typename... KArgs, typename... Args>
inline cudaError_t launch_pdl(void (*kern)(KArgs...), dim3 grid, dim3 block, size_t smem,
                              cudaStream_t st, Args... args) {
    return launch_pdl_if(true, kern, grid, block, smem, st, args...);
}

// SM count of the current device (cached per device)
int device_sms();

// Long-running kernels with fewer CTAs than SMs are launched without the
// programmatic attribute: launched early, while the previous kernel's CTAs
// drain, their CTAs were seen to land two to an SM instead of spreading out
// (a nine-CTA product took 3.18 ms per call with the attribute, 1.67 ms
// without).
inline bool pdl_for_grid(long long ctas) { return ctas >= device_sms(); }

// record a device-side failure in the plan (first writer wins)
__device__ inline void raise_status(DevPlan *plan, int code) {
    atomicCAS(&plan->status, 0, code);
}

}  // namespace tdg
