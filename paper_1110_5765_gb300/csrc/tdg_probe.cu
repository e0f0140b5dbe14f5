// tdgemm_fma_probe: the fused multiply-add rate of every SM's FP32 or FP64
// pipe, measured.  The packed forms (steps c and d) run on these pipes, so
// their roofline fraction is taken against this rate (the measured bf16
// peak of the tensor pipe does not apply to them).
//
// The patterns are the fastest of several measured on GB300.  FP32: each
// thread runs kChains independent chains x <- fma.rn.f32x2(x, a, b) (a = 1 -
// 2^-12, b = 2^-12: every chain converges to 1, no overflow or subnormals).
// FP64: the GEMM main loop's own pattern, acc[i][j] <- fma(a[i], b[j],
// acc[i][j]) over a 2 x 4 register tile with the accumulators as addends
// (chains through the multiplicand, or one shared operand for all chains,
// measured about 15 % slower on the FP64 pipe).  The launch holds a full
// occupancy of 256-thread CTAs on every SM.  Nothing is read or written in
// memory: the sum is compared with a NaN argument and stored only if equal,
// which never happens, but keeps the compiler from removing the work.
#include <cuda_runtime.h>
#include <stdint.h>

#include "tdg_common.cuh"
#include "tdg_internal.h"
#include "tdgemm.h"

namespace tdg {
namespace {

constexpr int kChains = 8;
constexpr int kThreads = 256;

__global__ void __launch_bounds__(kThreads) fma_probe_f32x2(long long iters, float never,
                                                            float *sink) {
    uint64_t x[kChains];
    uint64_t a2, b2;
    const float a = 1.0f - 1.0f / 4096.0f, b = 1.0f / 4096.0f;
    asm("mov.b64 %0, {%1, %1};" : "=l"(a2) : "f"(a));
    asm("mov.b64 %0, {%1, %1};" : "=l"(b2) : "f"(b));
#pragma unroll
    for (int c = 0; c < kChains; ++c) {
        const float v = (float)(threadIdx.x + c) * 1e-3f;
        asm("mov.b64 %0, {%1, %2};" : "=l"(x[c]) : "f"(v), "f"(-v));
    }
    for (long long i = 0; i < iters; ++i) {
#pragma unroll
        for (int c = 0; c < kChains; ++c)
            asm volatile("fma.rn.f32x2 %0, %0, %1, %2;" : "+l"(x[c]) : "l"(a2), "l"(b2));
    }
    float s = 0.f;
#pragma unroll
    for (int c = 0; c < kChains; ++c) {
        float lo, hi;
        asm("mov.b64 {%0, %1}, %2;" : "=f"(lo), "=f"(hi) : "l"(x[c]));
        s += lo + hi;
    }
    if (s == never) sink[threadIdx.x] = s;
}

__global__ void __launch_bounds__(kThreads) fma_probe_f64(long long iters, double never,
                                                          double *sink) {
    constexpr int TI = 2, TJ = kChains / TI;
    double a[TI], b[TJ], acc[TI][TJ];
#pragma unroll
    for (int i = 0; i < TI; ++i) a[i] = 1e-3 * (double)(threadIdx.x + i + 1);
#pragma unroll
    for (int j = 0; j < TJ; ++j) b[j] = 1e-4 * (double)(threadIdx.x + j + 1);
#pragma unroll
    for (int i = 0; i < TI; ++i)
#pragma unroll
        for (int j = 0; j < TJ; ++j) acc[i][j] = 0.0;
    for (long long it = 0; it < iters; ++it) {
#pragma unroll
        for (int i = 0; i < TI; ++i)
#pragma unroll
            for (int j = 0; j < TJ; ++j)
                asm volatile("fma.rn.f64 %0, %1, %2, %0;" : "+d"(acc[i][j]) : "d"(a[i]), "d"(b[j]));
    }
    double s = 0.0;
#pragma unroll
    for (int i = 0; i < TI; ++i)
#pragma unroll
        for (int j = 0; j < TJ; ++j) s += acc[i][j];
    if (s == never) sink[threadIdx.x] = s;
}

}  // namespace
}  // namespace tdg

extern "C" tdg_status tdgemm_fma_probe(tdg_dtype dtype, int64_t iters, double *flops,
                                       void *stream) {
    using namespace tdg;
    if (iters < 1 || !flops) {
        record_error("tdgemm_fma_probe: iters must be >= 1 and flops non-NULL");
        return TDG_EINVAL;
    }
    if (dtype != TDG_F32 && dtype != TDG_F64) {
        record_error("tdgemm_fma_probe: bad dtype");
        return TDG_EINVAL;
    }
    int dev = 0, sms = 0, per = 0;
    cudaGetDevice(&dev);
    cudaError_t e = cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    const void *kern = dtype == TDG_F32 ? (const void *)fma_probe_f32x2 : (const void *)fma_probe_f64;
    if (e == cudaSuccess) e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per, kern, kThreads, 0);
    if (e != cudaSuccess || sms < 1 || per < 1) {
        record_error("tdgemm_fma_probe: device query failed");
        return TDG_ECUDA;
    }
    const long long threads = (long long)sms * per * kThreads;
    cudaStream_t st = (cudaStream_t)stream;
    if (dtype == TDG_F32) {
        fma_probe_f32x2<<<sms * per, kThreads, 0, st>>>(iters, __builtin_nanf(""), nullptr);
        *flops = (double)threads * (double)iters * kChains * 2 /* lanes */ * 2 /* flop */;
    } else {
        fma_probe_f64<<<sms * per, kThreads, 0, st>>>(iters, __builtin_nan(""), nullptr);
        *flops = (double)threads * (double)iters * kChains * 2;
    }
    e = cudaGetLastError();
    if (e != cudaSuccess) {
        record_error(cudaGetErrorString(e));
        return TDG_ECUDA;
    }
    return TDG_OK;
}
