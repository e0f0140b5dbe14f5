// tdgemm_fma_probe: the fused multiply-add rate of every SM's FP32 or FP64
// pipe, measured.  The packed forms (steps c and d) run on these pipes, so
// their roofline fraction is taken against this rate (the measured bf16
// peak of the tensor pipe does not apply to them).
//
// Each thread runs kChains independent accumulation chains
// acc <- fma(a_c, b, acc), the accumulator as the addend as in the GEMM's main
// loop (with the accumulator as a multiplicand GB300's FP64 pipe measured
// about 15 % slower), enough to cover the pipe's latency; the launch holds a
// full occupancy of 256-thread CTAs on every SM.  a_c b is 2^-24 or so, so
// the sums stay near 1 (no overflow, no subnormals).  Nothing is read or
// written in memory: the chains' sum is compared with a NaN argument and
// stored only if equal, which never happens, but keeps the compiler from
// removing the work.
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
    uint64_t acc[kChains], a2[kChains], b2;
    const float b = 1.0f / 4096.0f;
    asm("mov.b64 %0, {%1, %1};" : "=l"(b2) : "f"(b));
#pragma unroll
    for (int c = 0; c < kChains; ++c) {
        const float a = (1.0f + (float)c / 64.0f) / 4096.0f;
        asm("mov.b64 %0, {%1, %2};" : "=l"(a2[c]) : "f"(a), "f"(-a));
        asm("mov.b64 %0, {%1, %1};" : "=l"(acc[c]) : "f"(1.0f + (float)threadIdx.x * 1e-3f));
    }
    for (long long i = 0; i < iters; ++i) {
#pragma unroll
        for (int c = 0; c < kChains; ++c)
            asm volatile("fma.rn.f32x2 %0, %1, %2, %0;" : "+l"(acc[c]) : "l"(a2[c]), "l"(b2));
    }
    float s = 0.f;
#pragma unroll
    for (int c = 0; c < kChains; ++c) {
        float lo, hi;
        asm("mov.b64 {%0, %1}, %2;" : "=f"(lo), "=f"(hi) : "l"(acc[c]));
        s += lo + hi;
    }
    if (s == never) sink[threadIdx.x] = s;
}

__global__ void __launch_bounds__(kThreads) fma_probe_f64(long long iters, double never,
                                                          double *sink) {
    double acc[kChains], a[kChains];
    const double b = 1.0 / 4096.0;
#pragma unroll
    for (int c = 0; c < kChains; ++c) {
        a[c] = (1.0 + (double)c / 64.0) / 4096.0;
        acc[c] = 1.0 + (double)threadIdx.x * 1e-3;
    }
    for (long long i = 0; i < iters; ++i) {
#pragma unroll
        for (int c = 0; c < kChains; ++c)
            asm volatile("fma.rn.f64 %0, %1, %2, %0;" : "+d"(acc[c]) : "d"(a[c]), "d"(b));
    }
    double s = 0.0;
#pragma unroll
    for (int c = 0; c < kChains; ++c) s += acc[c];
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
