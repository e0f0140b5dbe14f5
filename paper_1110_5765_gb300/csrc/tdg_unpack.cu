// Unfused step (d) and the distortion measurement.
//
// tdgemm_unpack: the packed GEMM can keep every slab's packed result r_bar
// (TDG_KEEP_PACKED).  This kernel unpacks them exactly as the fused epilogue
// does — eqs. 9-10 (symmetric) or 13-14 (asymmetric) — and exposes the
// integers r~ per output and slab (int64), plus C = sum_l r~ (s_A s_B)
// (eqs. 5, 2), so the integer domain can be compared bit for bit.  It also
// finishes a slab-split GEMM (few output tiles, many slabs: the slabs' packed
// products run in parallel and this kernel takes the sum over slabs in their
// order), then with alpha and beta as the fused epilogue applies them.
//
// tdgemm_snr: fp64 sums of ref^2, (C - ref)^2 and (C - ref) for eq. 20.
#include "tdg_common.cuh"
#include "tdg_internal.h"

namespace tdg {

namespace {

template <typename T>
__device__ inline T rint_d(T v) {
    if constexpr (sizeof(T) == 4) return rintf(v);
    else return rint(v);
}

template <typename T, int ASYM>
__global__ void unpack_kernel(GemmArgs<T> g, int W, int64_t *rint_out) {
    pdl_entry();
    if (g.plan->W != W) return;            // the planner chose another packing
    const long long total = g.M * g.N;
    const int q = g.plan->q;
    const T z = sizeof(T) == 4 ? (T)scalbnf(1.0f, -q) : (T)scalbn(1.0, -q);
    const T Q = sizeof(T) == 4 ? (T)scalbnf(1.0f, q) : (T)scalbn(1.0, q);
    for (long long e = (long long)blockIdx.x * blockDim.x + threadIdx.x; e < total;
         e += (long long)gridDim.x * blockDim.x) {
        const long long m = e / g.N, n = e % g.N;
        const long long i = m / g.L, jn = n / g.L;
        long long xr;
        int d = 0;
        if (ASYM) {
            const long long inblk = m % g.L;
            xr = i * g.P + inblk / W;
            d = (int)(inblk % W);
        } else {
            xr = m;
        }
        T c = T(0);
        for (int l = 0; l < g.nK; ++l) {
            const T rbar = g.Rbar[((long long)l * g.Mrows + xr) * g.N + n];
            T rt;
            if (ASYM) {
                T x = rbar;
                rt = rint_d(x);
                for (int k = 0; k < d; ++k) {
                    if constexpr (sizeof(T) == 4) x = __fmul_rn(Q, __fsub_rn(x, rt));
                    else x = __dmul_rn(Q, __dsub_rn(x, rt));
                    rt = rint_d(x);
                }
            } else {
                const T u = rint_d(rbar);
                T t;
                if constexpr (sizeof(T) == 4) {
                    t = rintf(__fmul_rn(z, u));
                    rt = __fmaf_rn(-Q, t, u);
                } else {
                    t = rint(__dmul_rn(z, u));
                    rt = __fma_rn(-Q, t, u);
                }
            }
            const T pr = g.pair[((long long)l * g.nM + i) * g.nN + jn];
            if constexpr (sizeof(T) == 4) c = __fmaf_rn(rt, pr, c);
            else c = __fma_rn(rt, pr, c);
            if (rint_out) rint_out[e * g.nK + l] = (int64_t)rt;
        }
        if (g.C) {
            // the GEMM epilogue: C = alpha c (beta == 0) or alpha c + beta C
            T *pc = g.C + m * g.ldc + n;
            if constexpr (sizeof(T) == 4)
                *pc = g.beta_zero ? __fmul_rn(g.alpha, c) : __fmaf_rn(g.alpha, c, __fmul_rn(g.beta, *pc));
            else
                *pc = g.beta_zero ? __dmul_rn(g.alpha, c) : __fma_rn(g.alpha, c, __dmul_rn(g.beta, *pc));
        }
    }
}

template <typename T>
__global__ void snr_kernel(const T *C, long long ldc, const double *ref, long long ldr,
                           long long M, long long N, double *out3) {
    double s_ref = 0, s_err2 = 0, s_err = 0;
    const long long total = M * N;
    for (long long e = (long long)blockIdx.x * blockDim.x + threadIdx.x; e < total;
         e += (long long)gridDim.x * blockDim.x) {
        const long long m = e / N, n = e % N;
        const double r = ref[m * ldr + n];
        const double err = (double)C[m * ldc + n] - r;
        s_ref += r * r;
        s_err2 += err * err;
        s_err += err;
    }
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
        s_ref += __shfl_xor_sync(0xffffffffu, s_ref, o);
        s_err2 += __shfl_xor_sync(0xffffffffu, s_err2, o);
        s_err += __shfl_xor_sync(0xffffffffu, s_err, o);
    }
    __shared__ double sh[3][32];
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    if (lane == 0) { sh[0][warp] = s_ref; sh[1][warp] = s_err2; sh[2][warp] = s_err; }
    __syncthreads();
    if (warp == 0) {
        const int nw = blockDim.x >> 5;
        s_ref = lane < nw ? sh[0][lane] : 0.0;
        s_err2 = lane < nw ? sh[1][lane] : 0.0;
        s_err = lane < nw ? sh[2][lane] : 0.0;
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) {
            s_ref += __shfl_xor_sync(0xffffffffu, s_ref, o);
            s_err2 += __shfl_xor_sync(0xffffffffu, s_err2, o);
            s_err += __shfl_xor_sync(0xffffffffu, s_err, o);
        }
        if (lane == 0) {
            atomicAdd(&out3[0], s_ref);
            atomicAdd(&out3[1], s_err2);
            atomicAdd(&out3[2], s_err);
        }
    }
}

}  // namespace

template <typename T>
cudaError_t launch_unpack(int form, int W, const GemmArgs<T> &g, int64_t *rint_out,
                          cudaStream_t st) {
    const long long total = g.M * g.N;
    const int grid = (int)min((total + 255) / 256, 152LL * 32);
    if (form == G_ASYM) return launch_pdl(unpack_kernel<T, 1>, dim3(grid), dim3(256), 0, st, g, W, rint_out);
    return launch_pdl(unpack_kernel<T, 0>, dim3(grid), dim3(256), 0, st, g, W, rint_out);
}

template cudaError_t launch_unpack<float>(int, int, const GemmArgs<float> &, int64_t *,
                                          cudaStream_t);
template cudaError_t launch_unpack<double>(int, int, const GemmArgs<double> &, int64_t *,
                                           cudaStream_t);

cudaError_t launch_snr(const void *C, long long ldc, int dtype, const double *ref, long long ldr,
                       long long M, long long N, double *out3, cudaStream_t st) {
    cudaError_t e = cudaMemsetAsync(out3, 0, 3 * sizeof(double), st);
    if (e != cudaSuccess) return e;
    const long long total = M * N;
    const int grid = (int)min((total + 255) / 256, 152LL * 8);
    if (dtype == TDG_F64)
        snr_kernel<double><<<grid, 256, 0, st>>>((const double *)C, ldc, ref, ldr, M, N, out3);
    else
        snr_kernel<float><<<grid, 256, 0, st>>>((const float *)C, ldc, ref, ldr, M, N, out3);
    return cudaGetLastError();
}

}  // namespace tdg
