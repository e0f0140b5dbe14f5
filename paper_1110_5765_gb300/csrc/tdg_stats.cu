// Step (a), first half: per-block statistics of op(A) and op(B).
//
// Sec. 3 gathers max/min of every L x L subblock during the block-major
// reorder; Sec. 5.B adds sigma.  Here one CTA reads one L x L tile of the
// stored matrix with 16-byte vector loads (one HBM pass) and produces
//   max|x|   exact,
//   sigma^2  sum x^2 / (valid elements), about zero; the sum in fp64 (fp32
//            inputs: per-thread double-float accumulation of exact squares,
//            then an fp64 tree).
// Non-finite inputs raise TDG_ENONFINITE in the plan's device status.
#include "tdg_common.cuh"
#include "tdg_internal.h"

namespace tdg {

namespace {

// max|x| is kept as the largest bit pattern of |x| (for non-negative IEEE
// values the integer order is the numeric order), which stays on the integer
// pipe; NaN/Inf are flagged separately.  Each thread keeps one running sum
// per vector lane so the dependent add chains run side by side.
struct Acc {
    float hi[4], lo[4];        // fp32 path: double-float sums of squares
    double d[2];               // fp64 path
    unsigned long long mbits;  // bit pattern of the largest |x|
    int bad;
};

__device__ inline void add_sq(Acc &a, int lane, float x) {
    // exact square as hi + err (TwoProduct), then TwoSum into (hi, lo)
    float p = __fmul_rn(x, x);
    float e = __fmaf_rn(x, x, -p);
    float t = __fadd_rn(a.hi[lane], p);
    float bp = __fsub_rn(t, a.hi[lane]);
    float err = __fadd_rn(__fsub_rn(a.hi[lane], __fsub_rn(t, bp)), __fsub_rn(p, bp));
    a.hi[lane] = t;
    a.lo[lane] = __fadd_rn(a.lo[lane], __fadd_rn(err, e));
    unsigned int b = __float_as_uint(x) & 0x7fffffffu;
    a.mbits = max(a.mbits, (unsigned long long)b);
    a.bad |= (b >= 0x7f800000u);
}

__device__ inline void add_sq(Acc &a, int lane, double x) {
    a.d[lane & 1] = __fma_rn(x, x, a.d[lane & 1]);
    unsigned long long b = (unsigned long long)__double_as_longlong(x) & 0x7fffffffffffffffull;
    a.mbits = max(a.mbits, b);
    a.bad |= (b >= 0x7ff0000000000000ull);
}

template <typename T>
__global__ void __launch_bounds__(256) block_stats_kernel(const T *__restrict__ X,
                                                          long long rows_s, long long cols_s,
                                                          long long ld, int L, int trans,
                                                          int nbc_op, double *__restrict__ mx,
                                                          double *__restrict__ var,
                                                          DevPlan *plan) {
    constexpr int VEC = 16 / sizeof(T);
    const int bj = blockIdx.x, bi = blockIdx.y;
    const long long r0b = (long long)bi * L, c0 = (long long)bj * L;
    const int rn = (int)min((long long)L, rows_s - r0b);
    const int cn = (int)min((long long)L, cols_s - c0);
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nwarp = blockDim.x >> 5;
    const bool vec_ok = (ld % VEC == 0) && ((reinterpret_cast<uintptr_t>(X) & 15) == 0);

    Acc a{{0.f, 0.f, 0.f, 0.f}, {0.f, 0.f, 0.f, 0.f}, {0.0, 0.0}, 0ull, 0};
    // rows in batches of four per warp so four 16-byte loads are in flight
    // before any of them is consumed
    constexpr int RB = 4;
    for (int c = lane * VEC; c < cn; c += 32 * VEC) {
        const bool vec = vec_ok && c + VEC <= cn;
        for (int r0 = warp; r0 < rn; r0 += RB * nwarp) {
            T v[RB][VEC];
#pragma unroll
            for (int u = 0; u < RB; ++u) {
                const int r = r0 + u * nwarp;
                const T *row = X + (r0b + r) * ld + c0 + c;
                if (r < rn && vec) {
                    if constexpr (sizeof(T) == 4) {
                        float4 q = __ldg(reinterpret_cast<const float4 *>(row));
                        v[u][0] = q.x; v[u][1] = q.y; v[u][2] = q.z; v[u][3] = q.w;
                    } else {
                        double2 q = __ldg(reinterpret_cast<const double2 *>(row));
                        v[u][0] = q.x; v[u][1] = q.y;
                    }
                } else {
#pragma unroll
                    for (int e = 0; e < VEC; ++e) v[u][e] = (r < rn && c + e < cn) ? row[e] : T(0);
                }
            }
#pragma unroll
            for (int u = 0; u < RB; ++u)
#pragma unroll
                for (int e = 0; e < VEC; ++e) add_sq(a, e, v[u][e]);
        }
    }
    double s;
    if (sizeof(T) == 4) {
        s = 0.0;
#pragma unroll
        for (int q = 0; q < 4; ++q) s += (double)a.hi[q] + (double)a.lo[q];
    } else {
        s = a.d[0] + a.d[1];
    }
    double m = (sizeof(T) == 4) ? (double)__uint_as_float((unsigned int)a.mbits)
                                : __longlong_as_double((long long)a.mbits);
    int bad = a.bad;
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
        s += __shfl_xor_sync(0xffffffffu, s, o);
        m = fmax(m, __shfl_xor_sync(0xffffffffu, m, o));
        bad |= __shfl_xor_sync(0xffffffffu, bad, o);
    }
    __shared__ double sh_s[32], sh_m[32];
    __shared__ int sh_b[32];
    if (lane == 0) { sh_s[warp] = s; sh_m[warp] = m; sh_b[warp] = bad; }
    __syncthreads();
    if (warp == 0) {
        s = lane < nwarp ? sh_s[lane] : 0.0;
        m = lane < nwarp ? sh_m[lane] : 0.0;
        bad = lane < nwarp ? sh_b[lane] : 0;
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) {
            s += __shfl_xor_sync(0xffffffffu, s, o);
            m = fmax(m, __shfl_xor_sync(0xffffffffu, m, o));
            bad |= __shfl_xor_sync(0xffffffffu, bad, o);
        }
        if (lane == 0) {
            long long idx = trans ? (long long)bj * nbc_op + bi : (long long)bi * nbc_op + bj;
            mx[idx] = m;
            var[idx] = s / ((double)rn * (double)cn);   // sigma^2 about zero
            if (bad) atomicExch(&plan->nonfinite, 1);
        }
    }
}

}  // namespace

template <typename T>
cudaError_t launch_block_stats(const T *X, long long rows_s, long long cols_s, long long ld,
                               int L, int trans, int nbc_op, double *mx, double *var,
                               DevPlan *plan, cudaStream_t st) {
    dim3 grid(cdiv_i(cols_s, L), cdiv_i(rows_s, L));
    block_stats_kernel<T><<<grid, 256, 0, st>>>(X, rows_s, cols_s, ld, L, trans, nbc_op, mx, var,
                                                plan);
    return cudaGetLastError();
}

template cudaError_t launch_block_stats<float>(const float *, long long, long long, long long,
                                               int, int, int, double *, double *, DevPlan *,
                                               cudaStream_t);
template cudaError_t launch_block_stats<double>(const double *, long long, long long,
                                                long long, int, int, int, double *, double *,
                                                DevPlan *, cudaStream_t);

}  // namespace tdg
