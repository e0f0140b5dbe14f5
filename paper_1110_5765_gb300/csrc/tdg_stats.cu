// Step (a), first half: per-block statistics of op(A) and op(B).
//
// Sec. 3 gathers max/min of every L x L subblock during the block-major
// reorder; Sec. 5.B adds sigma.  Here one CTA reads one L x L tile of the
// stored matrix with 16-byte vector loads (one HBM pass) and produces
//   max|x|   exact,
//   sigma^2  sum x^2 / (valid elements), about zero (fp32 inputs:
//            double-float accumulation of exact squares per thread and a
//            double-float tree over the block; fp64 inputs: fp64 throughout).
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

// (hi, lo) += (bh, bl) in double-float arithmetic (TwoSum of the high parts,
// low parts added to the error, then renormalised)
__device__ inline void df_add(float &hi, float &lo, float bh, float bl) {
    const float s = __fadd_rn(hi, bh);
    const float v = __fsub_rn(s, hi);
    const float e = __fadd_rn(__fsub_rn(hi, __fsub_rn(s, v)), __fsub_rn(bh, v));
    const float t = __fadd_rn(e, __fadd_rn(lo, bl));
    hi = __fadd_rn(s, t);
    lo = __fsub_rn(t, __fsub_rn(hi, s));
}

__device__ inline void add_sq(Acc &a, int lane, double x) {
    a.d[lane & 1] = __fma_rn(x, x, a.d[lane & 1]);
    unsigned long long b = (unsigned long long)__double_as_longlong(x) & 0x7fffffffffffffffull;
    a.mbits = max(a.mbits, b);
    a.bad |= (b >= 0x7ff0000000000000ull);
}

// One operand: the stored matrix rows_s x cols_s (leading dimension ld),
// op() transposed when trans; block (bi, bj) of the stored matrix is block
// (bj, bi) of op() then.  nbc_op = block columns of op().
template <typename T>
struct StatsOp {
    const T *X;
    long long rows_s, cols_s, ld;
    int trans, nbc_op, nbc_s;       // nbc_s = block columns of the stored matrix
    long long nblk;                 // blocks of the stored matrix
    double *mx, *var;
};

// Both operands in one launch: CTAs [0, A.nblk) take A's blocks, the rest B's.
template <typename T>
__global__ void __launch_bounds__(256) block_stats_kernel(StatsOp<T> A, StatsOp<T> B, int L,
                                                          DevPlan *plan) {
    pdl_entry();
    constexpr int VEC = 16 / sizeof(T);
    const bool isA = (long long)blockIdx.x < A.nblk;
    const StatsOp<T> &o = isA ? A : B;
    const long long blk = isA ? (long long)blockIdx.x : (long long)blockIdx.x - A.nblk;
    const long long bi = blk / o.nbc_s, bj = blk - bi * o.nbc_s;
    const T *__restrict__ X = o.X;
    const long long ld = o.ld;
    const long long r0b = bi * L, c0 = bj * L;
    const int rn = (int)min((long long)L, o.rows_s - r0b);
    const int cn = (int)min((long long)L, o.cols_s - c0);
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nwarp = blockDim.x >> 5;
    const bool vec_ok = (ld % VEC == 0) && ((reinterpret_cast<uintptr_t>(X) & 15) == 0);

    Acc a{{0.f, 0.f, 0.f, 0.f}, {0.f, 0.f, 0.f, 0.f}, {0.0, 0.0}, 0ull, 0};
    // rows in batches of eight per warp so eight 16-byte loads are in flight
    // before any of them is consumed
    constexpr int RB = 8;
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
    // block sum of squares and max|x|: fp32 inputs reduce (hi, lo) float pairs
    // with double-float additions and float bit patterns (GB300 runs fp64 at a
    // small fraction of the fp32 rate, so fp64 appears only once per block);
    // fp64 inputs reduce in fp64
    __shared__ float sh_h[32], sh_l[32];
    __shared__ double sh_d[32];
    __shared__ unsigned long long sh_m[32];
    __shared__ int sh_b[32];
    float hi = 0.f, lo = 0.f;
    double d = 0.0;
    if constexpr (sizeof(T) == 4) {
        hi = a.hi[0]; lo = a.lo[0];
#pragma unroll
        for (int q = 1; q < 4; ++q) df_add(hi, lo, a.hi[q], a.lo[q]);
    } else {
        d = a.d[0] + a.d[1];
    }
    unsigned long long mb = a.mbits;
    int bad = a.bad;
    auto warp_reduce = [&]() {
#pragma unroll
        for (int off = 16; off > 0; off >>= 1) {
            if constexpr (sizeof(T) == 4) {
                const float oh = __shfl_xor_sync(0xffffffffu, hi, off);
                const float ol = __shfl_xor_sync(0xffffffffu, lo, off);
                df_add(hi, lo, oh, ol);
            } else {
                d += __shfl_xor_sync(0xffffffffu, d, off);
            }
            mb = max(mb, (unsigned long long)__shfl_xor_sync(0xffffffffu, mb, off));
            bad |= __shfl_xor_sync(0xffffffffu, bad, off);
        }
    };
    warp_reduce();
    if (lane == 0) { sh_h[warp] = hi; sh_l[warp] = lo; sh_d[warp] = d; sh_m[warp] = mb; sh_b[warp] = bad; }
    __syncthreads();
    if (warp == 0) {
        const bool in = lane < nwarp;
        hi = in ? sh_h[lane] : 0.f;
        lo = in ? sh_l[lane] : 0.f;
        d = in ? sh_d[lane] : 0.0;
        mb = in ? sh_m[lane] : 0ull;
        bad = in ? sh_b[lane] : 0;
        warp_reduce();
        if (lane == 0) {
            const double ssum = sizeof(T) == 4 ? (double)hi + (double)lo : d;
            const double m = sizeof(T) == 4 ? (double)__uint_as_float((unsigned int)mb)
                                            : __longlong_as_double((long long)mb);
            long long idx = o.trans ? bj * o.nbc_op + bi : bi * o.nbc_op + bj;
            o.mx[idx] = m;
            o.var[idx] = ssum / ((double)rn * (double)cn);   // sigma^2 about zero
            if (bad) atomicExch(&plan->nonfinite, 1);
        }
    }
}

}  // namespace

template <typename T>
static StatsOp<T> stats_op(const T *X, long long rows_s, long long cols_s, long long ld, int L,
                           int trans, int nbc_op, double *mx, double *var) {
    StatsOp<T> o;
    o.X = X; o.rows_s = rows_s; o.cols_s = cols_s; o.ld = ld;
    o.trans = trans; o.nbc_op = nbc_op;
    o.nbc_s = cdiv_i(cols_s, L);
    o.nblk = (long long)cdiv_i(rows_s, L) * o.nbc_s;
    o.mx = mx; o.var = var;
    return o;
}

template <typename T>
cudaError_t launch_block_stats(const T *A, long long rows_a, long long cols_a, long long lda,
                               int trans_a, int nbc_a, double *mxA, double *varA, const T *B,
                               long long rows_b, long long cols_b, long long ldb, int trans_b,
                               int nbc_b, double *mxB, double *varB, int L, DevPlan *plan,
                               cudaStream_t st) {
    StatsOp<T> oa = stats_op(A, rows_a, cols_a, lda, L, trans_a, nbc_a, mxA, varA);
    StatsOp<T> ob = stats_op(B, rows_b, cols_b, ldb, L, trans_b, nbc_b, mxB, varB);
    const long long nb = oa.nblk + ob.nblk;
    if (nb > 0x7fffffffLL) return cudaErrorInvalidConfiguration;
    return launch_pdl(block_stats_kernel<T>, dim3((unsigned)nb), dim3(256), 0, st, oa, ob, L, plan);
}

#define TDG_STATS_INST(T)                                                                     \
    template cudaError_t launch_block_stats<T>(const T *, long long, long long, long long, int, \
                                               int, double *, double *, const T *, long long, \
                                               long long, long long, int, int, double *,        \
                                               double *, int, DevPlan *, cudaStream_t);
TDG_STATS_INST(float)
TDG_STATS_INST(double)

}  // namespace tdg
