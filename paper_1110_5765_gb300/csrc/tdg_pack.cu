// Steps (a) and (b) on the data: companding and rounding (eq. 3) fused with
// packing (eqs. 6, 7, 11) in one pass over each input.
//
// Every element is quantized as a~ = rint(fl_T(x * c_T)) with its block's
// compander and the packed number is built by Horner's rule,
//     acc = d_{W-1};  acc = fma(w, acc, d_i),  i = W-2 .. 0,
// with w = z for eqs. 6 and 11 and w = z^-1 for eq. 7.  Digits outside the
// L x L block or the matrix are zero (border clean-up, Sec. 2).
//
//   pack along k   out[l P + j][x]  (eq. 6 for A, eq. 7 for B, W = 1 for the
//                  unpacked operands and the plain copies):
//                    - x contiguous in the input: 16-byte vector loads of the
//                      W digit rows, vector stores, no shared memory;
//                    - k contiguous in the input: a TILE x TILE W tile (TILE =
//                      64 x-rows for fp32 with W <= 2, else 32) staged in
//                      shared memory with vector loads, then written along x.
//   pack along x   out[k][i P + j]  (eq. 11, asymmetric A), tile staged in
//                  shared memory.
//   k-major codes  out[x][k] (tensor-core forms): integer-valued fp16, or E4M3
//                  (round to nearest even, saturating).
//   fused codes    for companders that depend on their own block only (fixed
//                  bits, E4M3) and L <= 128: one 512-thread CTA per block
//                  reads it once into registers, reduces max|x| and sum x^2,
//                  writes c and s and encodes the codes.
// P = ceil(L / W) packed numbers per block.  Each kernel first reads the
// device plan and returns unless the planner chose its packing; the grids are
// capped and loop over tiles so that such early exits cost little.
#include <cuda_fp16.h>
#include <cuda_fp8.h>

#include <mutex>

#include "tdg_common.cuh"
#include "tdg_internal.h"
#include "tdg_pack.h"

namespace tdg {

namespace {

constexpr int TILE = 32;
constexpr int MAX_CTAS = 152 * 8;

template <typename T>
struct Src {
    const T *p;
    long long sx, sk;
    long long X, K;
    const T *c;       // nullptr: copy without companding
    long long cx, cl;
    int L;
};

template <typename T>
__device__ inline T quant(T v, T c, bool compand) {
    if (!compand) return v;
    if constexpr (sizeof(T) == 4) return rintf(__fmul_rn(v, c));
    else return rint(__dmul_rn(v, c));
}

template <typename T>
__device__ inline T fma_t(T a, T b, T c) {
    if constexpr (sizeof(T) == 4) return __fmaf_rn(a, b, c);
    else return __fma_rn(a, b, c);
}

// w = z = 2^-q (wsign < 0) or z^-1 = 2^q (wsign > 0), q from the device plan
template <typename T>
__device__ inline T pack_weight(const DevPlan *plan, int wsign) {
    int q = plan->q;
    if constexpr (sizeof(T) == 4) return scalbnf(1.0f, wsign < 0 ? -q : q);
    else return scalbn(1.0, wsign < 0 ? -q : q);
}

template <typename T>
struct VecT;
template <>
struct VecT<float> { static constexpr int n = 4; };
template <>
struct VecT<double> { static constexpr int n = 2; };

template <typename T>
__device__ inline void vload(const T *p, T *o) {
    if constexpr (sizeof(T) == 4) {
        float4 v = __ldg(reinterpret_cast<const float4 *>(p));
        o[0] = v.x; o[1] = v.y; o[2] = v.z; o[3] = v.w;
    } else {
        double2 v = __ldg(reinterpret_cast<const double2 *>(p));
        o[0] = v.x; o[1] = v.y;
    }
}

template <typename T>
__device__ inline void vstore(T *p, const T *o) {
    if constexpr (sizeof(T) == 4) *reinterpret_cast<float4 *>(p) = make_float4(o[0], o[1], o[2], o[3]);
    else *reinterpret_cast<double2 *>(p) = make_double2(o[0], o[1]);
}

// ------------------------------------------------------------------ pack along k,
// x contiguous in the input: one item = VEC consecutive x of one packed row
// (the loop of CTA vb of vg working on this operand)
template <typename T, int W>
__device__ __forceinline__ void pack_k_xc_body(const Src<T> &S, int P, T w, T *out, long long ldo,
                                               long long rows_out, int vec_ok, long long vb,
                                               long long vg) {
    constexpr int VEC = VecT<T>::n;
    const bool compand = S.c != nullptr;
    const int L = S.L;
    const long long nx = (S.X + VEC - 1) / VEC;
    const long long items = rows_out * nx;
    for (long long it = vb * blockDim.x + threadIdx.x; it < items; it += vg * blockDim.x) {
        const long long row = it / nx;                 // l * P + j
        const long long x = (it - row * nx) * VEC;
        const int l = (int)(row / P), j = (int)(row - (long long)l * P);
        const long long kbase = (long long)l * L + (long long)W * j;
        const long long klim = min((long long)(l + 1) * L, S.K);
        const T c = compand ? S.c[(x / L) * S.cx + (long long)l * S.cl] : T(1);
        T acc[VEC];
        const bool full = vec_ok && x + VEC <= S.X;
#pragma unroll
        for (int i = W - 1; i >= 0; --i) {
            const long long k = kbase + i;
            T d[VEC];
            if (k < klim && W * j + i < L) {
                const T *src = S.p + k * S.sk + x;
                if (full) {
                    vload(src, d);
                } else {
#pragma unroll
                    for (int e = 0; e < VEC; ++e) d[e] = (x + e < S.X) ? src[e] : T(0);
                }
#pragma unroll
                for (int e = 0; e < VEC; ++e) d[e] = quant(d[e], c, compand);
            } else {
#pragma unroll
                for (int e = 0; e < VEC; ++e) d[e] = T(0);
            }
#pragma unroll
            for (int e = 0; e < VEC; ++e) acc[e] = (i == W - 1) ? d[e] : fma_t(w, acc[e], d[e]);
        }
        T *dst = out + row * ldo + x;
        if (full) {
            vstore(dst, acc);
        } else {
#pragma unroll
            for (int e = 0; e < VEC; ++e)
                if (x + e < S.X) dst[e] = acc[e];
        }
    }
}

template <typename T, int W>
__global__ void __launch_bounds__(256) pack_k_xc_kernel(Src<T> S, int P, const DevPlan *plan,
                                                        int expectW, int wsign, T *out,
                                                        long long ldo, long long rows_out,
                                                        int vec_ok) {
    pdl_entry();
    if (expectW > 0 && plan->W != expectW) return;
    const T w = W > 1 ? pack_weight<T>(plan, wsign) : T(1);
    pack_k_xc_body<T, W>(S, P, w, out, ldo, rows_out, vec_ok, blockIdx.x, gridDim.x);
}

// ------------------------------------------------------------------ pack along k,
// k contiguous in the input: x-rows per tile of pack_k_kc_kernel (shared by
// the kernel and its launch), each tile TILE packed columns wide
template <typename T, int W>
constexpr int kc_tile() { return (sizeof(T) == 4 && W <= 2) ? 64 : 32; }

template <typename T, int W>
__device__ __forceinline__ void pack_k_kc_body(const Src<T> &S, int P, T w, T *out, long long ldo,
                                               long long rows_out, int vec_ok, long long vb,
                                               long long vg) {
    constexpr int VEC = VecT<T>::n;
    // fp32 with W <= 2: 64 x-rows per tile (a 33 KB tile, four times the
    // work per pass of the loop's fixed costs); else 32
    constexpr int TILE = kc_tile<T, W>();
    constexpr int NK = TILE * W;            // k values per tile row
    constexpr int PITCH = NK + 1;
    __shared__ T s[TILE * PITCH];
    __shared__ T crow[TILE];
    const bool compand = S.c != nullptr;
    const int L = S.L;
    const int jt = (P + TILE - 1) / TILE;
    const long long xt = (S.X + TILE - 1) / TILE;
    const int nK = (int)((S.K + L - 1) / L);
    const long long tiles = xt * nK * jt;
    for (long long t = vb; t < tiles; t += vg) {
        const long long xtile = t % xt;
        const long long r = t / xt;
        const int l = (int)(r / jt), j0 = (int)(r % jt) * TILE;
        const long long x0 = xtile * TILE;
        const long long kslab = (long long)l * L;
        const long long k0 = kslab + (long long)W * j0;
        const long long klim = min(kslab + L, S.K);
        __syncthreads();   // previous tile's readers are done with s / crow
        if (threadIdx.x < TILE) {
            const long long x = x0 + threadIdx.x;
            crow[threadIdx.x] = (compand && x < S.X) ? S.c[(x / L) * S.cx + (long long)l * S.cl] : T(1);
        }
        __syncthreads();
        constexpr int CH = NK / VEC;
        for (int e = threadIdx.x; e < TILE * CH; e += blockDim.x) {
            const int xr = e / CH, kc = (e % CH) * VEC;
            const long long x = x0 + xr, k = k0 + kc;
            T d[VEC];
            if (x < S.X && vec_ok && k + VEC <= klim) {
                vload(S.p + x * S.sx + k, d);
            } else {
#pragma unroll
                for (int q = 0; q < VEC; ++q)
                    d[q] = (x < S.X && k + q < klim) ? S.p[x * S.sx + k + q] : T(0);
            }
            const T c = crow[xr];
#pragma unroll
            for (int q = 0; q < VEC; ++q) {
                const bool valid = x < S.X && k + q < klim;
                s[xr * PITCH + kc + q] = valid ? quant(d[q], c, compand) : T(0);
            }
        }
        __syncthreads();
        for (int e = threadIdx.x; e < TILE * TILE; e += blockDim.x) {
            const int jr = e / TILE, xr = e % TILE;
            const int j = j0 + jr;
            const long long x = x0 + xr;
            const long long row = (long long)l * P + j;
            if (j >= P || x >= S.X || row >= rows_out) continue;
            const T *d = s + xr * PITCH + jr * W;
            T acc = d[W - 1];
#pragma unroll
            for (int i = W - 2; i >= 0; --i) acc = fma_t(w, acc, d[i]);
            out[row * ldo + x] = acc;
        }
    }
}

template <typename T, int W>
__global__ void __launch_bounds__(256) pack_k_kc_kernel(Src<T> S, int P, const DevPlan *plan,
                                                        int expectW, int wsign, T *out,
                                                        long long ldo, long long rows_out,
                                                        int vec_ok) {
    pdl_entry();
    if (expectW > 0 && plan->W != expectW) return;
    const T w = W > 1 ? pack_weight<T>(plan, wsign) : T(1);
    pack_k_kc_body<T, W>(S, P, w, out, ldo, rows_out, vec_ok, blockIdx.x, gridDim.x);
}

// Both operands of the symmetric form in one launch, A k-contiguous (eq. 6)
// and B x-contiguous (eq. 7), the layouts of C = A B with row-major A and B:
// the first 2 m CTAs alternate between the two (m = the smaller CTA count),
// the rest go to the operand with more, so every SM runs both kinds at once
// (the A pack is issue-bound, the B pack latency-bound).
template <typename T, int W>
__global__ void __launch_bounds__(256) pack_k_pair_kernel(Src<T> SA, Src<T> SB, int P,
                                                          const DevPlan *plan, int expectW,
                                                          T *outA, long long ldoA,
                                                          long long rowsA, int vecA, T *outB,
                                                          long long ldoB, long long rowsB,
                                                          int vecB, long long gA, long long gB) {
    pdl_entry();
    if (expectW > 0 && plan->W != expectW) return;
    const long long b = blockIdx.x, m = min(gA, gB);
    bool isA;
    long long vb;
    if (b < 2 * m) {
        isA = (b & 1) != 0;
        vb = b >> 1;
    } else {
        isA = gA > gB;
        vb = m + (b - 2 * m);
    }
    if (isA) {
        const T w = W > 1 ? pack_weight<T>(plan, -1) : T(1);
        pack_k_kc_body<T, W>(SA, P, w, outA, ldoA, rowsA, vecA, vb, gA);
    } else {
        const T w = W > 1 ? pack_weight<T>(plan, +1) : T(1);
        pack_k_xc_body<T, W>(SB, P, w, outB, ldoB, rowsB, vecB, vb, gB);
    }
}

// ------------------------------------------------------------------ plain k-major copy
// out[k][x] = in[x][k] of a k-contiguous operand without companding (the
// plain product's operands): 64 x 64 tiles through shared memory (s[x][k],
// pitch 65), 16-byte loads along k issued before any is used, 16-byte stores
// along x.  256 threads per CTA.
template <typename T>
__global__ void __launch_bounds__(256) transpose_copy_kernel(Src<T> S, const DevPlan *plan,
                                                             int expectW, T *out, long long ldo,
                                                             int vec_ok) {
    pdl_entry();
    if (expectW > 0 && plan->W != expectW) return;
    constexpr int VEC = VecT<T>::n;
    constexpr int TT = 64, PITCH = TT + 1;
    constexpr int NV = TT * TT / VEC / 256;     // vectors per thread and phase
    __shared__ T s[TT * PITCH];
    const long long xt = (S.X + TT - 1) / TT, kt = (S.K + TT - 1) / TT;
    for (long long t = blockIdx.x; t < xt * kt; t += gridDim.x) {
        const long long x0 = (t % xt) * TT, k0 = (t / xt) * TT;
        T v[NV][VEC];
#pragma unroll
        for (int u = 0; u < NV; ++u) {
            const int e = threadIdx.x + u * 256;
            const int xr = e / (TT / VEC), kc = (e % (TT / VEC)) * VEC;
            const long long x = x0 + xr, k = k0 + kc;
            if (x < S.X && vec_ok && k + VEC <= S.K) {
                vload(S.p + x * S.sx + k, v[u]);
            } else {
#pragma unroll
                for (int q = 0; q < VEC; ++q)
                    v[u][q] = (x < S.X && k + q < S.K) ? S.p[x * S.sx + k + q] : T(0);
            }
        }
        __syncthreads();   // the previous tile's readers are done with s
#pragma unroll
        for (int u = 0; u < NV; ++u) {
            const int e = threadIdx.x + u * 256;
            const int xr = e / (TT / VEC), kc = (e % (TT / VEC)) * VEC;
#pragma unroll
            for (int q = 0; q < VEC; ++q) s[xr * PITCH + kc + q] = v[u][q];
        }
        __syncthreads();
#pragma unroll
        for (int u = 0; u < NV; ++u) {
            const int e = threadIdx.x + u * 256;
            const int kr = e / (TT / VEC), xc = (e % (TT / VEC)) * VEC;
            const long long k = k0 + kr, x = x0 + xc;
            if (k >= S.K || x >= S.X) continue;
            T w[VEC];
#pragma unroll
            for (int q = 0; q < VEC; ++q) w[q] = s[(xc + q) * PITCH + kr];
            T *dst = out + k * ldo + x;
            if (vec_ok && x + VEC <= S.X) {
                vstore(dst, w);
            } else {
#pragma unroll
                for (int q = 0; q < VEC; ++q)
                    if (x + q < S.X) dst[q] = w[q];
            }
        }
    }
}

// ------------------------------------------------------------------ pack along x
// out[k][i*P + j] for j in [j0, j0 + 32) of row block i, k in [k0, k0 + 32)
template <typename T, int W>
__global__ void __launch_bounds__(256) pack_x_kernel(Src<T> S, int P, const DevPlan *plan,
                                                     int expectW, int wsign, T *out,
                                                     long long ldo) {
    pdl_entry();
    if (expectW > 0 && plan->W != expectW) return;
    constexpr int NX = TILE * W;
    constexpr int PITCH = TILE + 1;
    __shared__ T s[NX * PITCH];
    __shared__ T ccol[TILE];
    const T w = W > 1 ? pack_weight<T>(plan, wsign) : T(1);
    const bool compand = S.c != nullptr;
    const int L = S.L;
    const int jt = (P + TILE - 1) / TILE;
    const int nM = (int)((S.X + L - 1) / L);
    const long long kt = (S.K + TILE - 1) / TILE;
    const long long tiles = (long long)nM * jt * kt;
    for (long long t = blockIdx.x; t < tiles; t += gridDim.x) {
        const long long ktile = t % kt;
        const long long r = t / kt;
        const int i = (int)(r / jt), j0 = (int)(r % jt) * TILE;
        const long long k0 = ktile * TILE;
        const long long xblk0 = (long long)i * L;
        const long long xlim = min(xblk0 + L, S.X);
        const long long x0 = xblk0 + (long long)W * j0;
        __syncthreads();
        if (threadIdx.x < TILE) {
            const long long k = k0 + threadIdx.x;
            ccol[threadIdx.x] = (compand && k < S.K) ? S.c[(long long)i * S.cx + (k / L) * S.cl] : T(1);
        }
        __syncthreads();
        if (S.sk == 1) {
            for (int e = threadIdx.x; e < NX * TILE; e += blockDim.x) {
                const int xr = e / TILE, kc = e % TILE;
                const long long x = x0 + xr, k = k0 + kc;
                const bool valid = x < xlim && k < S.K;
                s[xr * PITCH + kc] = valid ? quant(S.p[x * S.sx + k], ccol[kc], compand) : T(0);
            }
        } else {
            for (int e = threadIdx.x; e < NX * TILE; e += blockDim.x) {
                const int kc = e / NX, xr = e % NX;
                const long long x = x0 + xr, k = k0 + kc;
                const bool valid = x < xlim && k < S.K;
                s[xr * PITCH + kc] = valid ? quant(S.p[x + k * S.sk], ccol[kc], compand) : T(0);
            }
        }
        __syncthreads();
        for (int e = threadIdx.x; e < TILE * TILE; e += blockDim.x) {
            const int kr = e / TILE, jr = e % TILE;
            const int j = j0 + jr;
            const long long k = k0 + kr;
            if (j >= P || k >= S.K) continue;
            const T *d = s + (jr * W) * PITCH + kr;
            T acc = d[(W - 1) * PITCH];
#pragma unroll
            for (int ii = W - 2; ii >= 0; --ii) acc = fma_t(w, acc, d[ii * PITCH]);
            out[k * ldo + (long long)i * P + j] = acc;
        }
    }
}

// ------------------------------------------------------------------ k-major codes
// out[x][k] as integer-valued fp16 or E4M3; the compander of a 64 x 64 tile
// is one value (tiles are 64-aligned and L % 64 == 0)
template <int FP8>
__device__ inline void encode8(const float *v, unsigned char *dst) {
    if constexpr (FP8) {
        uint2 w;
        uint32_t b[8];
#pragma unroll
        for (int i = 0; i < 8; ++i) b[i] = __nv_cvt_float_to_fp8(v[i], __NV_SATFINITE, __NV_E4M3);
        w.x = b[0] | (b[1] << 8) | (b[2] << 16) | (b[3] << 24);
        w.y = b[4] | (b[5] << 8) | (b[6] << 16) | (b[7] << 24);
        *reinterpret_cast<uint2 *>(dst) = w;
    } else {
        __half h[8];
#pragma unroll
        for (int i = 0; i < 8; ++i) h[i] = __float2half_rn(rintf(v[i]));
        *reinterpret_cast<uint4 *>(dst) = *reinterpret_cast<const uint4 *>(h);
    }
}

// k contiguous in the input: one item = 8 consecutive k of one row x
template <int FP8>
__global__ void __launch_bounds__(256) codes_kc_kernel(Src<float> S, unsigned char *out,
                                                       long long ldo, int vec_ok) {
    pdl_entry();
    constexpr int ES = FP8 ? 1 : 2;
    const long long nk8 = (S.K + 7) / 8;
    const long long items = S.X * nk8;
    for (long long it = (long long)blockIdx.x * blockDim.x + threadIdx.x; it < items;
         it += (long long)gridDim.x * blockDim.x) {
        const long long x = it / nk8, k = (it - x * nk8) * 8;
        const float c = S.c[(x / S.L) * S.cx + (k / S.L) * S.cl];
        const float *src = S.p + x * S.sx + k;
        float v[8];
        if (vec_ok && k + 8 <= S.K) {
            float4 a = __ldg(reinterpret_cast<const float4 *>(src));
            float4 b = __ldg(reinterpret_cast<const float4 *>(src + 4));
            v[0] = a.x; v[1] = a.y; v[2] = a.z; v[3] = a.w;
            v[4] = b.x; v[5] = b.y; v[6] = b.z; v[7] = b.w;
        } else {
#pragma unroll
            for (int i = 0; i < 8; ++i) v[i] = (k + i < S.K) ? src[i] : 0.f;
        }
#pragma unroll
        for (int i = 0; i < 8; ++i) v[i] = __fmul_rn(v[i], c);
        unsigned char *dst = out + (x * ldo + k) * ES;
        if (k + 8 <= ldo) {
            encode8<FP8>(v, dst);   // ldo is padded to 128: the tail lands in padding
        }
    }
}

// x contiguous in the input: 64 x 64 tiles transposed through shared memory
// (s[k][x], pitch 65: the row-wise writes and the column-wise reads of the
// store phase are free of bank conflicts).  A thread issues its four 16-byte
// loads of a tile before it uses any of them.  256 threads per CTA.
template <int FP8>
__global__ void __launch_bounds__(256) codes_xc_kernel(Src<float> S, unsigned char *out,
                                                       long long ldo, int vec_ok) {
    pdl_entry();
    constexpr int ES = FP8 ? 1 : 2;
    constexpr int T64 = 64;
    constexpr int PITCH = T64 + 1;               // floats
    constexpr int NLD = T64 * (T64 / 4) / 256;   // float4 loads per thread and tile
    constexpr int NST = T64 * (T64 / 8) / 256;   // 8-value stores per thread and tile
    __shared__ float s[T64 * PITCH];             // s[k][x]
    const long long xt = (S.X + T64 - 1) / T64, kt = (S.K + T64 - 1) / T64;
    for (long long t = blockIdx.x; t < xt * kt; t += gridDim.x) {
        const long long x0 = (t % xt) * T64, k0 = (t / xt) * T64;
        const float c = S.c[(x0 / S.L) * S.cx + (k0 / S.L) * S.cl];
        float v[NLD][4];
#pragma unroll
        for (int u = 0; u < NLD; ++u) {
            const int e = threadIdx.x + u * 256;
            const int kr = e / (T64 / 4), xc = (e % (T64 / 4)) * 4;
            const long long k = k0 + kr, x = x0 + xc;
            if (k < S.K && vec_ok && x + 4 <= S.X) {
                const float4 a = __ldg(reinterpret_cast<const float4 *>(S.p + k * S.sk + x));
                v[u][0] = a.x; v[u][1] = a.y; v[u][2] = a.z; v[u][3] = a.w;
            } else {
#pragma unroll
                for (int i = 0; i < 4; ++i)
                    v[u][i] = (k < S.K && x + i < S.X) ? S.p[k * S.sk + x + i] : 0.f;
            }
        }
        __syncthreads();   // the previous tile's readers are done with s
#pragma unroll
        for (int u = 0; u < NLD; ++u) {
            const int e = threadIdx.x + u * 256;
            const int kr = e / (T64 / 4), xc = (e % (T64 / 4)) * 4;
#pragma unroll
            for (int i = 0; i < 4; ++i) s[kr * PITCH + xc + i] = __fmul_rn(v[u][i], c);
        }
        __syncthreads();
        // store: rows x, 8 k per item
#pragma unroll
        for (int u = 0; u < NST; ++u) {
            const int e = threadIdx.x + u * 256;
            const int xr = e / (T64 / 8), kc = (e % (T64 / 8)) * 8;
            const long long x = x0 + xr, k = k0 + kc;
            if (x >= S.X || k >= ldo) continue;
            float w[8];
#pragma unroll
            for (int i = 0; i < 8; ++i) w[i] = (k + i < S.K) ? s[(kc + i) * PITCH + xr] : 0.f;
            encode8<FP8>(w, out + (x * ldo + k) * ES);
        }
    }
}

// ------------------------------------------------------------------ fused statistics + codes
// The tensor-core forms with companders that depend only on the block's own
// maximum (fixed bits: c = gamma / max|x|; E4M3: c = 448 / max|x|): one CTA
// per L x L block of op(X) (L <= 128) reads the block once, keeps it in
// registers, reduces max|x| (exact) and sum x^2 (double-float, as the
// statistics kernel does), sets c (fp64, rounded to fp32) and s = 1/c, and
// writes the block's codes out[x][k] -- the statistics pass, the compander
// kernel and the code pass of the general path in one read of the input.
struct FusedOp {
    Src<float> S;
    long long nbx, nbk;             // blocks along x and k
    double *mx, *var;               // per block, index bi * S.cx + bk * S.cl
    float *c;
    double *s;
    unsigned char *out;
};

__device__ inline void df_add2(float &hi, float &lo, float bh, float bl) {
    const float s = __fadd_rn(hi, bh);
    const float v = __fsub_rn(s, hi);
    const float e = __fadd_rn(__fsub_rn(hi, __fsub_rn(s, v)), __fsub_rn(bh, v));
    const float t = __fadd_rn(e, __fadd_rn(lo, bl));
    hi = __fadd_rn(s, t);
    lo = __fsub_rn(t, __fsub_rn(hi, s));
}

// exact square as hi + err (TwoProduct), TwoSum into (hi, lo)
__device__ inline void df_add_sq(float &hi, float &lo, float x) {
    const float p = __fmul_rn(x, x);
    const float e = __fmaf_rn(x, x, -p);
    const float t = __fadd_rn(hi, p);
    const float bp = __fsub_rn(t, hi);
    const float err = __fadd_rn(__fsub_rn(hi, __fsub_rn(t, bp)), __fsub_rn(p, bp));
    hi = t;
    lo = __fadd_rn(lo, __fadd_rn(err, e));
}

constexpr int kFusedThreads = 512;   // 32 values per thread at L = 128 (two CTAs, 32 warps per SM)

// block statistics of the values this thread holds, reduced over the CTA;
// thread 0 writes them with the compander, every thread returns c
template <int NVAL>
__device__ inline float fused_block_companders(const float (&v)[NVAL], const FusedOp &o,
                                               long long bx, long long bk, int xn, int kn,
                                               double gamma, DevPlan *plan) {
    __shared__ float red_h[32], red_l[32];
    __shared__ unsigned int red_m[32];
    __shared__ int red_b[32];
    __shared__ float c_sh;
    float hi = 0.f, lo = 0.f;
    unsigned int mb = 0;
    int bad = 0;
#pragma unroll
    for (int u = 0; u < NVAL; ++u) {
        const unsigned int b = __float_as_uint(v[u]) & 0x7fffffffu;
        mb = max(mb, b);
        bad |= (b >= 0x7f800000u);
        df_add_sq(hi, lo, v[u]);
    }
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    auto warp_reduce = [&]() {
#pragma unroll
        for (int off = 16; off > 0; off >>= 1) {
            const float oh = __shfl_xor_sync(0xffffffffu, hi, off);
            const float ol = __shfl_xor_sync(0xffffffffu, lo, off);
            df_add2(hi, lo, oh, ol);
            mb = max(mb, __shfl_xor_sync(0xffffffffu, mb, off));
            bad |= __shfl_xor_sync(0xffffffffu, bad, off);
        }
    };
    warp_reduce();
    if (lane == 0) { red_h[warp] = hi; red_l[warp] = lo; red_m[warp] = mb; red_b[warp] = bad; }
    __syncthreads();
    if (warp == 0) {
        const bool in = lane < kFusedThreads / 32;
        hi = in ? red_h[lane] : 0.f;
        lo = in ? red_l[lane] : 0.f;
        mb = in ? red_m[lane] : 0u;
        bad = in ? red_b[lane] : 0;
        warp_reduce();
        if (lane == 0) {
            const double m = (double)__uint_as_float(mb);
            const long long idx = bx * o.S.cx + bk * o.S.cl;
            // eq. 3's compander: c = gamma / max|x| in fp64, rounded to fp32
            const double c = m > 0.0 ? __ddiv_rn(gamma, m) : 0.0;
            o.mx[idx] = m;
            o.var[idx] = ((double)hi + (double)lo) / ((double)xn * (double)kn);
            o.c[idx] = (float)c;
            o.s[idx] = c > 0.0 ? __ddiv_rn(1.0, c) : 0.0;
            c_sh = (float)c;
            if (bad) atomicExch(&plan->nonfinite, 1);
        }
    }
    __syncthreads();
    return c_sh;
}

template <int FP8, int L>
__global__ void __launch_bounds__(kFusedThreads, 2)
    codes_stats_kernel(FusedOp A, FusedOp B, long long nblkA, double gamma, long long ldo,
                       DevPlan *plan) {
    pdl_entry();
    constexpr int ES = FP8 ? 1 : 2;
    constexpr int NV = L * L / kFusedThreads;    // values per thread: 32 at L = 128
    extern __shared__ float s_tile[];            // x-contiguous inputs: s[k][x], pitch L + 1
    const bool isA = (long long)blockIdx.x < nblkA;
    const FusedOp &o = isA ? A : B;
    const long long blk = isA ? (long long)blockIdx.x : (long long)blockIdx.x - nblkA;
    const long long bx = blk / o.nbk, bk = blk - bx * o.nbk;
    const Src<float> &S = o.S;
    const long long x0 = bx * L, k0 = bk * L;
    const int xn = (int)min((long long)L, S.X - x0), kn = (int)min((long long)L, S.K - k0);
    float v[NV];
    if (S.sk == 1) {
        // k contiguous: item = 8 consecutive k of one row x, loaded, counted
        // and encoded by the same thread
#pragma unroll
        for (int u = 0; u < NV / 8; ++u) {
            const int e = threadIdx.x + u * kFusedThreads;
            const int xr = e / (L / 8), kr = (e % (L / 8)) * 8;
            const float *src = S.p + (x0 + xr) * S.sx + k0 + kr;
            const bool full = xr < xn && kr + 8 <= kn && ((reinterpret_cast<uintptr_t>(src) & 15) == 0);
            if (full) {
                const float4 a = __ldg(reinterpret_cast<const float4 *>(src));
                const float4 b = __ldg(reinterpret_cast<const float4 *>(src + 4));
                v[8 * u] = a.x; v[8 * u + 1] = a.y; v[8 * u + 2] = a.z; v[8 * u + 3] = a.w;
                v[8 * u + 4] = b.x; v[8 * u + 5] = b.y; v[8 * u + 6] = b.z; v[8 * u + 7] = b.w;
            } else {
#pragma unroll
                for (int i = 0; i < 8; ++i)
                    v[8 * u + i] = (xr < xn && kr + i < kn) ? src[i] : 0.f;
            }
        }
        const float c = fused_block_companders(v, o, bx, bk, xn, kn, gamma, plan);
#pragma unroll
        for (int u = 0; u < NV / 8; ++u) {
            const int e = threadIdx.x + u * kFusedThreads;
            const int xr = e / (L / 8), kr = (e % (L / 8)) * 8;
            const long long k = k0 + kr;
            if (xr >= xn || k >= ldo) continue;
            float w[8];
#pragma unroll
            for (int i = 0; i < 8; ++i) w[i] = __fmul_rn(v[8 * u + i], c);
            encode8<FP8>(w, o.out + ((x0 + xr) * ldo + k) * ES);
        }
    } else {
        // x contiguous: 4 consecutive x of one row k per load, transposed
        // through shared memory for the k-contiguous codes
        constexpr int P = L + 1;
#pragma unroll
        for (int u = 0; u < NV / 4; ++u) {
            const int e = threadIdx.x + u * kFusedThreads;
            const int kr = e / (L / 4), xr = (e % (L / 4)) * 4;
            const float *src = S.p + (k0 + kr) * S.sk + x0 + xr;
            const bool full = kr < kn && xr + 4 <= xn && ((reinterpret_cast<uintptr_t>(src) & 15) == 0);
            if (full) {
                const float4 a = __ldg(reinterpret_cast<const float4 *>(src));
                v[4 * u] = a.x; v[4 * u + 1] = a.y; v[4 * u + 2] = a.z; v[4 * u + 3] = a.w;
            } else {
#pragma unroll
                for (int i = 0; i < 4; ++i)
                    v[4 * u + i] = (kr < kn && xr + i < xn) ? src[i] : 0.f;
            }
        }
        const float c = fused_block_companders(v, o, bx, bk, xn, kn, gamma, plan);
#pragma unroll
        for (int u = 0; u < NV / 4; ++u) {
            const int e = threadIdx.x + u * kFusedThreads;
            const int kr = e / (L / 4), xr = (e % (L / 4)) * 4;
#pragma unroll
            for (int i = 0; i < 4; ++i) s_tile[kr * P + xr + i] = v[4 * u + i];
        }
        __syncthreads();
        // items: 8 consecutive k of one row x, lanes along x (conflict-free
        // reads), encoded into the code tile cs[x][k] (row pitch CP bytes:
        // the lanes' 8- or 16-byte writes fall in distinct banks) ...
        constexpr int CP = FP8 ? L + 8 : 2 * L + 16;
        unsigned char *cs = reinterpret_cast<unsigned char *>(s_tile + L * P);
        for (int e = threadIdx.x; e < L * L / 8; e += kFusedThreads) {
            const int xr = e % L, kr = (e / L) * 8;
            float w[8];
#pragma unroll
            for (int i = 0; i < 8; ++i) w[i] = __fmul_rn(s_tile[(kr + i) * P + xr], c);
            encode8<FP8>(w, cs + xr * CP + kr * ES);
        }
        __syncthreads();
        // ... and copied out row by row: consecutive lanes write consecutive
        // 8 bytes (E4M3) or 16 bytes (fp16) of one row of codes
        constexpr int UB = FP8 ? 8 : 16;             // bytes per unit
        constexpr int UPR = L * ES / UB;             // units per row of the tile
        for (int e = threadIdx.x; e < L * UPR; e += kFusedThreads) {
            const int xr = e / UPR, u = e % UPR;
            const long long k = k0 + (long long)u * (UB / ES);
            if (xr >= xn || k >= ldo) continue;
            unsigned char *dst = o.out + ((x0 + xr) * ldo + k) * ES;
            if constexpr (FP8)
                *reinterpret_cast<uint2 *>(dst) = *reinterpret_cast<const uint2 *>(cs + xr * CP + u * UB);
            else
                *reinterpret_cast<uint4 *>(dst) = *reinterpret_cast<const uint4 *>(cs + xr * CP + u * UB);
        }
    }
}

// dynamic shared memory of codes_stats_kernel for x-contiguous inputs: the
// fp32 tile s[k][x] (pitch L + 1) and the code tile (pitch L + 8 or 2 L + 16 bytes)
constexpr size_t fused_xc_smem(int fp8, int L) {
    return (size_t)L * (L + 1) * sizeof(float) + (size_t)L * (fp8 ? L + 8 : 2 * L + 16);
}

template <typename T>
Src<T> make_src(const PackOperand<T> &o) {
    Src<T> S;
    S.p = o.src; S.sx = o.sx; S.sk = o.sk; S.X = o.X; S.K = o.K;
    S.c = o.c; S.cx = o.cx; S.cl = o.cl; S.L = o.L;
    return S;
}

int capped(long long n) { return (int)max(1LL, min(n, (long long)MAX_CTAS)); }

// Grid of at most `waves` full waves of resident CTAs for `kern` (occupancy
// x SMs, cached per device and kernel under a lock, since host threads may
// launch concurrently), so a grid-stride kernel never ends on a partial wave
// of long-running CTAs and an early exit costs few CTAs.
int resident_grid(const void *kern, long long n, int waves) {
    struct Entry { const void *k; int dev, ctas; };
    static Entry cache[128];
    static int ncache = 0;
    static std::mutex mu;
    int dev = 0;
    cudaGetDevice(&dev);
    int ctas = 0;
    {
        std::lock_guard<std::mutex> lock(mu);
        for (int i = 0; i < ncache; ++i)
            if (cache[i].k == kern && cache[i].dev == dev) ctas = cache[i].ctas;
    }
    if (!ctas) {
        int sms = 0, per = 0;
        cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
        if (sms <= 0) sms = 1;
        if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per, kern, 256, 0) != cudaSuccess || per < 1)
            per = 1;
        ctas = per * sms;
        std::lock_guard<std::mutex> lock(mu);
        if (ncache < 128) cache[ncache++] = {kern, dev, ctas};
    }
    return (int)max(1LL, min(n, (long long)ctas * waves));
}

template <typename T, int W>
cudaError_t launch_pack_k_w(const PackOperand<T> &o, const DevPlan *plan, int expectW, int wsign,
                            T *out, long long ldo, long long rows_out, cudaStream_t st) {
    constexpr int VEC = VecT<T>::n;
    Src<T> S = make_src(o);
    const int P = (o.L + W - 1) / W;
    const bool aligned_in = ((uintptr_t)o.src % 16 == 0);
    const bool aligned_out = ((uintptr_t)out % 16 == 0) && (ldo % VEC == 0);
    if (o.sx == 1) {
        const int vec_ok = aligned_in && aligned_out && (o.sk % VEC == 0);
        const long long items = rows_out * ((o.X + VEC - 1) / VEC);
        return launch_pdl(pack_k_xc_kernel<T, W>,
                          dim3(resident_grid((const void *)pack_k_xc_kernel<T, W>,
                                             (items + 255) / 256, 4)),
                          dim3(256), 0, st, S, P, plan, expectW, wsign, out, ldo, rows_out,
                          vec_ok);
    } else if (W == 1 && o.c == nullptr && o.sk == 1 && rows_out == o.K) {
        // plain copy: a straight transpose
        const int vec_ok = aligned_in && aligned_out && (o.sx % VEC == 0);
        const long long tiles = ((o.X + 63) / 64) * ((o.K + 63) / 64);
        return launch_pdl(transpose_copy_kernel<T>, dim3(capped(tiles)), dim3(256), 0, st, S, plan,
                          expectW, out, ldo, vec_ok);
    } else {
        const int vec_ok = aligned_in && (o.sx % VEC == 0) && o.sk == 1;
        constexpr int TK = kc_tile<T, W>();
        const long long tiles = ((o.X + TK - 1) / TK) * ((o.K + o.L - 1) / o.L) *
                                ((P + TK - 1) / TK);
        return launch_pdl(pack_k_kc_kernel<T, W>,
                          dim3(resident_grid((const void *)pack_k_kc_kernel<T, W>, tiles, 4)),
                          dim3(256), 0, st, S, P, plan, expectW, wsign, out, ldo, rows_out,
                          vec_ok);
    }
    return cudaGetLastError();
}

template <typename T, int W>
cudaError_t launch_pack_x_w(const PackOperand<T> &o, const DevPlan *plan, int expectW, int wsign,
                            T *out, long long ldo, cudaStream_t st) {
    Src<T> S = make_src(o);
    const int P = (o.L + W - 1) / W;
    const long long tiles = ((o.X + o.L - 1) / o.L) * ((P + TILE - 1) / TILE) *
                            ((o.K + TILE - 1) / TILE);
    return launch_pdl(pack_x_kernel<T, W>, dim3(capped(tiles)), dim3(256), 0, st, S, P, plan,
                      expectW, wsign, out, ldo);
    return cudaGetLastError();
}

}  // namespace

// The symmetric form's two packs (A with wsign -1, B with +1): one launch of
// pack_k_pair_kernel when A is k-contiguous and B x-contiguous, else B's pack
// and then A's.
template <typename T, int W>
cudaError_t launch_pack_k_pair_w(const PackOperand<T> &a, const PackOperand<T> &b,
                                 const DevPlan *plan, int expectW, T *outA, long long ldoA,
                                 long long rowsA, T *outB, long long ldoB, long long rowsB,
                                 cudaStream_t st) {
    constexpr int VEC = VecT<T>::n;
    const bool a_copy = W == 1 && a.c == nullptr && a.sk == 1 && rowsA == a.K;
    if (a.sx == 1 || a_copy || b.sx != 1) {
        cudaError_t e = launch_pack_k_w<T, W>(b, plan, expectW, +1, outB, ldoB, rowsB, st);
        if (e != cudaSuccess) return e;
        return launch_pack_k_w<T, W>(a, plan, expectW, -1, outA, ldoA, rowsA, st);
    }
    Src<T> SA = make_src(a), SB = make_src(b);
    const int P = (a.L + W - 1) / W;
    const int vecA = ((uintptr_t)a.src % 16 == 0) && (a.sx % VEC == 0) && a.sk == 1;
    const int vecB = ((uintptr_t)b.src % 16 == 0) && ((uintptr_t)outB % 16 == 0) &&
                     (ldoB % VEC == 0) && (b.sk % VEC == 0);
    constexpr int TK = kc_tile<T, W>();
    const long long tilesA = ((a.X + TK - 1) / TK) * ((a.K + a.L - 1) / a.L) * ((P + TK - 1) / TK);
    const long long blocksB = (rowsB * ((b.X + VEC - 1) / VEC) + 255) / 256;
    const void *kern = (const void *)pack_k_pair_kernel<T, W>;
    const long long gA = resident_grid(kern, tilesA, 2);
    const long long gB = resident_grid(kern, blocksB, 2);
    return launch_pdl(pack_k_pair_kernel<T, W>, dim3((unsigned)(gA + gB)), dim3(256), 0, st, SA,
                      SB, P, plan, expectW, outA, ldoA, rowsA, vecA, outB, ldoB, rowsB, vecB,
                      gA, gB);
}

template <typename T>
cudaError_t launch_pack_k_pair(const PackOperand<T> &a, const PackOperand<T> &b, int W,
                               const DevPlan *plan, int expectW, T *outA, long long ldoA,
                               long long rowsA, T *outB, long long ldoB, long long rowsB,
                               cudaStream_t st) {
    switch (W) {
        case 1: return launch_pack_k_pair_w<T, 1>(a, b, plan, expectW, outA, ldoA, rowsA, outB, ldoB, rowsB, st);
        case 2: return launch_pack_k_pair_w<T, 2>(a, b, plan, expectW, outA, ldoA, rowsA, outB, ldoB, rowsB, st);
        case 3: return launch_pack_k_pair_w<T, 3>(a, b, plan, expectW, outA, ldoA, rowsA, outB, ldoB, rowsB, st);
        case 4: return launch_pack_k_pair_w<T, 4>(a, b, plan, expectW, outA, ldoA, rowsA, outB, ldoB, rowsB, st);
    }
    return cudaErrorInvalidValue;
}

template <typename T>
cudaError_t launch_pack_k(const PackOperand<T> &o, int W, const DevPlan *plan, int expectW,
                          int wsign, T *out, long long ldo, long long rows_out, cudaStream_t st) {
    switch (W) {
        case 1: return launch_pack_k_w<T, 1>(o, plan, expectW, wsign, out, ldo, rows_out, st);
        case 2: return launch_pack_k_w<T, 2>(o, plan, expectW, wsign, out, ldo, rows_out, st);
        case 3: return launch_pack_k_w<T, 3>(o, plan, expectW, wsign, out, ldo, rows_out, st);
        case 4: return launch_pack_k_w<T, 4>(o, plan, expectW, wsign, out, ldo, rows_out, st);
    }
    return cudaErrorInvalidValue;
}

template <typename T>
cudaError_t launch_pack_x(const PackOperand<T> &o, int W, const DevPlan *plan, int expectW,
                          int wsign, T *out, long long ldo, cudaStream_t st) {
    switch (W) {
        case 1: return launch_pack_x_w<T, 1>(o, plan, expectW, wsign, out, ldo, st);
        case 2: return launch_pack_x_w<T, 2>(o, plan, expectW, wsign, out, ldo, st);
        case 3: return launch_pack_x_w<T, 3>(o, plan, expectW, wsign, out, ldo, st);
        case 4: return launch_pack_x_w<T, 4>(o, plan, expectW, wsign, out, ldo, st);
    }
    return cudaErrorInvalidValue;
}

cudaError_t launch_codes(const PackOperand<float> &o, int fp8, void *out, long long ldo,
                         cudaStream_t st) {
    Src<float> S = make_src(o);
    unsigned char *ob = reinterpret_cast<unsigned char *>(out);
    const bool aligned = ((uintptr_t)o.src % 16 == 0) && ((uintptr_t)out % 16 == 0) && ldo % 8 == 0;
    if (o.sk == 1) {
        const int vec_ok = aligned && (o.sx % 4 == 0);
        const long long items = o.X * ((o.K + 7) / 8);
        const int g = capped((items + 255) / 256);
        return fp8 ? launch_pdl(codes_kc_kernel<1>, dim3(g), dim3(256), 0, st, S, ob, ldo, vec_ok)
                   : launch_pdl(codes_kc_kernel<0>, dim3(g), dim3(256), 0, st, S, ob, ldo, vec_ok);
    } else {
        const int vec_ok = aligned && o.sx == 1 && (o.sk % 4 == 0);
        const long long tiles = ((o.X + 63) / 64) * ((o.K + 63) / 64);
        const int g = capped(tiles);
        return fp8 ? launch_pdl(codes_xc_kernel<1>, dim3(g), dim3(256), 0, st, S, ob, ldo, vec_ok)
                   : launch_pdl(codes_xc_kernel<0>, dim3(g), dim3(256), 0, st, S, ob, ldo, vec_ok);
    }
    return cudaGetLastError();
}

cudaError_t launch_codes_stats(const PackOperand<float> &a, double *mxA, double *varA,
                               float *cA, double *sA, void *outA, const PackOperand<float> *b,
                               double *mxB, double *varB, float *cB, double *sB, void *outB,
                               int fp8, double gamma, long long ldo, DevPlan *plan,
                               cudaStream_t st) {
    const int L = a.L;
    if (L > 128 || L % 64) return cudaErrorInvalidValue;
    auto op = [&](const PackOperand<float> &o, double *mx, double *var, float *c, double *s,
                  void *out) {
        FusedOp f;
        f.S = make_src(o);
        f.nbx = (o.X + L - 1) / L;
        f.nbk = (o.K + L - 1) / L;
        f.mx = mx; f.var = var; f.c = c; f.s = s;
        f.out = reinterpret_cast<unsigned char *>(out);
        return f;
    };
    FusedOp fa = op(a, mxA, varA, cA, sA, outA);
    FusedOp fb = b ? op(*b, mxB, varB, cB, sB, outB) : fa;
    const long long na = fa.nbx * fa.nbk, nb = b ? fb.nbx * fb.nbk : 0;
    if (na + nb > 0x7fffffffLL) return cudaErrorInvalidConfiguration;
    const bool xc = a.sk != 1 || (b && b->sk != 1);
    const size_t smem = xc ? fused_xc_smem(fp8, L) : 0;
    auto kern = L == 128 ? (fp8 ? codes_stats_kernel<1, 128> : codes_stats_kernel<0, 128>)
                         : (fp8 ? codes_stats_kernel<1, 64> : codes_stats_kernel<0, 64>);
    static std::once_flag attr_once;
    cudaError_t attr_err = cudaSuccess;
    std::call_once(attr_once, [&]() {
        // the L = 128 tiles need 82-99 KB of dynamic shared memory
        for (int f8 = 0; f8 < 2; ++f8) {
            cudaError_t e = cudaFuncSetAttribute(f8 ? codes_stats_kernel<1, 128> : codes_stats_kernel<0, 128>,
                                                 cudaFuncAttributeMaxDynamicSharedMemorySize,
                                                 (int)fused_xc_smem(f8, 128));
            if (e != cudaSuccess) attr_err = e;
        }
    });
    if (attr_err != cudaSuccess) return attr_err;
    return launch_pdl(kern, dim3((unsigned)(na + nb)), dim3(kFusedThreads), smem, st, fa, fb, na,
                      gamma, ldo, plan);
}

template cudaError_t launch_pack_k_pair<float>(const PackOperand<float> &, const PackOperand<float> &,
                                               int, const DevPlan *, int, float *, long long,
                                               long long, float *, long long, long long,
                                               cudaStream_t);
template cudaError_t launch_pack_k_pair<double>(const PackOperand<double> &,
                                                const PackOperand<double> &, int,
                                                const DevPlan *, int, double *, long long,
                                                long long, double *, long long, long long,
                                                cudaStream_t);
template cudaError_t launch_pack_k<float>(const PackOperand<float> &, int, const DevPlan *, int, int,
                                          float *, long long, long long, cudaStream_t);
template cudaError_t launch_pack_k<double>(const PackOperand<double> &, int, const DevPlan *, int,
                                           int, double *, long long, long long, cudaStream_t);
template cudaError_t launch_pack_x<float>(const PackOperand<float> &, int, const DevPlan *, int, int,
                                          float *, long long, cudaStream_t);
template cudaError_t launch_pack_x<double>(const PackOperand<double> &, int, const DevPlan *, int,
                                           int, double *, long long, cudaStream_t);

}  // namespace tdg
