// Steps (a) and (b) on the data: companding and rounding (eq. 3) fused with
// packing (eqs. 6, 7, 11) in one pass over each input.
//
// Each CTA stages a tile of op(X) in shared memory with loads that are
// coalesced along whichever stored dimension is contiguous, quantizes it on
// the way in (a~ = rint(fl_T(x * c_T)) with the block's compander), and writes
// packed numbers by Horner's rule,
//     acc = d_{W-1};  acc = fma(w, acc, d_i),  i = W-2 .. 0,
// coalesced along the output's contiguous dimension.  Digits outside the
// L x L block or the matrix are zero (border clean-up, Sec. 2).
//
//   pack along k   (eq. 6 with w = z for A, eq. 7 with w = z^-1 for B, and
//                   W = 1 for the unpacked operands):  out[l P + j][x]
//   pack along x   (eq. 11, asymmetric A, w = z):       out[k][i P + j]
//   k-major codes  (tensor-core forms): out[x][k] as integer-valued fp16 or
//                   as E4M3 (c = 448 / max|x|, round to nearest even,
//                   saturating)
// P = ceil(L / W) packed numbers per block (zero digits pad a ragged block).
#include <cuda_fp16.h>
#include <cuda_fp8.h>

#include "tdg_common.cuh"
#include "tdg_internal.h"

namespace tdg {

namespace {

constexpr int TILE = 32;

// op(X)[x][k] lives at src[x * sx + k * sk]; its compander (if any) at
// c[(x / L) * cx + (k / L) * cl].
template <typename T>
struct Src {
    const T *p;
    long long sx, sk;
    long long X, K;
    const T *c;       // nullptr: copy without companding
    long long cx, cl;
    int L;
    __device__ inline T load_q(long long x, long long k) const {
        if (x >= X || k >= K) return T(0);
        T v = p[x * sx + k * sk];
        if (c == nullptr) return v;
        T ct = c[(x / L) * cx + (k / L) * cl];
        if constexpr (sizeof(T) == 4) return rintf(__fmul_rn(v, ct));
        else return rint(__dmul_rn(v, ct));
    }
};

// w = z = 2^-q (wsign < 0) or z^-1 = 2^q (wsign > 0), q from the device plan
template <typename T>
__device__ inline T pack_weight(const DevPlan *plan, int wsign) {
    int q = plan->q;
    if constexpr (sizeof(T) == 4) return scalbnf(1.0f, wsign < 0 ? -q : q);
    else return scalbn(1.0, wsign < 0 ? -q : q);
}

template <typename T>
__device__ inline T fma_t(T a, T b, T c) {
    if constexpr (sizeof(T) == 4) return __fmaf_rn(a, b, c);
    else return __fma_rn(a, b, c);
}

// Load a (nx x nk) region of op(X) starting at (x0, k0) into s[xr][kc]
// (row pitch `pitch`), coalescing along the contiguous stored dimension.
// Elements at or beyond (xlim, klim) are zero.
template <typename T>
__device__ inline void stage_tile(const Src<T> &S, T *s, int pitch, long long x0, long long k0,
                                  int nx, int nk, long long xlim, long long klim) {
    const int n = nx * nk;
    if (S.sk == 1) {
        for (int e = threadIdx.x; e < n; e += blockDim.x) {
            int xr = e / nk, kc = e % nk;
            long long x = x0 + xr, k = k0 + kc;
            s[xr * pitch + kc] = (x < xlim && k < klim) ? S.load_q(x, k) : T(0);
        }
    } else {
        for (int e = threadIdx.x; e < n; e += blockDim.x) {
            int kc = e / nx, xr = e % nx;
            long long x = x0 + xr, k = k0 + kc;
            s[xr * pitch + kc] = (x < xlim && k < klim) ? S.load_q(x, k) : T(0);
        }
    }
}

// out[l*P + j][x] for j in [j0, j0 + 32), x in [x0, x0 + 32)
template <typename T, int W>
__global__ void __launch_bounds__(256) pack_k_kernel(Src<T> S, int P, const DevPlan *plan,
                                                     int expectW, int wsign, T *out,
                                                     long long ldo, long long rows_out) {
    if (plan->W != expectW) return;   // the device planner chose another packing
    const T w = W > 1 ? pack_weight<T>(plan, wsign) : T(1);
    extern __shared__ __align__(16) unsigned char smem_raw[];
    T *s = reinterpret_cast<T *>(smem_raw);
    const int pitch = TILE * W + 1;
    const int L = S.L;
    const int jt = cdiv_i(P, TILE);
    const long long l = blockIdx.y / jt;
    const int j0 = (blockIdx.y % jt) * TILE;
    const long long x0 = (long long)blockIdx.x * TILE;
    const long long kslab0 = l * L;
    const long long klim = min(kslab0 + L, S.K);   // digits stop at the block edge
    const long long k0 = kslab0 + (long long)W * j0;
    stage_tile(S, s, pitch, x0, k0, TILE, TILE * W, S.X, klim);
    __syncthreads();
    for (int e = threadIdx.x; e < TILE * TILE; e += blockDim.x) {
        int jr = e / TILE, xr = e % TILE;
        int j = j0 + jr;
        long long x = x0 + xr;
        if (j >= P || x >= S.X || l * P + j >= rows_out) continue;
        const T *d = s + xr * pitch + jr * W;
        T acc = d[W - 1];
#pragma unroll
        for (int i = W - 2; i >= 0; --i) acc = fma_t(w, acc, d[i]);
        out[(l * P + j) * ldo + x] = acc;
    }
}

// out[k][i*P + j] for j in [j0, j0 + 32) of row block i, k in [k0, k0 + 32)
template <typename T, int W>
__global__ void __launch_bounds__(256) pack_x_kernel(Src<T> S, int P, const DevPlan *plan,
                                                     int expectW, int wsign, T *out,
                                                     long long ldo) {
    if (plan->W != expectW) return;
    const T w = W > 1 ? pack_weight<T>(plan, wsign) : T(1);
    extern __shared__ __align__(16) unsigned char smem_raw[];
    T *s = reinterpret_cast<T *>(smem_raw);
    const int pitch = TILE + 1;
    const int L = S.L;
    const int jt = cdiv_i(P, TILE);
    const long long i = blockIdx.x / jt;
    const int j0 = (blockIdx.x % jt) * TILE;
    const long long k0 = (long long)blockIdx.y * TILE;
    const long long xblk0 = i * L;
    const long long xlim = min(xblk0 + L, S.X);
    const long long x0 = xblk0 + (long long)W * j0;
    stage_tile(S, s, pitch, x0, k0, TILE * W, TILE, xlim, S.K);
    __syncthreads();
    for (int e = threadIdx.x; e < TILE * TILE; e += blockDim.x) {
        int kr = e / TILE, jr = e % TILE;
        int j = j0 + jr;
        long long k = k0 + kr;
        if (j >= P || k >= S.K) continue;
        const T *d = s + (jr * W) * pitch + kr;
        T acc = d[(W - 1) * pitch];
#pragma unroll
        for (int ii = W - 2; ii >= 0; --ii) acc = fma_t(w, acc, d[ii * pitch]);
        out[k * ldo + i * P + j] = acc;
    }
}

// k-major quantized codes for the tensor-core forms: out[x][k]
template <int FP8>
__global__ void __launch_bounds__(256) codes_kernel(Src<float> S, void *out, long long ldo) {
    __shared__ float s[TILE][TILE + 1];
    const long long x0 = (long long)blockIdx.y * TILE, k0 = (long long)blockIdx.x * TILE;
    // stage raw products x*c (rounded in fp32); the integer form rounds below
    if (S.sk == 1) {
        for (int e = threadIdx.x; e < TILE * TILE; e += blockDim.x) {
            int xr = e / TILE, kc = e % TILE;
            long long x = x0 + xr, k = k0 + kc;
            float v = 0.f;
            if (x < S.X && k < S.K)
                v = __fmul_rn(S.p[x * S.sx + k * S.sk], S.c[(x / S.L) * S.cx + (k / S.L) * S.cl]);
            s[xr][kc] = v;
        }
    } else {
        for (int e = threadIdx.x; e < TILE * TILE; e += blockDim.x) {
            int kc = e / TILE, xr = e % TILE;
            long long x = x0 + xr, k = k0 + kc;
            float v = 0.f;
            if (x < S.X && k < S.K)
                v = __fmul_rn(S.p[x * S.sx + k * S.sk], S.c[(x / S.L) * S.cx + (k / S.L) * S.cl]);
            s[xr][kc] = v;
        }
    }
    __syncthreads();
    for (int e = threadIdx.x; e < TILE * TILE; e += blockDim.x) {
        int xr = e / TILE, kc = e % TILE;
        long long x = x0 + xr, k = k0 + kc;
        if (x >= S.X || k >= S.K) continue;
        float v = s[xr][kc];
        if constexpr (FP8) {
            __nv_fp8_storage_t b = __nv_cvt_float_to_fp8(v, __NV_SATFINITE, __NV_E4M3);
            reinterpret_cast<uint8_t *>(out)[x * ldo + k] = b;
        } else {
            reinterpret_cast<__half *>(out)[x * ldo + k] = __float2half_rn(rintf(v));
        }
    }
}

template <typename T>
Src<T> make_src(const PackOperand<T> &o) {
    Src<T> S;
    S.p = o.src; S.sx = o.sx; S.sk = o.sk; S.X = o.X; S.K = o.K;
    S.c = o.c; S.cx = o.cx; S.cl = o.cl; S.L = o.L;
    return S;
}

template <typename T, int W>
cudaError_t launch_pack_k_w(const PackOperand<T> &o, const DevPlan *plan, int expectW, int wsign,
                            T *out, long long ldo, long long rows_out, cudaStream_t st) {
    Src<T> S = make_src(o);
    int P = (o.L + W - 1) / W;
    int nK = cdiv_i(o.K, o.L);
    dim3 grid(cdiv_i(o.X, TILE), nK * cdiv_i(P, TILE));
    size_t sm = (size_t)TILE * (TILE * W + 1) * sizeof(T);
    pack_k_kernel<T, W><<<grid, 256, sm, st>>>(S, P, plan, expectW, wsign, out, ldo, rows_out);
    return cudaGetLastError();
}

template <typename T, int W>
cudaError_t launch_pack_x_w(const PackOperand<T> &o, const DevPlan *plan, int expectW, int wsign,
                            T *out, long long ldo, cudaStream_t st) {
    Src<T> S = make_src(o);
    int P = (o.L + W - 1) / W;
    int nM = cdiv_i(o.X, o.L);
    dim3 grid(nM * cdiv_i(P, TILE), cdiv_i(o.K, TILE));
    size_t sm = (size_t)(TILE * W) * (TILE + 1) * sizeof(T);
    pack_x_kernel<T, W><<<grid, 256, sm, st>>>(S, P, plan, expectW, wsign, out, ldo);
    return cudaGetLastError();
}

}  // namespace

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
    dim3 grid(cdiv_i(o.K, TILE), cdiv_i(o.X, TILE));
    if (fp8) codes_kernel<1><<<grid, 256, 0, st>>>(S, out, ldo);
    else codes_kernel<0><<<grid, 256, 0, st>>>(S, out, ldo);
    return cudaGetLastError();
}

template cudaError_t launch_pack_k<float>(const PackOperand<float> &, int, const DevPlan *, int, int,
                                          float *, long long, long long, cudaStream_t);
template cudaError_t launch_pack_k<double>(const PackOperand<double> &, int, const DevPlan *, int, int,
                                          double *, long long, long long, cudaStream_t);
template cudaError_t launch_pack_x<float>(const PackOperand<float> &, int, const DevPlan *, int, int,
                                          float *, long long, cudaStream_t);
template cudaError_t launch_pack_x<double>(const PackOperand<double> &, int, const DevPlan *, int, int,
                                          double *, long long, cudaStream_t);

}  // namespace tdg
