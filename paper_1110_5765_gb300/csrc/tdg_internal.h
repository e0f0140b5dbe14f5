// Host-side declarations shared by the translation units of the library.
#pragma once

#include <cuda.h>
#include <cuda_runtime.h>
#include <stdint.h>

#include "tdg_common.cuh"

namespace tdg {

enum GemmForm { G_PLAIN = 0, G_SYM = 1, G_ASYM = 2 };

// One operand of a pack kernel: op(X)[x][k] = src[x * sx + k * sk], x < X,
// k < K, with per-block companders c[(x / L) * cx + (k / L) * cl] (nullptr:
// plain copy).
template <typename T>
struct PackOperand {
    const T *src;
    long long sx, sk, X, K;
    const T *c;
    long long cx, cl;
    int L;
};

// Per L x L block max|x| and sigma^2 of op(A) and op(B), one launch.  Each
// operand is given as stored (rows_s x cols_s, leading dimension ld) with
// trans = 1 when op() transposes it; nbc = block columns of op(); results
// go to mx / var at op() block index i * nbc + j.
template <typename T>
cudaError_t launch_block_stats(const T *A, long long rows_a, long long cols_a, long long lda,
                               int trans_a, int nbc_a, double *mxA, double *varA, const T *B,
                               long long rows_b, long long cols_b, long long ldb, int trans_b,
                               int nbc_b, double *mxB, double *varB, int L, DevPlan *plan,
                               cudaStream_t st);

// Planner: per-slab aggregates into agg (4 nK + kLevelRecDoubles (kMaxW - 1)
// kMaxLevels doubles of workspace: the aggregates, then one record per
// candidate (W, level)), the
// choice of W / z / companders into *plan, then c, s per block and the
// de-companding factors.
// scales_done: c and s per block were already written (the fused tensor-core
// path), so the compander kernel is not launched.
template <typename T>
cudaError_t launch_planner(const PlanParams &pp, const double *mA, const double *eA,
                           const double *mB, const double *eB, const double *stab,
                           DevPlan *plan, double *agg, T *cA, double *sA, T *cB, double *sB,
                           T *pair, cudaStream_t st, bool scales_done = false);

// Launch order of the tiles of a mixed (Sec. 6) launch: the tiles of
// unaccelerated inner kernels first, then the accelerated ones, each group in
// row-major order; tile (tm, tn) of the tiles_m x ntn grid of bm x bn tiles
// lies in inner kernel (tm bm / L, tn bn / L).
cudaError_t launch_tile_order(const unsigned char *mask, int nN, int L, int bm, int bn,
                              long long tiles_m, long long ntn, int *order, cudaStream_t st);

// Measured throughput scaling F_W of an accelerated inner kernel over a
// conventional one (Sec. 5.B), by packing W (index 2..4; <= 0: not measured).
struct Speedups {
    double fw[kMaxW + 1];
};

// Sec. 6 inner-kernel control: per-kernel predicted S/N and the mask of
// kernels that run packed (mode 1: S/N >= thr; mode 2: the k best; mode 3:
// the fewest best whose predicted acceleration reaches F through the F_W of
// the packing the device planner chose).
cudaError_t launch_kernel_control(const PlanParams &pp, const double *mA, const double *vA,
                                  const double *mB, const double *vB, const DevPlan *plan,
                                  int mode, double thr, long long k, double F,
                                  const Speedups &fw, double *ratio, unsigned char *mask,
                                  cudaStream_t st);

// Pack kernels run only when the device plan's W equals expectW (expectW = 0:
// always); W is the
// packing of the kernel itself; wsign < 0 packs with z, > 0 with z^-1;
// rows_out bounds the rows written to the k-major output.
template <typename T>
cudaError_t launch_pack_k(const PackOperand<T> &o, int W, const DevPlan *plan, int expectW,
                          int wsign, T *out, long long ldo, long long rows_out, cudaStream_t st);

template <typename T>
cudaError_t launch_pack_x(const PackOperand<T> &o, int W, const DevPlan *plan, int expectW,
                          int wsign, T *out, long long ldo, cudaStream_t st);

cudaError_t launch_codes(const PackOperand<float> &o, int fp8, void *out, long long ldo,
                         cudaStream_t st);

// Tensor-core forms whose compander depends only on the block's own maximum
// (c = gamma / max|x|: fixed bits, or gamma = 448 for E4M3): statistics,
// companders (c in fp32, s = 1/c in fp64) and codes of op(A) and, when b is
// given, op(B) in one launch reading each input once.  L in {64, 128}.
cudaError_t launch_codes_stats(const PackOperand<float> &a, double *mxA, double *varA,
                               float *cA, double *sA, void *outA, const PackOperand<float> *b,
                               double *mxB, double *varB, float *cB, double *sB, void *outB,
                               int fp8, double gamma, long long ldo, DevPlan *plan,
                               cudaStream_t st);

// Arguments of the CUDA-core packed GEMM (steps c and d).
template <typename T>
struct GemmArgs {
    const DevPlan *plan;
    long long M, N, K;      // op sizes
    long long Mrows;        // rows of the A operand's x extent: M, or nM*P (asym)
    long long Krows;        // rows (k) of both operands: nK*P (sym), K (asym, plain)
    int L, P;               // block size, packed numbers per block
    int nM, nK, nN;
    const T *pair;          // [l][i][j] de-companding factors
    T *C;
    long long ldc;
    T alpha, beta;
    int beta_zero;
    T *Rbar;                // nullable: keep packed slab results
    // nullable: Sec. 6 mask per L x L inner kernel (symmetric form only).  A
    // CTA tile whose kernel's mask is 0 computes the conventional product from
    // the plain operands in the same launch.
    const unsigned char *kmask;
    // nullable (with kmask): tile to run for each CTA index, the
    // conventional-product tiles first (they take about W times longer, so
    // starting them first keeps the last wave short)
    const int *tile_order;
    const T *cApx, *cBpx;   // pair-exact companders [(i nK + l) nN + j] (else unused)
    int ntn;                // set by the launcher: tiles per row of the 1-D tile grid
    long long ntiles;       // set by the launcher: tiles in the grid
    // slab splitting (needs Rbar): > 1 asks for that many groups of slabs, each
    // CTA computing one tile over one group and storing its packed slab
    // results; the launcher sets spg (slabs per group) and the final count
    int groups, spg;
    // test of the bounded waits: > 0 makes every CTA's first wait for operand
    // tiles wait on a barrier nothing completes, giving up after this many ns
    long long stall_ns;
    // fp32 symmetric W = 2: whether the second rounding of eq. 10 may use the
    // add-subtract form (|z u| < 2^22, see the kernel): 1 known yes, 0 known
    // no, -1 decided on the device (both variants queued, one runs)
    int small_t;
};

// 2-D TMA map over a row-major [rows][cols] array with leading dimension ld
// (elements), box {box_cols, box_rows}.  CUDA_ERROR_NOT_SUPPORTED when the
// driver entry point is missing, CUDA_ERROR_INVALID_VALUE when the base or
// the row pitch is not 16-byte aligned.
CUresult encode_map_2d(CUtensorMap *m, CUtensorMapDataType dt, size_t esz, const void *base,
                       long long cols, long long rows, long long ld, int box_cols, int box_rows,
                       CUtensorMapSwizzle sw);

// A k-major operand of the CUDA-core GEMM: [rows = k][cols = x], pitch ld.
struct GemmOperand {
    const void *base;
    long long cols, rows, ld;
};
struct GemmOperands {
    GemmOperand a, b;       // the operands of the launch's form
    GemmOperand pa, pb;     // plain op(A)^T and op(B) for mixed tiles (g.kmask)
};

// Builds the tensor maps for its tile shape and launches.  Returns cudaErrorNotSupported when no
// kernel exists for (T, form, W), cudaErrorInvalidValue when an operand
// cannot be mapped.
template <typename T>
cudaError_t launch_packed_gemm(int form, int W, const GemmArgs<T> &g, const GemmOperands &ops,
                               cudaStream_t st);

// Pair-exact companders (eq. 26 per (i, l, j)): c_A, c_B per pair and the
// de-companding factors, then the symmetric product with per-CTA companding
// and packing (one L x L output block per CTA, L = pair_exact_tile(dtype),
// W in {2, 4}, op(A) and op(B) row-major through ops.a = {A, K, M, lda} and
// ops.b = {B, N, K, ldb}).
int pair_exact_tile(int dtype);
int pair_exact_bk();
template <typename T>
cudaError_t launch_px_scales(const PlanParams &pp, const double *mA, const double *vA,
                             const double *mB, const double *vB, const DevPlan *plan, T *cA,
                             T *cB, T *pair, cudaStream_t st);
template <typename T>
cudaError_t launch_px_gemm(int W, const GemmArgs<T> &g, const GemmOperands &ops, cudaStream_t st);

// Tile shape the packed GEMM uses for (T, form): operand boxes are
// {box_x_a, bk} for A and {box_x_b, bk} for B.
void packed_gemm_boxes(int dtype, int form, int W, int *box_x_a, int *box_x_b, int *bk);

template <typename T>
cudaError_t launch_unpack(int form, int W, const GemmArgs<T> &g, int64_t *rint_out,
                          cudaStream_t st);

// store a message for tdgemm_last_error() on this thread
void record_error(const char *msg);

cudaError_t launch_snr(const void *C, long long ldc, int dtype, const double *ref, long long ldr,
                       long long M, long long N, double *out3, cudaStream_t st);

// Tensor-core forms (tcgen05): C = sum_l (s_A s_B) * (A~_l B~_l^T) with both
// code operands k-major: A~ [M][K], B~ [N][K] (fp16 integers or e4m3).
struct TcArgs {
    const DevPlan *plan;
    long long M, N, K;
    int L, nM, nK, nN;
    const float *pair;
    float *C;
    long long ldc;
    float alpha, beta;
    int beta_zero;
    int c_tma;            // 1: C written by TMA stores through mapC (beta = 0, C 16-byte aligned)
};
cudaError_t launch_tc_gemm(int fp8, const TcArgs &a, const CUtensorMap &mapA,
                           const CUtensorMap &mapB, const CUtensorMap &mapC, cudaStream_t st);
void tc_gemm_c_box(int *box_cols, int *box_rows);
void tc_gemm_boxes(int fp8, int *box_rows_a, int *box_rows_b, int *box_k);

}  // namespace tdg
