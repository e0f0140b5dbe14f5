/*
 * CPU oracle for the companded-and-packed GEMM (Anastasia & Andreopoulos,
 * "Throughput-Distortion Computation of Generic Matrix Multiplication").
 *
 * TEST INFRASTRUCTURE ONLY.  Nothing in the product path may link, load or
 * call this file; it exists so that tests, the smoke check and the benchmark's
 * CPU baseline can check the CUDA path against a plain restatement of the
 * paper.  It shares no code, header or constant with the CUDA library.
 *
 * Plain loops, one output at a time, in the order the equations are written.
 * Built with -O2 -ffp-contract=off so that every a*b+c below is a separately
 * rounded multiply and add, and every fma()/fmaf() is a single rounding.
 * The default IEEE rounding mode (round to nearest, ties to even) is assumed;
 * rint()/rintf() then implement the paper's [[x]] (round to integer).
 *
 * Matrices are dense row-major with the transpose already applied: op(A) is
 * M x K, op(B) is K x N.  Blocks are L x L; a border block holds only the
 * valid elements, the rest is zero padding (Sec. 2, "cleanup" at borders).
 * Per-block companders c and their inverses s = 1/c arrive as fp64 arrays
 * computed by the Python side of the oracle.
 */
#include <math.h>
#include <stdint.h>
#include <stddef.h>

#define CDIV(a, b) (((a) + (b) - 1) / (b))

/* ------------------------------------------------------------------ */
/* Eq. 3: a~ = [[c_A a]] inside each L x L block (the product rounded in the
 * working type T, then rounded to the nearest integer).                 */
/* ------------------------------------------------------------------ */
void orc_compand_f32(const float *X, int64_t rows, int64_t cols, int L,
                     const double *c, float *Xq)
{
    int64_t nbc = CDIV(cols, L);
    for (int64_t r = 0; r < rows; ++r)
        for (int64_t k = 0; k < cols; ++k) {
            float cT = (float)c[(r / L) * nbc + k / L];
            float prod = X[r * cols + k] * cT;
            Xq[r * cols + k] = rintf(prod);
        }
}

void orc_compand_f64(const double *X, int64_t rows, int64_t cols, int L,
                     const double *c, double *Xq)
{
    int64_t nbc = CDIV(cols, L);
    for (int64_t r = 0; r < rows; ++r)
        for (int64_t k = 0; k < cols; ++k) {
            double prod = X[r * cols + k] * c[(r / L) * nbc + k / L];
            Xq[r * cols + k] = rint(prod);
        }
}

/* ------------------------------------------------------------------ */
/* Eqs. 6, 7, 11: packing W quantized values into one number,
 *   x_bar = sum_i w^i d_i,  evaluated by Horner's rule from the last digit:
 *   acc = d_{W-1};  acc = fma(w, acc, d_i) for i = W-2 .. 0.
 * w = z for eq. 6 and eq. 11, w = z^-1 for eq. 7.
 *
 * pack_cols: digits run along the column index inside each L-wide column
 * block; column block l, packed column j takes columns l*L + W*j + i.
 * Output has nb*P columns, P = ceil(L / W).  Digits that fall outside the
 * block or the matrix are zero.                                          */
/* ------------------------------------------------------------------ */
void orc_pack_cols_f32(const float *Xq, int64_t rows, int64_t cols, int L, int W,
                       float w, float *Xbar)
{
    int64_t nb = CDIV(cols, L);
    int P = (L + W - 1) / W;
    for (int64_t r = 0; r < rows; ++r)
        for (int64_t l = 0; l < nb; ++l)
            for (int j = 0; j < P; ++j) {
                float d[8] = {0};
                for (int i = 0; i < W; ++i) {
                    int64_t inblk = (int64_t)W * j + i;
                    int64_t k = l * L + inblk;
                    d[i] = (inblk < L && k < cols) ? Xq[r * cols + k] : 0.0f;
                }
                float acc = d[W - 1];
                for (int i = W - 2; i >= 0; --i) acc = fmaf(w, acc, d[i]);
                Xbar[r * (nb * P) + l * P + j] = acc;
            }
}

void orc_pack_cols_f64(const double *Xq, int64_t rows, int64_t cols, int L, int W,
                       double w, double *Xbar)
{
    int64_t nb = CDIV(cols, L);
    int P = (L + W - 1) / W;
    for (int64_t r = 0; r < rows; ++r)
        for (int64_t l = 0; l < nb; ++l)
            for (int j = 0; j < P; ++j) {
                double d[8] = {0};
                for (int i = 0; i < W; ++i) {
                    int64_t inblk = (int64_t)W * j + i;
                    int64_t k = l * L + inblk;
                    d[i] = (inblk < L && k < cols) ? Xq[r * cols + k] : 0.0;
                }
                double acc = d[W - 1];
                for (int i = W - 2; i >= 0; --i) acc = fma(w, acc, d[i]);
                Xbar[r * (nb * P) + l * P + j] = acc;
            }
}

/* pack_rows: digits run along the row index inside each L-tall row block;
 * output has nb*P rows.                                                  */
void orc_pack_rows_f32(const float *Xq, int64_t rows, int64_t cols, int L, int W,
                       float w, float *Xbar)
{
    int64_t nb = CDIV(rows, L);
    int P = (L + W - 1) / W;
    for (int64_t l = 0; l < nb; ++l)
        for (int j = 0; j < P; ++j)
            for (int64_t c = 0; c < cols; ++c) {
                float d[8] = {0};
                for (int i = 0; i < W; ++i) {
                    int64_t inblk = (int64_t)W * j + i;
                    int64_t r = l * L + inblk;
                    d[i] = (inblk < L && r < rows) ? Xq[r * cols + c] : 0.0f;
                }
                float acc = d[W - 1];
                for (int i = W - 2; i >= 0; --i) acc = fmaf(w, acc, d[i]);
                Xbar[(l * P + j) * cols + c] = acc;
            }
}

void orc_pack_rows_f64(const double *Xq, int64_t rows, int64_t cols, int L, int W,
                       double w, double *Xbar)
{
    int64_t nb = CDIV(rows, L);
    int P = (L + W - 1) / W;
    for (int64_t l = 0; l < nb; ++l)
        for (int j = 0; j < P; ++j)
            for (int64_t c = 0; c < cols; ++c) {
                double d[8] = {0};
                for (int i = 0; i < W; ++i) {
                    int64_t inblk = (int64_t)W * j + i;
                    int64_t r = l * L + inblk;
                    d[i] = (inblk < L && r < rows) ? Xq[r * cols + c] : 0.0;
                }
                double acc = d[W - 1];
                for (int i = W - 2; i >= 0; --i) acc = fma(w, acc, d[i]);
                Xbar[(l * P + j) * cols + c] = acc;
            }
}

/* ------------------------------------------------------------------ */
/* Symmetric form, one output (m, n):
 *   for each slab l:  r_bar = sum_j a_bar[m, lP+j] b_bar[lP+j, n]   (eq. 8,
 *                     an fma chain in ascending j starting at +0),
 *                     u = [[r_bar]]                                 (eq. 9)
 *                     r~ = u - z^-1 [[z u]]                         (eq. 10)
 *                     C += r~ * (s_A,il s_B,lj)                      (eqs. 5, 2)
 * The de-companding factor is the fp64 product s_A s_B rounded to T; the
 * sum over l is an fma chain in ascending l starting at +0.
 * Computes the output rows [r0, r1) and columns [c0, c1); when rint_out is
 * not NULL it receives r~ for every (m, n, l) of that window.            */
/* ------------------------------------------------------------------ */
void orc_sym_gemm_f32(const float *Abar, const float *Bbar, int64_t M, int64_t N,
                      int64_t nK, int P, int L, int q, const double *sA,
                      const double *sB, int64_t r0, int64_t r1, int64_t c0,
                      int64_t c1, int64_t *rint_out, float *Cacc)
{
    int64_t nN = CDIV(N, L);
    int64_t Kp = nK * P;
    float z = ldexpf(1.0f, -q), Q = ldexpf(1.0f, q);
    (void)M;
    for (int64_t m = r0; m < r1; ++m)
        for (int64_t n = c0; n < c1; ++n) {
            float acc = 0.0f;
            for (int64_t l = 0; l < nK; ++l) {
                float rbar = 0.0f;
                for (int j = 0; j < P; ++j)
                    rbar = fmaf(Abar[m * Kp + l * P + j], Bbar[(l * P + j) * N + n], rbar);
                float u = rintf(rbar);
                float t = rintf(z * u);
                float rt = u - Q * t;
                float pair = (float)(sA[(m / L) * nK + l] * sB[l * nN + n / L]);
                acc = fmaf(rt, pair, acc);
                if (rint_out)
                    rint_out[((m - r0) * (c1 - c0) + (n - c0)) * nK + l] = (int64_t)rt;
            }
            Cacc[(m - r0) * (c1 - c0) + (n - c0)] = acc;
        }
}

void orc_sym_gemm_f64(const double *Abar, const double *Bbar, int64_t M, int64_t N,
                      int64_t nK, int P, int L, int q, const double *sA,
                      const double *sB, int64_t r0, int64_t r1, int64_t c0,
                      int64_t c1, int64_t *rint_out, double *Cacc)
{
    int64_t nN = CDIV(N, L);
    int64_t Kp = nK * P;
    double z = ldexp(1.0, -q), Q = ldexp(1.0, q);
    (void)M;
    for (int64_t m = r0; m < r1; ++m)
        for (int64_t n = c0; n < c1; ++n) {
            double acc = 0.0;
            for (int64_t l = 0; l < nK; ++l) {
                double rbar = 0.0;
                for (int j = 0; j < P; ++j)
                    rbar = fma(Abar[m * Kp + l * P + j], Bbar[(l * P + j) * N + n], rbar);
                double u = rint(rbar);
                double t = rint(z * u);
                double rt = u - Q * t;
                double pair = sA[(m / L) * nK + l] * sB[l * nN + n / L];
                acc = fma(rt, pair, acc);
                if (rint_out)
                    rint_out[((m - r0) * (c1 - c0) + (n - c0)) * nK + l] = (int64_t)rt;
            }
            Cacc[(m - r0) * (c1 - c0) + (n - c0)] = acc;
        }
}

/* ------------------------------------------------------------------ */
/* Asymmetric form, one output (m, n).  Output row m lies in row block
 * i = m / L at in-block row W*j + d; its packed row is i*P + j (eq. 11).
 *   for each slab l:  r_bar = sum_k a_bar[iP+j, k] b~[k, n] over the slab's
 *                     valid k, ascending, fma chain from +0         (eq. 12)
 *                     x = r_bar; repeat for e = 0 .. d:
 *                        r~_e = [[x]];  x = z^-1 (x - r~_e)         (eqs. 13-14)
 *                     r~ = r~_d;  C += r~ (s_A s_B)                  (eqs. 5, 2)
 * The packed product is recomputed for every digit d: slow, but each output
 * is computed on its own.                                                */
/* ------------------------------------------------------------------ */
void orc_asym_gemm_f32(const float *Abar, const float *Bq, int64_t M, int64_t N,
                       int64_t K, int P, int L, int W, int q, const double *sA,
                       const double *sB, int64_t r0, int64_t r1, int64_t c0,
                       int64_t c1, int64_t *rint_out, float *Cacc)
{
    int64_t nK = CDIV(K, L), nN = CDIV(N, L);
    float Q = ldexpf(1.0f, q);
    (void)M; (void)W;
    for (int64_t m = r0; m < r1; ++m) {
        int64_t i = m / L, inblk = m % L;
        int64_t pr = i * P + inblk / W;
        int d = (int)(inblk % W);
        for (int64_t n = c0; n < c1; ++n) {
            float acc = 0.0f;
            for (int64_t l = 0; l < nK; ++l) {
                float rbar = 0.0f;
                int64_t kend = (l + 1) * L < K ? (l + 1) * L : K;
                for (int64_t k = l * L; k < kend; ++k)
                    rbar = fmaf(Abar[pr * K + k], Bq[k * N + n], rbar);
                float x = rbar, rt = 0.0f;
                for (int e = 0; e <= d; ++e) {
                    rt = rintf(x);
                    if (e < d) x = Q * (x - rt);
                }
                float pair = (float)(sA[i * nK + l] * sB[l * nN + n / L]);
                acc = fmaf(rt, pair, acc);
                if (rint_out)
                    rint_out[((m - r0) * (c1 - c0) + (n - c0)) * nK + l] = (int64_t)rt;
            }
            Cacc[(m - r0) * (c1 - c0) + (n - c0)] = acc;
        }
    }
}

void orc_asym_gemm_f64(const double *Abar, const double *Bq, int64_t M, int64_t N,
                       int64_t K, int P, int L, int W, int q, const double *sA,
                       const double *sB, int64_t r0, int64_t r1, int64_t c0,
                       int64_t c1, int64_t *rint_out, double *Cacc)
{
    int64_t nK = CDIV(K, L), nN = CDIV(N, L);
    double Q = ldexp(1.0, q);
    (void)M; (void)W;
    for (int64_t m = r0; m < r1; ++m) {
        int64_t i = m / L, inblk = m % L;
        int64_t pr = i * P + inblk / W;
        int d = (int)(inblk % W);
        for (int64_t n = c0; n < c1; ++n) {
            double acc = 0.0;
            for (int64_t l = 0; l < nK; ++l) {
                double rbar = 0.0;
                int64_t kend = (l + 1) * L < K ? (l + 1) * L : K;
                for (int64_t k = l * L; k < kend; ++k)
                    rbar = fma(Abar[pr * K + k], Bq[k * N + n], rbar);
                double x = rbar, rt = 0.0;
                for (int e = 0; e <= d; ++e) {
                    rt = rint(x);
                    if (e < d) x = Q * (x - rt);
                }
                double pair = sA[i * nK + l] * sB[l * nN + n / L];
                acc = fma(rt, pair, acc);
                if (rint_out)
                    rint_out[((m - r0) * (c1 - c0) + (n - c0)) * nK + l] = (int64_t)rt;
            }
            Cacc[(m - r0) * (c1 - c0) + (n - c0)] = acc;
        }
    }
}

/* ------------------------------------------------------------------ */
/* Conventional GEMM in T (the W = 1, no-companding case of Sec. 7):
 * C[m,n] = sum_k a[m,k] b[k,n], an fma chain in ascending k from +0.
 * In fp64 this is also the exact reference the SNR of eq. 20 is taken
 * against (inputs promoted to fp64 by the caller).                     */
/* ------------------------------------------------------------------ */
void orc_gemm_f32(const float *A, const float *B, int64_t M, int64_t N, int64_t K,
                  int64_t r0, int64_t r1, int64_t c0, int64_t c1, float *C)
{
    (void)M;
    for (int64_t m = r0; m < r1; ++m)
        for (int64_t n = c0; n < c1; ++n) {
            float acc = 0.0f;
            for (int64_t k = 0; k < K; ++k) acc = fmaf(A[m * K + k], B[k * N + n], acc);
            C[(m - r0) * (c1 - c0) + (n - c0)] = acc;
        }
}

void orc_gemm_f64(const double *A, const double *B, int64_t M, int64_t N, int64_t K,
                  int64_t r0, int64_t r1, int64_t c0, int64_t c1, double *C)
{
    (void)M;
    for (int64_t m = r0; m < r1; ++m)
        for (int64_t n = c0; n < c1; ++n) {
            double acc = 0.0;
            for (int64_t k = 0; k < K; ++k) acc = fma(A[m * K + k], B[k * N + n], acc);
            C[(m - r0) * (c1 - c0) + (n - c0)] = acc;
        }
}

/* ------------------------------------------------------------------ */
/* Eq. 4 taken literally on integers: per slab, r~ = sum_k a~ b~ in exact
 * 64-bit integer arithmetic, then C += r~ (s_A s_B) in fp32 (eqs. 5, 2).
 * Inputs are integer-valued floats.  This is the quantized-GEMM form that
 * runs on tensor cores with integer-valued 16-bit operands.              */
/* ------------------------------------------------------------------ */
void orc_int_gemm_f32(const float *Aq, const float *Bq, int64_t M, int64_t N,
                      int64_t K, int L, const double *sA, const double *sB,
                      int64_t r0, int64_t r1, int64_t c0, int64_t c1,
                      int64_t *rint_out, float *Cacc)
{
    int64_t nK = CDIV(K, L), nN = CDIV(N, L);
    (void)M;
    for (int64_t m = r0; m < r1; ++m)
        for (int64_t n = c0; n < c1; ++n) {
            float acc = 0.0f;
            for (int64_t l = 0; l < nK; ++l) {
                int64_t r = 0;
                int64_t kend = (l + 1) * L < K ? (l + 1) * L : K;
                for (int64_t k = l * L; k < kend; ++k)
                    r += (int64_t)Aq[m * K + k] * (int64_t)Bq[k * N + n];
                float pair = (float)(sA[(m / L) * nK + l] * sB[l * nN + n / L]);
                acc = fmaf((float)r, pair, acc);
                if (rint_out)
                    rint_out[((m - r0) * (c1 - c0) + (n - c0)) * nK + l] = r;
            }
            Cacc[(m - r0) * (c1 - c0) + (n - c0)] = acc;
        }
}

/* Per-slab sums of 8-bit floating-point codes: every product of two e4m3
 * values is exact in fp64 and a slab of up to 2^12 of them sums exactly in
 * fp64, so r = sum_k a~ b~ is exact; it is then rounded once to fp32 and
 * de-companded as above.                                                  */
void orc_fp8_gemm_f32(const double *Aq, const double *Bq, int64_t M, int64_t N,
                      int64_t K, int L, const double *sA, const double *sB,
                      int64_t r0, int64_t r1, int64_t c0, int64_t c1, float *Cacc)
{
    int64_t nK = CDIV(K, L), nN = CDIV(N, L);
    (void)M;
    for (int64_t m = r0; m < r1; ++m)
        for (int64_t n = c0; n < c1; ++n) {
            float acc = 0.0f;
            for (int64_t l = 0; l < nK; ++l) {
                double r = 0.0;
                int64_t kend = (l + 1) * L < K ? (l + 1) * L : K;
                for (int64_t k = l * L; k < kend; ++k) r += Aq[m * K + k] * Bq[k * N + n];
                float pair = (float)(sA[(m / L) * nK + l] * sB[l * nN + n / L]);
                acc = fmaf((float)r, pair, acc);
            }
            Cacc[(m - r0) * (c1 - c0) + (n - c0)] = acc;
        }
}

/* ------------------------------------------------------------------ */
/* OCP 8-bit E4M3 ("fn" variant) encoder written from the format: 1 sign,
 * 4 exponent bits (bias 7), 3 fraction bits, no infinities, largest finite
 * 448, smallest subnormal 2^-9.  Round to nearest, ties to even; values
 * beyond 448 saturate to +-448.  Returns the decoded value as a double.  */
/* ------------------------------------------------------------------ */
double orc_e4m3_rn_sat(double x)
{
    if (isnan(x)) return x;
    double ax = fabs(x);
    double sgn = x < 0 ? -1.0 : 1.0;
    if (ax == 0.0) return sgn * 0.0;
    int e;
    frexp(ax, &e);              /* ax = f * 2^e, f in [0.5, 1) */
    int E = e - 1;              /* ax in [2^E, 2^(E+1)) */
    if (E < -6) E = -6;         /* subnormal range shares the 2^-6 spacing base */
    double spacing = ldexp(1.0, E - 3);
    double k = ax / spacing;    /* exact: spacing is a power of two */
    double kr = rint(k);        /* ties to even */
    double v = kr * spacing;
    if (v > 448.0) v = 448.0;
    return sgn * v;
}

void orc_e4m3_array(const double *x, int64_t n, double *out)
{
    for (int64_t i = 0; i < n; ++i) out[i] = orc_e4m3_rn_sat(x[i]);
}

/* alpha/beta epilogue: C = alpha*Cacc            (beta == 0, C not read)
 *                      C = fma(alpha, Cacc, beta*Cin)  otherwise          */
void orc_epilogue_f32(const float *Cacc, const float *Cin, int64_t n, double alpha,
                      double beta, float *out)
{
    float a = (float)alpha, b = (float)beta;
    for (int64_t i = 0; i < n; ++i)
        out[i] = (beta == 0.0) ? a * Cacc[i] : fmaf(a, Cacc[i], b * Cin[i]);
}

void orc_epilogue_f64(const double *Cacc, const double *Cin, int64_t n, double alpha,
                      double beta, double *out)
{
    for (int64_t i = 0; i < n; ++i)
        out[i] = (beta == 0.0) ? alpha * Cacc[i] : fma(alpha, Cacc[i], beta * Cin[i]);
}
