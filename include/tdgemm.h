/*
 * tdgemm — throughput-distortion GEMM on one GB300 (sm_103a).
 *
 * C ABI of the companded-and-packed matrix product of Anastasia &
 * Andreopoulos, "Throughput-Distortion Computation of Generic Matrix
 * Multiplication" (the paper):
 *
 *     C = alpha * op(A) * op(B) + beta * C,   op(A): M x K,  op(B): K x N
 *
 * computed through four steps on the device:
 *   (a) per L x L block statistics and companders, then companding and
 *       rounding of every input element                      (Sec. 3.A, eq. 3,
 *                                                              Sec. 5, eqs. 15-27)
 *   (b) packing W quantized values into one floating-point number
 *       (symmetric form, eqs. 6-7; asymmetric form, eq. 11)
 *   (c) the packed multiply-accumulate, W results per FMA  (eqs. 8, 12)
 *   (d) unpacking, de-companding and rescaling              (eqs. 9-10, 13-14, 5, 2)
 * plus a tensor-core form of (c) on the companded integers (the integer
 * processing of Remark 1, on 16-bit float carriers) and on 8-bit E4M3 codes.
 *
 * Conventions (all entry points):
 *   - Matrices are row-major.  op(X) = X for trans 'N'/'n', X^T for 'T'/'t'.
 *     lda, ldb, ldc are leading dimensions in elements of the stored matrix.
 *   - A, B, C are device pointers owned by the caller; they must stay valid
 *     until the work queued on `stream` has finished.  `stream` is a
 *     cudaStream_t (NULL = the legacy default stream).
 *   - The plan owns every other device buffer (statistics, companders, packed
 *     operands) and frees it in tdgemm_plan_destroy.
 *   - All device work is queued on `stream` (tdgemm_run_host_async also
 *     uses a copy stream of the plan's); no entry point synchronises the
 *     host except tdgemm_plan_info, tdgemm_unpack (when given host buffers)
 *     and tdgemm_run_host.
 *   - Argument errors are returned at once and leave the plan unchanged.
 *     Conditions found on the device (non-finite input, unreachable target)
 *     are written to a device status word that tdgemm_plan_info reads.
 *   - A plan is not thread-safe; distinct plans are independent.
 *   - Every failing call records a message readable with tdgemm_last_error()
 *     (thread-local).
 */
#ifndef TDGEMM_H
#define TDGEMM_H

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef struct tdgemm_plan_s *tdgemm_plan_t;

/* Working type T of the packed arithmetic (Sec. 7: sGEMM / dGEMM). */
typedef enum { TDG_F32 = 0, TDG_F64 = 1 } tdg_dtype;

/* Form of step (c):
 *   TDG_PLAIN   conventional product in T, no companding (W = 1, Sec. 7 "plain")
 *   TDG_SYM     symmetric packing, eqs. 6-10
 *   TDG_ASYM    asymmetric packing, eqs. 11-14
 *   TDG_TC_INT  companded integers (eq. 3) multiplied on tensor cores as
 *               integer-valued fp16 operands; every per-slab sum is an integer
 *               below 2^24, so the fp32 accumulation equals eq. 4 exactly
 *               (Remark 1's integer processing).  fp32 inputs only.
 *   TDG_TC_FP8  per-block companded E4M3 codes (c = 448 / max|x|) on tensor
 *               cores with fp32 accumulation.  fp32 inputs only.            */
typedef enum {
    TDG_PLAIN = 0,
    TDG_SYM = 1,
    TDG_ASYM = 2,
    TDG_TC_INT = 3,
    TDG_TC_FP8 = 4
} tdg_form;

typedef enum {
    TDG_OK = 0,
    TDG_EINVAL = 1,          /* bad argument                                   */
    TDG_ENOMEM = 2,          /* device allocation failed                       */
    TDG_ECUDA = 3,           /* a CUDA call failed (message in last_error)     */
    TDG_EUNSUPPORTED = 4,    /* valid but not built (e.g. TC form with f64)    */
    TDG_EUNREACHABLE = 5,    /* target SNR not met at any W > 1, no fallback   */
    TDG_ETIMEOUT = 6,        /* a device wait exceeded its iteration budget    */
    TDG_ENONFINITE = 7,      /* NaN or Inf found in an input block             */
    TDG_ESTATE = 8           /* call out of order (e.g. gemm before pack)      */
} tdg_status;

/* flags for tdgemm_plan */
#define TDG_ALLOW_FALLBACK 0x1u  /* target unmet at every W > 1: compute the plain
                                    product (W = 1, Sec. 6) instead of failing  */
#define TDG_KEEP_PACKED    0x2u  /* tdgemm_gemm also stores every packed slab
                                    result r_bar for tdgemm_unpack              */
#define TDG_PAIR_EXACT     0x8u  /* companders of eq. 26 per subblock product (i, l, j)
                                    within the call's R_max instead of one split
                                    Gamma_A, Gamma_B per call; SYM form, transA =
                                    transB = 'N', L = 128 (fp32) or 64 (fp64), W
                                    in {2, 4} (target mode: W = 2); each CTA then
                                    compands and packs its own operand tiles      */
#define TDG_NOISE_RMS      0x4u  /* planner: the representation noise s(R_max, W),
                                    measured with uniform integer inputs (Sec. 4.B),
                                    scaled by 3 kappa_A kappa_B, the blocks' crest
                                    factors kappa = sigma / max (the rounding error
                                    of the packed sums follows their RMS).  The
                                    default; the flag is accepted and changes
                                    nothing.  Uniform sources: no change.        */
#define TDG_NOISE_UNIFORM  0x10u /* planner: s(R_max, W) as measured, unscaled
                                    (the paper's model of eq. 21 with the Sec. 4.B
                                    calibration as it stands); pessimistic by
                                    several dB for peaky (Gaussian, Laplacian)
                                    sources.  Not with TDG_NOISE_RMS.            */

/* What the planner chose, read back by tdgemm_plan_info (synchronises). */
typedef struct {
    int32_t W_used;          /* packing used; 1 = plain product                 */
    int32_t q;               /* z = 2^-q (eq. 15)                               */
    int32_t gamma_a;         /* |a~| <= gamma_a, c_A = gamma_a / max|A_il|      */
    int32_t gamma_b;
    int64_t r_max;           /* L * gamma_a * gamma_b (eq. 17)                  */
    int32_t w_ef;            /* error-free packing limit for r_max (eq. 16)     */
    int32_t level;           /* R_max candidate index in target mode, else -1   */
    double pred_snr_db;      /* model SNR, eqs. 19-21 (NaN if not modelled)     */
    int64_t workspace_bytes; /* device memory the plan owns                     */
    int32_t device_status;   /* tdg_status found on the device by the last pack */
    int32_t carrier;         /* TC forms: 16 = fp16 integer carrier, 8 = e4m3   */
} tdgemm_info;

/*
 * Create a plan: shapes, block size and packing as the paper poses the
 * problem (Sec. 2: M x K by K x N split into L x L subblocks; eq. 1 block
 * size; W packings; Sec. 6 distortion target).
 *
 *   transA, transB  'N' or 'T'
 *   M, N, K         >= 1
 *   lda, ldb, ldc   leading dimensions (elements) of the stored A, B, C
 *   L               block size, a multiple of 16 in [16, 1024]; the TC forms
 *                   need a multiple of 64
 *   W               packing factor 1..4 (SYM, ASYM); PLAIN and TC forms: 1
 *   dtype, form     see above
 *   target_snr_db   distortion target in dB (used when bits == 0)
 *   bits            > 0: fixed-bit companding, gamma = 2^(bits-1) - 1, W as
 *                   given (SYM, ASYM: bits in 2..20; TC_INT: 2..12 with
 *                   L * gamma^2 below 2^24)
 *   flags           TDG_ALLOW_FALLBACK | TDG_KEEP_PACKED | TDG_NOISE_RMS |
 *                   TDG_NOISE_UNIFORM | TDG_PAIR_EXACT
 *
 * On success *plan receives a new plan holding all device workspace for these
 * shapes (allocated on the current device).  On error *plan is left NULL.
 */
tdg_status tdgemm_plan(tdgemm_plan_t *plan, char transA, char transB, int64_t M, int64_t N,
                       int64_t K, int64_t lda, int64_t ldb, int64_t ldc, int L, int W,
                       tdg_dtype dtype, tdg_form form, double target_snr_db, int bits,
                       uint32_t flags);

/*
 * Give the planner the measured representation-noise RMSE s(R_max, W) of
 * Sec. 4.B / eq. 18 for packing W of this plan's dtype, form and L:
 * s[i] belongs to the R_max level t0 + i, where level t means
 * R_t = ((4 + t mod 4) << (t div 4)) / 4 in integer arithmetic (four levels
 * per octave); a negative entry marks a level that was not measured.  Host array, copied.  Without a table the planner uses
 * only levels inside the error-free region of Prop. 1 (s = 0).
 */
tdg_status tdgemm_set_rep_noise(tdgemm_plan_t plan, int W, const double *s, int t0, int n);

/*
 * Manual parameters, bypassing the planner (the measurement protocol of
 * Sec. 4.B uses c_A = c_B = 1): every block gets compander c_A (c_B) and the
 * packing coefficient is z = 2^-q.  q in 1..60, c > 0.
 */
tdg_status tdgemm_set_manual(tdgemm_plan_t plan, int q, double c_a, double c_b);

/*
 * Throughput-distortion control over inner kernels (Sec. 6).  Inner kernel
 * (i, j) is the L x L output block C_ij = sum_l A_il B_lj.  With control on,
 * each call of tdgemm_quantize_pack predicts, from the block statistics and
 * the companders the planner chose, the ratio S_ij / N_ij of that inner
 * kernel (the noise model of eq. 19 restricted to its K / L block products,
 * representation noise s of the chosen packing as in the plan's options) and
 * accelerates (packs) only some of them; tdgemm_gemm computes the rest with
 * the conventional product (W = 1), so the output is exact there.
 *
 *   mode 0   control off (every inner kernel follows the plan; default)
 *   mode 1   SNR threshold: accelerate the inner kernels whose predicted
 *            10 log10(S_ij / N_ij) >= value (dB)
 *   mode 2   fraction: accelerate the ceil(value * nM * nN) inner kernels
 *            of highest predicted S_ij / N_ij (ties to the lower row-major
 *            index); value in [0, 1]
 *   mode 3   throughput (Sec. 6 (ii)): value = F >= 1, the required
 *            acceleration of the product over the conventional one.  With
 *            T = nM * nN inner kernels, each accelerated one taking 1 / F_W
 *            of a conventional one's time (F_W of the packing the planner
 *            chose, from tdgemm_set_speedup), accelerate the
 *            k = ceil(T (1 - 1/F) / (1 - 1/F_W)) kernels of highest
 *            predicted S_ij / N_ij (as mode 2): the fewest whose predicted
 *            throughput T / ((T - k) + k / F_W) reaches F; none if F_W <= 1,
 *            all if F >= F_W.  Needs F_W for every W the planner may choose.
 *
 * Valid for the SYM form with a planned (fixed-bit or target) plan without
 * TDG_KEEP_PACKED, at most 16384 inner kernels, and L a multiple of the GEMM
 * CTA tile (128 for fp32, 64 for fp64); TDG_EINVAL otherwise.  A plan whose
 * planner fell back to W = 1 accelerates nothing.  Both kinds of inner kernel
 * run in one GEMM launch (each CTA tile lies inside one inner kernel).
 * Changing the setting requires tdgemm_quantize_pack again (TDG_ESTATE from
 * tdgemm_gemm otherwise).  Allocates the mask, ratio and plain-operand buffers
 * on the first call that turns control on; they are freed with the plan.
 */
tdg_status tdgemm_set_kernel_control(tdgemm_plan_t plan, int mode, double value);

/*
 * The measured throughput scaling F_W of Sec. 5.B: how many times faster an
 * accelerated (packed, W) inner kernel runs than a conventional one on this
 * GPU, measured offline for the plan's dtype, form and L (the package ships
 * such a table, measured on GB300).  Used by throughput control (mode 3).
 * W in 2..4, speedup > 0 and finite.
 */
tdg_status tdgemm_set_speedup(tdgemm_plan_t plan, int W, double speedup);

/*
 * Copy the inner-kernel mask of the last tdgemm_quantize_pack to host memory:
 * out[i * nN + j] = 1 where inner kernel (i, j) is accelerated, else 0;
 * n >= nM * nN bytes.  Synchronises the plan's last stream.  TDG_ESTATE when
 * control is off or nothing was packed.
 */
tdg_status tdgemm_kernel_mask(tdgemm_plan_t plan, uint8_t *out, int64_t n);

/*
 * Steps (a) and (b): block statistics, planner, companders, companding and
 * packing of A and B into the plan's workspace.  A and B are device pointers
 * in the plan's dtype (fp32 for the TC forms).
 */
tdg_status tdgemm_quantize_pack(tdgemm_plan_t plan, const void *A, const void *B,
                                void *stream);

/*
 * Steps (a) and (b) for A alone, reusing B: its statistics, companders and
 * packed (or copied, or coded) form from the last tdgemm_quantize_pack, whose
 * B the caller keeps unchanged in place (for a product repeated with a fixed
 * right operand, e.g. inference with fixed weights).  Valid when B's
 * companders do not depend on A: fixed-bit and manual plans, the PLAIN and the
 * TC_FP8 forms; TDG_EINVAL for distortion-target plans (their Gamma_A, Gamma_B
 * come from both operands), TDG_ESTATE before any tdgemm_quantize_pack or after
 * tdgemm_set_manual / tdgemm_set_kernel_control.  Non-finite values in B were
 * reported by the pack that processed B, not again here.
 */
tdg_status tdgemm_quantize_pack_a(tdgemm_plan_t plan, const void *A, void *stream);

/*
 * Steps (c) and (d): packed multiply-accumulate with unpacking,
 * de-companding and the sum over slabs fused into the accumulator
 * registers, then C = alpha * C_acc + beta * C (C not read when beta == 0).
 * Requires a preceding tdgemm_quantize_pack on the same plan.
 */
tdg_status tdgemm_gemm(tdgemm_plan_t plan, void *C, double alpha, double beta, void *stream);

/* tdgemm_quantize_pack followed by tdgemm_gemm. */
tdg_status tdgemm_run(tdgemm_plan_t plan, const void *A, const void *B, void *C, double alpha,
                      double beta, void *stream);

/*
 * The same with HOST buffers: A, B and C are host pointers (pinned memory
 * gives asynchronous copies); the plan copies A and B to device staging
 * buffers it owns, runs, copies C back and synchronises `stream`.  When C is
 * pinned memory the device can address, beta == 0 and the form is PLAIN, SYM
 * or ASYM (without slab splitting or TDG_PAIR_EXACT), the GEMM writes C in
 * place over the CPU-GPU link instead of a staged copy back.
 */
tdg_status tdgemm_run_host(tdgemm_plan_t plan, const void *A, const void *B, void *C,
                           double alpha, double beta, void *stream);

/*
 * The same, pipelined for a sequence of products with HOST buffers: queues
 * the copies of A and B (and of C when beta != 0) on a copy stream the plan
 * owns, into the first of two device staging sets that the computation
 * queued earlier no longer reads, then the computation on `stream` after
 * them, and the copy of C back (unless C is written in place, as above); it
 * returns without synchronising.  The copies of one call therefore run while
 * the computation of the previous call does.  A, B and C must be pinned host
 * memory (page-locked, cudaHostAlloc / cudaHostRegister: TDG_EINVAL
 * otherwise) and must stay unchanged (A, B) and unread (C) until `stream`
 * has finished the call's work; successive calls on one plan must use the
 * same `stream`.  Results are bit-identical to tdgemm_run_host's.
 */
tdg_status tdgemm_run_host_async(tdgemm_plan_t plan, const void *A, const void *B, void *C,
                                 double alpha, double beta, void *stream);

/*
 * Unfused step (d) for checking the integer domain: needs TDG_KEEP_PACKED and
 * a preceding tdgemm_gemm.  rint_out (device, nullable) receives the unpacked
 * integers r~ of every output and slab as int64, layout [m][n][l]
 * (M x N x ceil(K/L)); C (device, nullable, ldc) receives the de-companded
 * sum over slabs (alpha = 1, beta = 0).  SYM and ASYM forms only.
 */
tdg_status tdgemm_unpack(tdgemm_plan_t plan, int64_t *rint_out, void *C, void *stream);

/* Read what the planner chose (synchronises the plan's last stream). */
tdg_status tdgemm_plan_info(tdgemm_plan_t plan, tdgemm_info *out);

/* Free the plan and its workspace (synchronises the device first). */
tdg_status tdgemm_plan_destroy(tdgemm_plan_t plan);

/*
 * Output distortion against a reference (eq. 20 measured): accumulates
 * sum(ref^2), sum((C - ref)^2), sum(C - ref) in fp64 over the M x N outputs
 * into out3[0..2] (device pointer, overwritten).  C is in `dtype` with
 * leading dimension ldc; ref is fp64 with leading dimension ldr.
 */
tdg_status tdgemm_snr(const void *C, int64_t ldc, tdg_dtype dtype, const double *ref,
                      int64_t ldr, int64_t M, int64_t N, double *out3, void *stream);

/*
 * One-shot fixed-bit product that allocates nothing:
 *     C = alpha * op(A) * op(B) + beta * C
 * with the statistics, companders, de-companding factors and packed operands
 * in one static device array of 32 MiB that the library holds on every GPU
 * that loads it, instead of plan workspace from cudaMalloc.  For callers that
 * may not allocate device memory where they call: frameworks whose allocator
 * owns the whole device and forbids libraries' side allocations, plug-ins
 * handed only the buffers they compute on, and latency-bound services that
 * must not allocate (or synchronise the device) on first use.
 *   form     TDG_SYM or TDG_ASYM; W 1..4; bits 2..20 (gamma = 2^(bits-1) - 1);
 *            other arguments as in tdgemm_plan / tdgemm_gemm.  A, B, C device.
 * Results equal those of tdgemm_plan + tdgemm_run with the same arguments.
 * Device-side conditions are not reported: a NaN or Inf in A or B leaves
 * non-finite values in C and the call still returns TDG_OK (the plan-based
 * path reports it through tdgemm_plan_info).  M, N, K <= 2^31.
 * A product whose workspace exceeds the 32 MiB is rejected with TDG_EINVAL
 * before any device work.  Every call reuses the same array (it keeps the
 * previous call's contents; each call clears what must start at zero), so
 * calls whose device work overlaps — different streams, or threads sharing a
 * device — race: order them on one stream.  The first call on a device looks
 * up the array's device address (with that device current) and caches it.
 * The paper has no counterpart to this entry point.
 */
tdg_status tdgemm_run_static(char transA, char transB, int64_t M, int64_t N, int64_t K,
                             int64_t lda, int64_t ldb, int64_t ldc, int L, int W,
                             tdg_dtype dtype, tdg_form form, int bits, const void *A,
                             const void *B, void *C, double alpha, double beta, void *stream);

/*
 * Test of the device-side failure path (the library's own, not the paper's):
 * every device wait is bounded and, when its limit passes, the kernel records
 * TDG_ETIMEOUT, lets the copies it issued land, frees what it holds and
 * returns.  With limit_ns > 0, every later tdgemm_gemm of this plan makes the
 * CUDA-core GEMM kernel's first wait for its operand tiles wait instead on a
 * barrier that nothing completes, for limit_ns nanoseconds; the kernel then
 * takes that path, tdgemm_plan_info reports device_status TDG_ETIMEOUT, and
 * C is left unspecified.  The next tdgemm_quantize_pack clears the status.
 * 0 turns the test off.  PLAIN, SYM and ASYM forms without TDG_PAIR_EXACT;
 * limit_ns in [0, 1e9]; TDG_EINVAL otherwise.
 */
tdg_status tdgemm_set_wait_test(tdgemm_plan_t plan, int64_t limit_ns);

/*
 * Measurement aid for the roofline of the CUDA-core forms (not part of the
 * paper's method): one launch of independent fused multiply-add chains on
 * every SM, no memory traffic, on `stream` (asynchronous; time it with
 * events around the call).  dtype TDG_F32 runs the packed fma.rn.f32x2 the
 * fp32 GEMM uses, TDG_F64 scalar fma.rn.f64.  iters >= 1 chain steps per
 * thread; *flops (host) receives the floating-point operations the launch
 * performs (2 per fused multiply-add).
 */
tdg_status tdgemm_fma_probe(tdg_dtype dtype, int64_t iters, double *flops, void *stream);

/* Message of the last failing call on this thread ("" if none). */
const char *tdgemm_last_error(void);

/* Library version string. */
const char *tdgemm_version(void);

#ifdef __cplusplus
}
#endif

#endif /* TDGEMM_H */
