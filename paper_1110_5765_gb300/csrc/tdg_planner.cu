// Step (a), second half: choosing W, z and the companders on the device.
//
// * Fixed-bit mode: gamma_A = gamma_B = 2^(bits-1) - 1, R_max = L gamma^2
//   (eq. 17 with c = gamma / max|x|), z = 2^-q by eq. 15, W as requested.
// * Target mode (Prop. 4, eqs. 26-27, and Sec. 6 with one W per call): the
//   noise of eq. 21 summed over all subblock products (i, l, j) factorises
//   into four per-slab aggregates, so every candidate R_max level costs O(1):
//     N = L T1 / (12 gB^2) + L T2 / (12 gA^2) + T3 (L/144 + s^2) / (gA gB)^2,
//     S = L sum_l (sum_i sigma_A^2)(sum_j sigma_B^2).
//   For each W from the request down to 2 the CTA evaluates every level in
//   parallel, takes the argmin of N (eq. 27's argmax of the SNR; ties go to the
//   lower level) and keeps the first W whose SNR meets the target.  Otherwise
//   W = 1 (plain product) with TDG_ALLOW_FALLBACK, else TDG_EUNREACHABLE.
// * Manual mode: given q and uniform companders (the Sec. 4.B protocol).
// Then a grid-wide kernel writes c (in T) and s = 1/c (fp64) per block and the
// de-companding factors (T)(s_A,il s_B,lj) for every (l, i, j).
#include <math.h>

#include "tdg_common.cuh"
#include "tdg_internal.h"

namespace tdg {

namespace {


// The plain product (form PLAIN, or the W = 1 fallback of target mode for the
// packed forms) uses no companders.
__device__ inline bool needs_companders(const PlanParams &pp, const DevPlan &a) {
    if (pp.form == TDG_PLAIN) return false;
    if ((pp.form == TDG_SYM || pp.form == TDG_ASYM) && pp.mode == MODE_TARGET && a.W == 1)
        return false;
    return true;
}

__device__ inline int t_max_for(int p) { return p == 24 ? 4 * 24 : 4 * 40; }


// eq. 21 summed over (i, l, j); operation order as written above.  With rms
// the representation term is scaled by the blocks' crest factors (s measured
// on uniform integers, RMS = max / sqrt(3)): 9 s^2 sum(sigma_A^2 sigma_B^2).
__device__ inline double model_noise(const DevPlan &a, int L, double gA, double gB, double s,
                                     int rms) {
    double t1 = __ddiv_rn(__dmul_rn((double)L, a.T1), __dmul_rn(__dmul_rn(12.0, gB), gB));
    double t2 = __ddiv_rn(__dmul_rn((double)L, a.T2), __dmul_rn(__dmul_rn(12.0, gA), gA));
    const double g2 = __dmul_rn(__dmul_rn(__dmul_rn(gA, gA), gB), gB);
    if (!rms) {
        double t3 = __ddiv_rn(__dmul_rn(a.T3, __dadd_rn(__ddiv_rn((double)L, 144.0), __dmul_rn(s, s))), g2);
        return __dadd_rn(__dadd_rn(t1, t2), t3);
    }
    double t3 = __ddiv_rn(__dmul_rn(a.T3, __ddiv_rn((double)L, 144.0)), g2);
    double t4 = __ddiv_rn(__dmul_rn(__dmul_rn(9.0, __ddiv_rn(a.S, (double)L)), __dmul_rn(s, s)), g2);
    return __dadd_rn(__dadd_rn(__dadd_rn(t1, t2), t3), t4);
}

__device__ inline double snr_db(double S, double N) {
    return N <= 0.0 ? INFINITY : 10.0 * log10(S / N);
}

// S / L, T1, T2, T3: products of the per-slab aggregates summed over slabs by
// one warp (lanes over l, then a fixed xor tree); every caller gets the same
// bits.
__device__ inline void slab_totals(const PlanParams &pp, const double *__restrict__ agg,
                                   double &S, double &T1, double &T2, double &T3) {
    const int lane = threadIdx.x & 31;
    S = T1 = T2 = T3 = 0.0;
    if (pp.mode != MODE_MANUAL) {
        for (int l = lane; l < pp.nK; l += 32) {
            const double X = __ldcg(&agg[4 * (long long)l]), MA = __ldcg(&agg[4 * (long long)l + 1]);
            const double Y = __ldcg(&agg[4 * (long long)l + 2]), MB = __ldcg(&agg[4 * (long long)l + 3]);
            S += X * Y;
            T1 += X * MB;
            T2 += Y * MA;
            T3 += MA * MB;
        }
    }
#pragma unroll
    for (int off = 16; off > 0; off >>= 1) {
        S += __shfl_xor_sync(0xffffffffu, S, off);
        T1 += __shfl_xor_sync(0xffffffffu, T1, off);
        T2 += __shfl_xor_sync(0xffffffffu, T2, off);
        T3 += __shfl_xor_sync(0xffffffffu, T3, off);
    }
}

__device__ inline double rho_of(double T1, double T2) {
    return (T1 <= 0.0 || T2 <= 0.0) ? 1.0 : sqrt(T2 / T1);
}

// Per-slab aggregates (slab_aggregate_warp): one warp per slab on its own SM
// (GB300's fp64 rate is a small fraction of fp32, so the sums are spread over
// the GPU rather than serialised on one SM).  The last warp to finish (a
// counter in the plan record, no waiting) sums the slabs and forms rho once,
// for every candidate and the decision to read.
__global__ void __launch_bounds__(32) slab_aggregates_kernel(PlanParams pp,
                                                             const double *__restrict__ mA,
                                                             const double *__restrict__ vA,
                                                             const double *__restrict__ mB,
                                                             const double *__restrict__ vB,
                                                             double *__restrict__ agg,
                                                             DevPlan *plan) {
    pdl_entry();
    if (pp.mode == MODE_MANUAL) return;
    slab_aggregate_warp((int)blockIdx.x, pp.nM, pp.nK, pp.nN, mA, vA, mB, vB, agg);
    unsigned int prev = 0;
    if ((threadIdx.x & 31) == 0) {      // the lane that wrote this slab's aggregates
        __threadfence();
        prev = atomicAdd(&plan->aggs_done, 1u);
    }
    prev = __shfl_sync(0xffffffffu, prev, 0);
    if (prev + 1 != gridDim.x) return;
    __threadfence();
    double S, T1, T2, T3;
    slab_totals(pp, agg, S, T1, T2, T3);
    if ((threadIdx.x & 31) == 0) {
        plan->tS = S;
        plan->tT1 = T1;
        plan->tT2 = T2;
        plan->tT3 = T3;
        plan->trho = rho_of(T1, T2);
    }
}

// The slab sums and rho the last aggregate CTA wrote (zero for manual plans,
// which launch no aggregates)
__device__ inline void load_totals(const PlanParams &pp, const DevPlan *plan, double &S, double &T1,
                                   double &T2, double &T3, double &rho) {
    if (pp.mode == MODE_MANUAL) {
        S = T1 = T2 = T3 = 0.0;
        rho = rho_of(0.0, 0.0);
        return;
    }
    S = __ldcg(&plan->tS);
    T1 = __ldcg(&plan->tT1);
    T2 = __ldcg(&plan->tT2);
    T3 = __ldcg(&plan->tT3);
    rho = __ldcg(&plan->trho);
}

// Target mode, packed forms: every candidate (W, R_max level t) evaluated in
// full by one lane (companders, z, representation noise, model noise and
// SNR), 32 candidates per CTA spread over SMs: fp64 divisions, square roots
// and logarithms are slow on GB300 and would serialise on one SM.  n < 0
// marks a level without usable companders or representation-noise value.
struct LevelRec {
    double n, pred, s;
    long long R;
    int gA, gB, q, Wef;
};
static_assert(sizeof(LevelRec) == kLevelRecDoubles * sizeof(double), "planner workspace record");

// a candidate record written by another CTA of the same grid: read from L2
__device__ inline LevelRec load_rec(const LevelRec *p) {
    LevelRec r;
    r.n = __ldcg(&p->n);
    r.pred = __ldcg(&p->pred);
    r.s = __ldcg(&p->s);
    r.R = __ldcg(&p->R);
    r.gA = __ldcg(&p->gA);
    r.gB = __ldcg(&p->gB);
    r.q = __ldcg(&p->q);
    r.Wef = __ldcg(&p->Wef);
    return r;
}

// The plan, decided by one full warp: fixed bits, manual parameters, the
// tensor-core forms, or (target mode, packed forms) the choice among the
// candidate records res: for W from the request down to 2 the level of least
// model noise (eq. 27's argmax of the SNR; ties to the lower level), the first
// W whose SNR meets the target; else the plain product (fallback) or
// TDG_EUNREACHABLE.  Lane 0 writes the plan.
__device__ void decide_plan(const PlanParams &pp, const double *__restrict__ agg,
                            const double *__restrict__ stab, const LevelRec *res, DevPlan *plan) {
    const int lane = threadIdx.x & 31;
    const int L = pp.L;
    double S, T1, T2, T3, rho;
    load_totals(pp, plan, S, T1, T2, T3, rho);
    DevPlan a{};
    a.S = (double)L * S;
    a.T1 = T1;
    a.T2 = T2;
    a.T3 = T3;
    a.status = 0;
    a.level = -1;
    a.pred_snr = NAN;
    a.s_rep = 0.0;

    if (pp.form == TDG_PLAIN) {
        a.W = 1; a.q = 0; a.gA = a.gB = 0; a.R = 0; a.Wef = 0;
    } else if (pp.form == TDG_TC_FP8) {
        a.W = 1; a.q = 0; a.gA = a.gB = (int)kFp8Max; a.R = 0; a.Wef = 0;
    } else if (pp.form == TDG_TC_INT) {
        int gA, gB;
        if (pp.mode == MODE_FIXED) {
            gA = gB = (1 << (pp.bits - 1)) - 1;
        } else {
            split_gammas((long long)kTcIntExact, L, rho, gA, gB);
            gA = min(gA, kTcIntMaxGamma);
            gB = min(min(gB, kTcIntMaxGamma), (int)((long long)kTcIntExact / ((long long)L * gA)));
        }
        a.W = 1; a.gA = gA; a.gB = gB; a.R = (long long)L * gA * gB;
        a.q = q_for(a.R); a.Wef = w_ef(a.R, a.q, pp.p);
        a.pred_snr = snr_db(a.S, model_noise(a, L, gA, gB, 0.0, pp.noise_rms));
        if (pp.mode == MODE_TARGET && a.pred_snr < pp.target_db) a.status = TDG_EUNREACHABLE;
    } else if (pp.mode == MODE_MANUAL) {
        a.W = pp.Wreq; a.q = pp.manual_q; a.gA = a.gB = 0; a.R = 0; a.Wef = 0;
    } else if (pp.mode == MODE_FIXED) {
        int g = (1 << (pp.bits - 1)) - 1;
        a.W = pp.Wreq; a.gA = a.gB = g; a.R = (long long)L * g * g;
        a.q = q_for(a.R); a.Wef = w_ef(a.R, a.q, pp.p);
        double s = -1.0;
        if (a.W <= a.Wef) {
            s = 0.0;
        } else if (stab) {
            int tbest = -1;
            for (int t = 0; t <= t_max_for(pp.p); ++t)
                if (r_level(t) <= a.R) tbest = t;
            if (tbest >= pp.t0 && tbest < pp.t0 + pp.nt)
                s = stab[(pp.Wreq - 2) * pp.nt + (tbest - pp.t0)];
        }
        if (s >= 0.0) {
            a.pred_snr = snr_db(a.S, model_noise(a, L, g, g, s, pp.noise_rms));
            a.s_rep = s;
        }
    } else {  // MODE_TARGET, packed forms
        int t_lo = 0;
        while (r_level(t_lo) < L) ++t_lo;
        const int t_hi = t_max_for(pp.p);
        bool chosen = false;
        DevPlan first{};
        bool have_first = false;
        for (int W = pp.Wreq; W >= 2 && !chosen; --W) {
            // argmin of N over the levels (ties to the lower level); N >= 0,
            // so its bit pattern orders like its value (integer compares)
            // every load of the lane's levels issued before any is used
            constexpr int kPerLane = (kMaxLevels + 31) / 32;
            double nv[kPerLane];
#pragma unroll
            for (int u = 0; u < kPerLane; ++u) {
                const int t = t_lo + lane + 32 * u;
                nv[u] = t <= t_hi ? __ldcg(&res[(W - 2) * kMaxLevels + t].n) : -1.0;
            }
            unsigned long long bn = ~0ull;
            int bt = -1;
#pragma unroll
            for (int u = 0; u < kPerLane; ++u) {     // lanes scan ascending t
                if (nv[u] < 0.0) continue;
                const unsigned long long nb = (unsigned long long)__double_as_longlong(nv[u]);
                if (nb < bn) { bn = nb; bt = t_lo + lane + 32 * u; }
            }
#pragma unroll
            for (int off = 16; off > 0; off >>= 1) {
                const unsigned long long n2 = __shfl_xor_sync(0xffffffffu, bn, off);
                const int t2 = __shfl_xor_sync(0xffffffffu, bt, off);
                if (t2 >= 0 && (bt < 0 || n2 < bn || (n2 == bn && t2 < bt))) {
                    bn = n2;
                    bt = t2;
                }
            }
            const int t = bt;                          // the same in every lane
            if (t < 0) continue;
            const LevelRec r = load_rec(&res[(W - 2) * kMaxLevels + t]);
            DevPlan c = a;
            c.W = W;
            c.q = r.q;
            c.gA = r.gA;
            c.gB = r.gB;
            c.R = r.R;
            c.Wef = r.Wef;
            c.level = t;
            c.pred_snr = r.pred;
            c.s_rep = r.s;
            if (!have_first) { first = c; have_first = true; }
            if (c.pred_snr >= pp.target_db) { a = c; chosen = true; }
        }
        if (!chosen) {
            if (pp.allow_fallback) {
                a.W = 1; a.q = 0; a.gA = a.gB = 0; a.R = 0; a.Wef = 0; a.level = -1;
                a.pred_snr = INFINITY;
            } else if (have_first) {
                a = first;
                a.status = TDG_EUNREACHABLE;
            } else {
                a.W = pp.Wreq; a.q = q_for(L); a.gA = a.gB = 1; a.R = L; a.Wef = 0;
                a.status = TDG_EUNREACHABLE;
            }
        }
    }
    if (lane == 0) {
        const int nf = __ldcg(&plan->nonfinite);
        a.nonfinite = nf;
        if (nf && a.status == 0) a.status = TDG_ENONFINITE;
        *plan = a;
    }
}

// Target mode, packed forms: each lane evaluates one candidate (W, R_max
// level t) in full -- companders, z, representation noise, model noise and
// SNR -- 32 candidates per CTA spread over SMs (fp64 divisions, square roots
// and logarithms are slow on GB300 and would serialise on one SM).  The last
// CTA to finish (a counter in the plan, no waiting) then decides the plan
// from all records.  n < 0 marks a level without usable companders or
// representation-noise value.
__global__ void __launch_bounds__(32) level_kernel(PlanParams pp, const double *__restrict__ agg,
                                                   const double *__restrict__ stab,
                                                   LevelRec *res, DevPlan *plan) {
    pdl_entry();
    const int L = pp.L;
    const int lane = threadIdx.x;
    int t_lo = 0;
    while (r_level(t_lo) < L) ++t_lo;
    const int t_hi = t_max_for(pp.p);
    const int nlev = t_hi - t_lo + 1;
    const int per_w = (nlev + 31) / 32;                 // CTAs per W
    const int W = pp.Wreq - (int)blockIdx.x / per_w;
    const int t = t_lo + ((int)blockIdx.x % per_w) * 32 + lane;
    double S, T1, T2, T3, rho;
    load_totals(pp, plan, S, T1, T2, T3, rho);
    if (W >= 2 && t <= t_hi) {
        DevPlan a{};
        a.S = (double)L * S; a.T1 = T1; a.T2 = T2; a.T3 = T3;
        LevelRec r{};
        r.n = -1.0;
        const long long Rt = r_level(t);
        r.q = q_for(Rt);
        split_gammas(Rt, L, rho, r.gA, r.gB);
        if (r.gA >= 1) {
            r.R = (long long)L * r.gA * r.gB;
            r.Wef = w_ef(r.R, r.q, pp.p);
            double sv = -1.0;
            if (W <= r.Wef) sv = 0.0;
            else if (stab && t >= pp.t0 && t < pp.t0 + pp.nt) sv = stab[(W - 2) * pp.nt + (t - pp.t0)];
            if (sv >= 0.0) {
                r.n = model_noise(a, L, r.gA, r.gB, sv, pp.noise_rms);
                r.pred = snr_db(a.S, r.n);
                r.s = sv > 0.0 ? sv : 0.0;
            }
        }
        res[(W - 2) * kMaxLevels + t] = r;
    }
    // the records of this CTA are written: count it; the last one decides
    __threadfence();
    __syncwarp();
    unsigned int prev = 0;
    if (lane == 0) prev = atomicAdd(&plan->levels_done, 1u);
    prev = __shfl_sync(0xffffffffu, prev, 0);
    if (prev + 1 == gridDim.x) {
        __threadfence();
        decide_plan(pp, agg, stab, res, plan);
    }
}

// The plan for every mode but the packed forms' target mode (one warp).
__global__ void __launch_bounds__(32) planner_kernel(PlanParams pp, const double *__restrict__ agg,
                                                     const double *__restrict__ stab,
                                                     const LevelRec *res, DevPlan *plan) {
    pdl_entry();
    decide_plan(pp, agg, stab, res, plan);
}

// c = gamma / max|x| (fp64, rounded to T for eq. 3), s = 1/c, per block.
template <typename T>
__global__ void scales_kernel(PlanParams pp, const double *__restrict__ mA,
                              const double *__restrict__ mB, const DevPlan *__restrict__ plan,
                              T *cA, double *sA, T *cB, double *sB) {
    pdl_entry();
    const long long nAblk = (long long)pp.nM * pp.nK, nBblk = (long long)pp.nK * pp.nN;
    const long long idx = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    const DevPlan a = *plan;
    if (!needs_companders(pp, a)) return;  // plain product: nothing to compand
    for (long long k = idx; k < nAblk + nBblk; k += (long long)gridDim.x * blockDim.x) {
        const bool isA = k < nAblk;
        const long long b = isA ? k : k - nAblk;
        double m = isA ? mA[b] : mB[b];
        double c;
        if (pp.mode == MODE_MANUAL) c = isA ? pp.manual_cA : pp.manual_cB;
        else c = m > 0.0 ? __ddiv_rn((double)(isA ? a.gA : a.gB), m) : 0.0;
        double s = c > 0.0 ? __ddiv_rn(1.0, c) : 0.0;
        if (isA) { cA[b] = (T)c; sA[b] = s; }
        else { cB[b] = (T)c; sB[b] = s; }
    }
}

// (T)(s_A,il * s_B,lj) for every (l, i, j), layout [l][i][j]
template <typename T>
__global__ void pairs_kernel(PlanParams pp, const double *__restrict__ sA,
                             const double *__restrict__ sB, const DevPlan *__restrict__ plan,
                             T *pair) {
    pdl_entry();
    if (!needs_companders(pp, *plan)) return;
    const long long n = (long long)pp.nK * pp.nM * pp.nN;
    for (long long k = (long long)blockIdx.x * blockDim.x + threadIdx.x; k < n;
         k += (long long)gridDim.x * blockDim.x) {
        long long j = k % pp.nN, r = k / pp.nN;
        long long i = r % pp.nM, l = r / pp.nM;
        pair[k] = (T)__dmul_rn(sA[i * pp.nK + l], sB[l * pp.nN + j]);
    }
}

// ---- Sec. 6: per inner kernel R_ij, predicted S_ij / N_ij with the call's
// companders.  One warp per inner kernel: lane u computes the terms of slab
// l0 + u, then every lane adds them in ascending l (the oracle's order), so
// the FP64 divisions spread over the warp while the sums keep their order.
__device__ inline void kernel_terms(const PlanParams &pp, const DevPlan &a, double va,
                                    double vb, double ma, double mb, double &s_out,
                                    double &n_out) {
    const double L = (double)pp.L;
    const double gA2 = __dmul_rn((double)a.gA, (double)a.gA), gB2 = __dmul_rn((double)a.gB, (double)a.gB);
    const double s = a.s_rep;
    const double ma2 = __dmul_rn(ma, ma), mb2 = __dmul_rn(mb, mb);
    s_out = __dmul_rn(__dmul_rn(L, va), vb);
    double n = __dadd_rn(__ddiv_rn(__dmul_rn(__dmul_rn(L, va), mb2), __dmul_rn(12.0, gB2)),
                         __ddiv_rn(__dmul_rn(__dmul_rn(L, vb), ma2), __dmul_rn(12.0, gA2)));
    if (pp.noise_rms) {
        n = __dadd_rn(n, __ddiv_rn(__dmul_rn(__dmul_rn(ma2, mb2), __ddiv_rn(L, 144.0)),
                                   __dmul_rn(gA2, gB2)));
        n = __dadd_rn(n, __ddiv_rn(__dmul_rn(__dmul_rn(__dmul_rn(9.0, va), vb), __dmul_rn(s, s)),
                                   __dmul_rn(gA2, gB2)));
    } else {
        n = __dadd_rn(n, __ddiv_rn(__dmul_rn(__dmul_rn(ma2, mb2),
                                             __dadd_rn(__ddiv_rn(L, 144.0), __dmul_rn(s, s))),
                                   __dmul_rn(gA2, gB2)));
    }
    n_out = n;
}

__global__ void kernel_ratio_kernel(PlanParams pp, const double *__restrict__ mA,
                                    const double *__restrict__ vA, const double *__restrict__ mB,
                                    const double *__restrict__ vB, const DevPlan *__restrict__ plan,
                                    double *ratio) {
    pdl_entry();
    const long long T = (long long)pp.nM * pp.nN;
    const long long t = ((long long)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    const int lane = threadIdx.x & 31;
    if (t >= T) return;                      // uniform per warp
    const int i = (int)(t / pp.nN), j = (int)(t % pp.nN);
    const DevPlan a = *plan;
    if (a.W < 2) {
        if (lane == 0) ratio[t] = 0.0;
        return;
    }
    double S = 0.0, N = 0.0;
    for (int l0 = 0; l0 < pp.nK; l0 += 32) {
        const int l = l0 + lane;
        double sv = 0.0, nv = 0.0;
        if (l < pp.nK)
            kernel_terms(pp, a, vA[(long long)i * pp.nK + l], vB[(long long)l * pp.nN + j],
                         mA[(long long)i * pp.nK + l], mB[(long long)l * pp.nN + j], sv, nv);
        const int cnt = min(32, pp.nK - l0);
        for (int u = 0; u < cnt; ++u) {
            S = __dadd_rn(S, __shfl_sync(0xffffffffu, sv, u));
            N = __dadd_rn(N, __shfl_sync(0xffffffffu, nv, u));
        }
    }
    if (lane == 0) ratio[t] = N > 0.0 ? __ddiv_rn(S, N) : INFINITY;
}

// Sec. 6 (ii): the fewest of T inner kernels whose acceleration makes the
// product's predicted throughput T / ((T - k) + k / F_W) reach F, i.e.
// k = ceil(T (1 - 1/F) / (1 - 1/F_W)); none if F <= 1 or F_W <= 1, all if
// F >= F_W.  Every operation rounded as written (the oracle's order).
__device__ inline long long kernels_for_throughput(long long T, double F, double fw) {
    if (!(F > 1.0) || !(fw > 1.0)) return 0;
    if (F >= fw) return T;
    const double x = __ddiv_rn(__dmul_rn((double)T, __dsub_rn(1.0, __ddiv_rn(1.0, F))),
                               __dsub_rn(1.0, __ddiv_rn(1.0, fw)));
    const long long k = (long long)ceil(x);
    return k < 0 ? 0 : (k > T ? T : k);
}

// mode 1: ratio >= thr;  mode 2: rank (descending ratio, ties to the lower
// index) below k, counted against the ratios staged through shared memory;
// mode 3: as mode 2 with k from the throughput target.  Ratios are
// non-negative (or +inf), so their bit patterns order like the values and the
// O(T^2) rank count runs on the integer pipe.  A plan that fell back to W = 1
// accelerates nothing.
constexpr int kMaskThreads = 128, kMaskChunk = 2048;
__global__ void __launch_bounds__(kMaskThreads)
    kernel_mask_kernel(long long T, int mode, double thr, long long k, double F, Speedups fw,
                       const DevPlan *__restrict__ plan, const double *__restrict__ ratio,
                       unsigned char *mask) {
    pdl_entry();
    __shared__ unsigned long long chunk[kMaskChunk];
    const long long t = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    const int W = plan->W;
    const bool fell_back = W < 2;            // uniform
    if (mode == 3 && !fell_back) k = kernels_for_throughput(T, F, fw.fw[min(W, kMaxW)]);
    if (fell_back || mode == 1) {
        if (t < T) mask[t] = fell_back ? 0 : (ratio[t] >= thr ? 1 : 0);
        return;
    }
    const unsigned long long r =
        t < T ? (unsigned long long)__double_as_longlong(ratio[t]) : 0ull;
    long long rank = 0;
    for (long long c0 = 0; c0 < T; c0 += kMaskChunk) {
        const int n = (int)min((long long)kMaskChunk, T - c0);
        __syncthreads();
        for (int u = threadIdx.x; u < n; u += kMaskThreads)
            chunk[u] = (unsigned long long)__double_as_longlong(ratio[c0 + u]);
        __syncthreads();
        const long long tl = t - c0;         // ties count below this index
        for (int u = 0; u < n; ++u) {
            const unsigned long long ru = chunk[u];
            rank += (ru > r || (ru == r && u < tl)) ? 1 : 0;
        }
    }
    if (t < T) mask[t] = rank < k ? 1 : 0;
}

// One CTA: each thread counts the conventional tiles in its contiguous chunk
// of the row-major tile list, a block-wide exclusive scan gives every chunk
// its first position in both groups, and the chunk is written out.
constexpr int kOrderThreads = 1024;
__global__ void __launch_bounds__(kOrderThreads)
    tile_order_kernel(const unsigned char *__restrict__ mask, int nN, int L, int bm, int bn,
                      long long tiles_m, long long ntn, int *__restrict__ order) {
    pdl_entry();
    __shared__ long long scan[kOrderThreads];
    const long long n = tiles_m * ntn;
    const long long chunk = (n + kOrderThreads - 1) / kOrderThreads;
    const long long t0 = min(n, (long long)threadIdx.x * chunk), t1 = min(n, t0 + chunk);
    auto conventional = [&](long long t) {
        const long long tm = t / ntn, tn = t - tm * ntn;
        return mask[(tm * bm / L) * nN + (tn * bn / L)] == 0;
    };
    long long mine = 0;
    for (long long t = t0; t < t1; ++t) mine += conventional(t) ? 1 : 0;
    scan[threadIdx.x] = mine;
    __syncthreads();
    for (int off = 1; off < kOrderThreads; off <<= 1) {     // inclusive scan
        const long long v = threadIdx.x >= off ? scan[threadIdx.x - off] : 0;
        __syncthreads();
        scan[threadIdx.x] += v;
        __syncthreads();
    }
    const long long total_conv = scan[kOrderThreads - 1];
    long long pc = scan[threadIdx.x] - mine;                 // conventional tiles before t0
    long long pp = total_conv + (t0 - pc);                   // accelerated tiles before t0, offset
    for (long long t = t0; t < t1; ++t) {
        if (conventional(t)) order[pc++] = (int)t;
        else order[pp++] = (int)t;
    }
}

}  // namespace

cudaError_t launch_tile_order(const unsigned char *mask, int nN, int L, int bm, int bn,
                              long long tiles_m, long long ntn, int *order, cudaStream_t st) {
    return launch_pdl(tile_order_kernel, dim3(1), dim3(kOrderThreads), 0, st, mask, nN, L, bm,
                      bn, tiles_m, ntn, order);
}

cudaError_t launch_kernel_control(const PlanParams &pp, const double *mA, const double *vA,
                                  const double *mB, const double *vB, const DevPlan *plan,
                                  int mode, double thr, long long k, double F,
                                  const Speedups &fw, double *ratio, unsigned char *mask,
                                  cudaStream_t st) {
    const long long T = (long long)pp.nM * pp.nN;
    cudaError_t e = launch_pdl(kernel_ratio_kernel, dim3((unsigned)((T * 32 + 255) / 256)),
                               dim3(256), 0, st, pp, mA, vA, mB, vB, plan, ratio);
    if (e != cudaSuccess) return e;
    return launch_pdl(kernel_mask_kernel,
                      dim3((unsigned)((T + kMaskThreads - 1) / kMaskThreads)), dim3(kMaskThreads),
                      0, st, T, mode, thr, k, F, fw, plan, (const double *)ratio, mask);
}

template <typename T>
cudaError_t launch_planner(const PlanParams &pp, const double *mA, const double *eA,
                           const double *mB, const double *eB, const double *stab,
                           DevPlan *plan, double *agg, T *cA, double *sA, T *cB, double *sB,
                           T *pair, cudaStream_t st, bool scales_done) {
    // agg: 4 nK per-slab aggregates, then one record per candidate (W, level)
    LevelRec *res = reinterpret_cast<LevelRec *>(agg + 4 * (long long)pp.nK);
    if (pp.mode != MODE_MANUAL) {
        cudaError_t e0 = launch_pdl(slab_aggregates_kernel, dim3(pp.nK), dim3(32), 0, st, pp, mA, eA,
                                    mB, eB, agg, plan);
        if (e0 != cudaSuccess) return e0;
    }
    cudaError_t e;
    if (pp.mode == MODE_TARGET && (pp.form == TDG_SYM || pp.form == TDG_ASYM)) {
        // every candidate level, the plan decided by the last CTA to finish
        int t_lo = 0;
        while (r_level(t_lo) < pp.L) ++t_lo;
        const int nlev = (pp.p == 24 ? 4 * 24 : 4 * 40) - t_lo + 1;
        const int ctas = max(1, (pp.Wreq - 1) * ((nlev + 31) / 32));
        e = launch_pdl(level_kernel, dim3(ctas), dim3(32), 0, st, pp, (const double *)agg, stab,
                       res, plan);
    } else {
        e = launch_pdl(planner_kernel, dim3(1), dim3(32), 0, st, pp, (const double *)agg, stab,
                       (const LevelRec *)res, plan);
    }
    if (e != cudaSuccess) return e;
    if (!scales_done) {
        long long nblk = (long long)pp.nM * pp.nK + (long long)pp.nK * pp.nN;
        int g = (int)min((nblk + 255) / 256, 4096LL);
        e = launch_pdl(scales_kernel<T>, dim3(g), dim3(256), 0, st, pp, mA, mB,
                       (const DevPlan *)plan, cA, sA, cB, sB);
        if (e != cudaSuccess) return e;
    }
    long long np = (long long)pp.nK * pp.nM * pp.nN;
    int g = (int)min((np + 255) / 256, 8192LL);
    return launch_pdl(pairs_kernel<T>, dim3(g), dim3(256), 0, st, pp, (const double *)sA,
                      (const double *)sB, (const DevPlan *)plan, pair);
}

template cudaError_t launch_planner<float>(const PlanParams &, const double *, const double *,
                                           const double *, const double *, const double *,
                                           DevPlan *, double *, float *, double *, float *,
                                           double *, float *, cudaStream_t, bool);
template cudaError_t launch_planner<double>(const PlanParams &, const double *, const double *,
                                            const double *, const double *, const double *,
                                            DevPlan *, double *, double *, double *, double *,
                                            double *, double *, cudaStream_t, bool);

}  // namespace tdg
