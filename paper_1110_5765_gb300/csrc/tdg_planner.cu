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

constexpr int kPlanThreads = 256;

// The plain product (form PLAIN, or the W = 1 fallback of target mode for the
// packed forms) uses no companders.
__device__ inline bool needs_companders(const PlanParams &pp, const DevPlan &a) {
    if (pp.form == TDG_PLAIN) return false;
    if ((pp.form == TDG_SYM || pp.form == TDG_ASYM) && pp.mode == MODE_TARGET && a.W == 1)
        return false;
    return true;
}

__device__ inline int t_max_for(int p) { return p == 24 ? 4 * 24 : 4 * 40; }

// integer compander split of eq. 26 for a budget R: gA = floor(sqrt((R/L) rho))
__device__ inline void split_gammas(long long R, int L, double rho, int &gA, int &gB) {
    long long G = R / L;
    if (G < 1) { gA = gB = 0; return; }
    double v = __dsqrt_rn(__dmul_rn(__ddiv_rn((double)R, (double)L), rho));
    long long a = (long long)floor(v);
    if (a < 1) a = 1;
    if (a > G) a = G;
    long long b = R / ((long long)L * a);
    if (b < 1) b = 1;
    gA = (int)min(a, (long long)INT32_MAX);
    gB = (int)min(b, (long long)INT32_MAX);
}

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

__global__ void __launch_bounds__(kPlanThreads) planner_kernel(
    PlanParams pp, const double *__restrict__ mA, const double *__restrict__ vA,
    const double *__restrict__ mB, const double *__restrict__ vB,
    const double *__restrict__ stab, DevPlan *plan) {
    __shared__ double red[4][kPlanThreads];
    __shared__ double best_n[kPlanThreads];
    __shared__ int best_t[kPlanThreads];
    const int tid = threadIdx.x;
    const int L = pp.L;

    // ---- per-slab aggregates X_l, Y_l, MA_l, MB_l and their products
    double S = 0, T1 = 0, T2 = 0, T3 = 0;
    if (pp.mode != MODE_MANUAL) {
        for (int l = tid; l < pp.nK; l += kPlanThreads) {
            double X = 0, MA = 0, Y = 0, MB = 0;
            for (int i = 0; i < pp.nM; ++i) {
                X += vA[(long long)i * pp.nK + l];
                double m = mA[(long long)i * pp.nK + l];
                MA += m * m;
            }
            for (int j = 0; j < pp.nN; ++j) {
                Y += vB[(long long)l * pp.nN + j];
                double m = mB[(long long)l * pp.nN + j];
                MB += m * m;
            }
            S += X * Y;
            T1 += X * MB;
            T2 += Y * MA;
            T3 += MA * MB;
        }
    }
    red[0][tid] = S; red[1][tid] = T1; red[2][tid] = T2; red[3][tid] = T3;
    __syncthreads();
    for (int o = kPlanThreads / 2; o > 0; o >>= 1) {
        if (tid < o)
            for (int k = 0; k < 4; ++k) red[k][tid] += red[k][tid + o];
        __syncthreads();
    }
    DevPlan a;
    a.S = (double)L * red[0][0];
    a.T1 = red[1][0];
    a.T2 = red[2][0];
    a.T3 = red[3][0];
    const double rho = (a.T1 <= 0.0 || a.T2 <= 0.0) ? 1.0 : sqrt(a.T2 / a.T1);
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
            double bn = INFINITY;
            int bt = -1;
            for (int t = t_lo + tid; t <= t_hi; t += kPlanThreads) {
                long long Rt = r_level(t);
                int q = q_for(Rt);
                int gA, gB;
                split_gammas(Rt, L, rho, gA, gB);
                if (gA < 1) continue;
                long long R = (long long)L * gA * gB;
                double s = -1.0;
                if (W <= w_ef(R, q, pp.p)) {
                    s = 0.0;
                } else if (stab && t >= pp.t0 && t < pp.t0 + pp.nt) {
                    s = stab[(W - 2) * pp.nt + (t - pp.t0)];
                }
                if (s < 0.0) continue;
                double n = model_noise(a, L, gA, gB, s, pp.noise_rms);
                if (n < bn) { bn = n; bt = t; }
            }
            best_n[tid] = bn;
            best_t[tid] = bt;
            __syncthreads();
            for (int o = kPlanThreads / 2; o > 0; o >>= 1) {
                if (tid < o) {
                    double n2 = best_n[tid + o];
                    int t2 = best_t[tid + o];
                    if (t2 >= 0 && (best_t[tid] < 0 || n2 < best_n[tid] ||
                                    (n2 == best_n[tid] && t2 < best_t[tid]))) {
                        best_n[tid] = n2;
                        best_t[tid] = t2;
                    }
                }
                __syncthreads();
            }
            const int t = best_t[0];
            const double n = best_n[0];
            __syncthreads();
            if (t < 0) continue;
            DevPlan c = a;
            long long Rt = r_level(t);
            c.W = W;
            c.q = q_for(Rt);
            split_gammas(Rt, L, rho, c.gA, c.gB);
            c.R = (long long)L * c.gA * c.gB;
            c.Wef = w_ef(c.R, c.q, pp.p);
            c.level = t;
            c.pred_snr = snr_db(a.S, n);
            {
                double sc = 0.0;
                if (!(c.W <= w_ef(c.R, c.q, pp.p)) && stab && t >= pp.t0 && t < pp.t0 + pp.nt)
                    sc = stab[(c.W - 2) * pp.nt + (t - pp.t0)];
                c.s_rep = sc > 0.0 ? sc : 0.0;
            }
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
    if (tid == 0) {
        int nf = plan->nonfinite;
        a.nonfinite = nf;
        if (nf && a.status == 0) a.status = TDG_ENONFINITE;
        *plan = a;
    }
}

// c = gamma / max|x| (fp64, rounded to T for eq. 3), s = 1/c, per block.
template <typename T>
__global__ void scales_kernel(PlanParams pp, const double *__restrict__ mA,
                              const double *__restrict__ mB, const DevPlan *__restrict__ plan,
                              T *cA, double *sA, T *cB, double *sB) {
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

// mode 1: ratio >= thr;  mode 2: rank (descending ratio, ties to the lower
// index) below k, counted against the ratios staged through shared memory.
// Ratios are non-negative (or +inf), so their bit patterns order like the
// values and the O(T^2) rank count runs on the integer pipe.  A plan that fell
// back to W = 1 accelerates nothing.
constexpr int kMaskThreads = 128, kMaskChunk = 2048;
__global__ void __launch_bounds__(kMaskThreads)
    kernel_mask_kernel(long long T, int mode, double thr, long long k,
                       const DevPlan *__restrict__ plan, const double *__restrict__ ratio,
                       unsigned char *mask) {
    __shared__ unsigned long long chunk[kMaskChunk];
    const long long t = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    const bool fell_back = plan->W < 2;      // uniform
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

}  // namespace

cudaError_t launch_kernel_control(const PlanParams &pp, const double *mA, const double *vA,
                                  const double *mB, const double *vB, const DevPlan *plan,
                                  int mode, double thr, long long k, double *ratio,
                                  unsigned char *mask, cudaStream_t st) {
    const long long T = (long long)pp.nM * pp.nN;
    kernel_ratio_kernel<<<(int)((T * 32 + 255) / 256), 256, 0, st>>>(pp, mA, vA, mB, vB, plan,
                                                                      ratio);
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return e;
    kernel_mask_kernel<<<(int)((T + kMaskThreads - 1) / kMaskThreads), kMaskThreads, 0, st>>>(
        T, mode, thr, k, plan, ratio, mask);
    return cudaGetLastError();
}

template <typename T>
cudaError_t launch_planner(const PlanParams &pp, const double *mA, const double *eA,
                           const double *mB, const double *eB, const double *stab,
                           DevPlan *plan, T *cA, double *sA, T *cB, double *sB, T *pair,
                           cudaStream_t st) {
    planner_kernel<<<1, kPlanThreads, 0, st>>>(pp, mA, eA, mB, eB, stab, plan);
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return e;
    long long nblk = (long long)pp.nM * pp.nK + (long long)pp.nK * pp.nN;
    int g = (int)min((nblk + 255) / 256, 4096LL);
    scales_kernel<T><<<g, 256, 0, st>>>(pp, mA, mB, plan, cA, sA, cB, sB);
    e = cudaGetLastError();
    if (e != cudaSuccess) return e;
    long long np = (long long)pp.nK * pp.nM * pp.nN;
    g = (int)min((np + 255) / 256, 8192LL);
    pairs_kernel<T><<<g, 256, 0, st>>>(pp, sA, sB, plan, pair);
    return cudaGetLastError();
}

template cudaError_t launch_planner<float>(const PlanParams &, const double *, const double *,
                                           const double *, const double *, const double *,
                                           DevPlan *, float *, double *, float *, double *,
                                           float *, cudaStream_t);
template cudaError_t launch_planner<double>(const PlanParams &, const double *, const double *,
                                            const double *, const double *, const double *,
                                            DevPlan *, double *, double *, double *, double *,
                                            double *, cudaStream_t);

}  // namespace tdg
