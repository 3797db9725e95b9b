// moss_finalize.cu -- estimators and variances in FP64 on the device.
//
//   MOSS-4 (Sec. 4.1.2, Theorems 2-3): p_i = 2 phi^(1)_i / Gamma,
//     n_i = m_i / (K p_i), i in {1,3,4,5,6}; n_2 = Lambda_3 - n_4 - 2 n_5 - 4 n_6
//     (eq. 2); Var(n_i) = n_i/K (1/p_i - n_i); Var(n_2) of Theorem 3.  The
//     collisions r = w are triangles, each reached by 6 ordered draws of
//     probability 1/Gamma, so they also estimate the triangle count.
//   MOSS-5 (Theorems 6-10, Sec. 5.1.3): eta^(l)_i = m^(l)_i / (K_l p^(l)_i),
//     p^(l)_i = 2 phi^(l)_i / Gamma^(l); classes of Omega_1 and Omega_2 are
//     mixed with lambda^(1) = V2/(V1+V2), lambda^(2) = V1/(V1+V2); eta_2 =
//     Lambda_4 - sum_{Omega_3*} phi^(3)_i eta_i with the variance of Theorem 10
//     and the covariances Cov(eta_i, eta_j) = -eta_i eta_j sum_l a_i a_j / K_l.
//   The unknown eta in a variance is replaced by the estimate (one source) or
//   by the pooled value (m1 + m2) / (K1 p1 + K2 p2) (two sources).
//   MOSS-4 with MOSS-4Min (Sec. 4.2, Theorems 1 and 5): a MOSS-4Min hit of
//     class i in {3, 5, 6} whose CIS has c centred 3-paths was drawn with
//     probability 2 c / Gamma-check, so n-check_i = Gamma-check / (2 K-check)
//     sum_c m_{i,c} / c; Var(n-check_i) = (S_i - n_i^2) / K-check with
//     S_i = n_i Gamma-check h_i / 2, h_i the mean of 1/c over the class
//     (sum_c m_{i,c}/c^2 over sum_c m_{i,c}/c; 1, 1, 1/3 without hits, the
//     values of Theorem 4).  Both variances take the plug-in
//     n_i = (K n-hat_i + K-check n-check_i) / (K + K-check), the weights are
//     V_other / (V_1 + V_2) (Theorem 1), n_2 follows eq. (2).
#include "../../include/moss.h"
#include "moss_internal.cuh"

namespace moss {

namespace {

// Sec. 4.1.2: copies of M_1^(4) in M_1..M_6 (phi^(1)) and of M_2^(4) (phi^(2))
__device__ const double kPhi4[6][2] = {{1, 0}, {0, 1}, {4, 0}, {2, 1}, {6, 2}, {12, 4}};
// Table 2: forks, 5-paths, 4-stars in M_1^(5)..M_21^(5)
__device__ const double kPhi5[21][3] = {
    {0, 1, 0},  {0, 0, 1},  {1, 0, 0},   {1, 2, 0},   {2, 2, 0},   {0, 5, 0},   {2, 1, 0},
    {2, 0, 1},  {4, 4, 0},  {4, 7, 0},   {5, 2, 1},   {4, 4, 1},   {6, 6, 0},   {10, 10, 1},
    {9, 6, 1},  {12, 6, 2}, {10, 14, 0}, {20, 24, 1}, {20, 18, 2}, {36, 36, 3}, {60, 60, 5}};

__device__ __forceinline__ double u128_to_double(u128 x) {
    return (double)(uint64_t)(x >> 64) * 18446744073709551616.0 + (double)(uint64_t)x;
}

__device__ __forceinline__ double warp_sum_d(double v) {
#pragma unroll
    for (int d = 16; d > 0; d >>= 1) v += __shfl_xor_sync(0xffffffffu, v, d);
    return v;
}

// MOSS-5 with one warp: lane i is class i (1..21); the sums over classes
// (the eta_2 identity, its variance, the concentrations) are warp sums.
// hits0/hits1: counts of the two sub-methods (either may be null); cov
// (nullable, 22 x 22 row-major) receives the covariance matrix.
__device__ void finalize5_warp(const FinalizeIn &in, const uint64_t *hits0, const uint64_t *hits1,
                               const DevTotals *tot, moss_result *out, double *cov) {
    const int i = threadIdx.x & 31;
    const bool cls = i >= 1 && i <= 21;
    const double G0 = u128_to_double(tot->gamma[1]), G1 = u128_to_double(tot->gamma[2]);
    const double K0 = (double)in.K[0], K1 = (double)in.K[1];
    const bool av0 = in.K[0] > 0 && G0 > 0, av1 = in.K[1] > 0 && G1 > 0;
    const uint64_t h0 = (i < kSlots && hits0) ? hits0[i] : 0, h1 = (i < kSlots && hits1) ? hits1[i] : 0;
    const double f0 = cls ? kPhi5[i - 1][0] : 0.0, f1 = cls ? kPhi5[i - 1][1] : 0.0, f3 = cls ? kPhi5[i - 1][2] : 0.0;
    const bool s0 = av0 && f0 > 0, s1 = av1 && f1 > 0;
    double p0 = 0.0, p1 = 0.0, e0 = 0.0, e1 = 0.0;
    if (s0) {
        p0 = 2.0 * f0 / G0;                               // Theorem 6
        e0 = (double)h0 / (K0 * p0);
    }
    if (s1) {
        p1 = 2.0 * f1 / G1;                               // Theorem 8
        e1 = (double)h1 / (K1 * p1);
    }
    double est = 0.0, var = 0.0, plug = 0.0, a0 = 0.0, a1 = 0.0;
    if (cls && i != 2 && (s0 || s1)) {
        if (s0 != s1) {
            const double e = s0 ? e0 : e1, K = s0 ? K0 : K1, p = s0 ? p0 : p1;
            plug = e;
            est = e;
            var = e / K * (1.0 / p - e);                  // Theorems 7, 9
            if (s0) a0 = 1.0; else a1 = 1.0;
        } else {
            const double e = ((double)h0 + (double)h1) / (K0 * p0 + K1 * p1);
            plug = e;
            const double V1 = fmax(e / K0 * (1.0 / p0 - e), 0.0);
            const double V2 = fmax(e / K1 * (1.0 / p1 - e), 0.0);
            if (V1 + V2 > 0.0) {
                a0 = V2 / (V1 + V2);
                a1 = V1 / (V1 + V2);
                var = V1 * V2 / (V1 + V2);                // Theorem 10
            } else {
                a0 = a1 = 0.5;
                var = 0.0;
            }
            est = a0 * e0 + a1 * e1;
        }
    }
    // eta_2 = Lambda_4 - sum_{Omega_3*} phi^(3)_i eta_i and its variance
    const bool om3 = cls && i != 2 && f3 > 0;
    const double s = warp_sum_d(om3 ? f3 * est : 0.0);
    double v2 = warp_sum_d(om3 ? f3 * f3 * var : 0.0);
    // sum_{i != j} phi_i phi_j Cov(i, j), Cov = -sum_l b_i b_j / K_l with
    // b_i = phi_i a^(l)_i plug_i: per l, (sum b)^2 - sum b^2
    const double b0 = om3 ? f3 * (a0 * plug) : 0.0, b1 = om3 ? f3 * (a1 * plug) : 0.0;
    const double sb0 = warp_sum_d(b0), sbb0 = warp_sum_d(b0 * b0);
    const double sb1 = warp_sum_d(b1), sbb1 = warp_sum_d(b1 * b1);
    if (av0) v2 -= (sb0 * sb0 - sbb0) / K0;
    if (av1) v2 -= (sb1 * sb1 - sbb1) / K1;
    if (i == 2) {
        est = u128_to_double(tot->lambda4) - s;
        var = v2;
    }
    const double t = warp_sum_d(cls ? est : 0.0);         // concentrations (Sec. 6.3)
    if (i < kSlots) {
        out->hits[0][i] = h0;
        out->hits[1][i] = h1;
        out->est[i] = est;
        out->var[i] = var;
        out->lambda[0][i] = a0;
        out->lambda[1][i] = a1;
        out->conc[i] = (cls && t != 0.0) ? est / t : 0.0;
    }
    if (i == 0) {
        out->k = 5;
        out->n_classes = 21;
        out->K[0] = in.K[0];
        out->K[1] = in.K[1];
        out->triangles = 0.0;
        out->triangles_var = 0.0;
    }
    if (cov) {
        // lane j fills column j; Cov(eta_i, eta_j) = -plug_i plug_j sum_l a_i a_j / K_l
        // off the diagonal, and row/column 2 from the linear identity
        const bool colj = cls && i != 2;
        const double c0 = a0 * plug, c1 = a1 * plug;
        double c2 = 0.0;
        for (int r = 0; r < kSlots; ++r) {
            const double c0r = __shfl_sync(0xffffffffu, c0, r), c1r = __shfl_sync(0xffffffffu, c1, r);
            const bool rowr = r >= 1 && r <= 21 && r != 2;
            double c = 0.0;
            if (rowr && colj) {
                if (r == i) {
                    c = var;
                } else {
                    if (av0) c -= c0r * c0 / K0;
                    if (av1) c -= c1r * c1 / K1;
                }
            }
            if (i < kSlots && r != 2) cov[r * kSlots + i] = c;
            if (rowr && kPhi5[r - 1][2] > 0) c2 -= kPhi5[r - 1][2] * c;
        }
        __syncwarp();
        if (colj) {
            cov[2 * kSlots + i] = c2;
            cov[i * kSlots + 2] = c2;
        } else if (i == 2) {
            cov[2 * kSlots + 2] = var;
        } else if (i < kSlots) {
            cov[2 * kSlots + i] = 0.0;
        }
    }
}

// k = 4, alone (MOSS-4) or mixed with MOSS-4Min, with one warp: lane i is
// class i (1..6); the eta_2 identity, its variance and the covariances are
// formed on every lane from the values of classes 4, 5, 6 gathered by
// shuffles, in the order the formulas are written; the concentrations' sum
// is a warp sum.
__device__ void finalize4_warp(const FinalizeIn &in, const uint64_t *hits0, const uint64_t *hits1,
                               const DevTotals *tot, moss_result *out, double *cov) {
    const int i = threadIdx.x & 31;
    const bool cls = i >= 1 && i <= 6, mix = in.mix != 0;
    const double G = u128_to_double(tot->gamma[0]), Gm = mix ? u128_to_double(tot->gamma[3]) : 0.0;
    const double K = (double)in.K[0], Km = (double)in.K[1];
    const bool av0 = in.K[0] > 0 && G > 0, av1 = mix && in.K[1] > 0 && Gm > 0;
    const uint64_t h0 = (i < kSlots && hits0) ? hits0[i] : 0, h1 = (i < kSlots && hits1) ? hits1[i] : 0;
    const bool s0 = av0 && cls && i != 2;
    double p = 0.0, e4 = 0.0;
    if (s0) {
        p = 2.0 * kPhi4[i - 1][0] / G;                    // Theorem 2
        e4 = (double)h0 / (K * p);
    }
    // MOSS-4Min: classes 3, 5, 6 from their (class, c) slots (Theorems 4, 5)
    const int first = i == 3 ? 0 : (i == 5 ? 4 : 10), nslot = i == 3 ? 4 : (i == 5 ? 6 : (i == 6 ? 12 : 0));
    const bool s1 = av1 && nslot > 0;
    double em = 0.0, h = 0.0;
    if (s1) {
        double sa = 0.0, sb = 0.0;
        for (int c = 1; c <= nslot; ++c) {
            const double m = (double)hits1[first + c - 1];
            sa += m / c;
            sb += m / (c * c);
        }
        em = Gm / (2.0 * Km) * sa;
        h = sa > 0 ? sb / sa : (i == 6 ? 1.0 / 3.0 : 1.0);
    }
    double est = 0.0, var = 0.0, plug = 0.0, a0 = 0.0, a1 = 0.0;
    if (s0 != s1) {
        if (s0) {
            plug = est = e4;
            var = e4 / K * (1.0 / p - e4);                 // Theorem 3
            a0 = 1.0;
        } else {
            plug = est = em;
            var = (em * Gm * h / 2.0 - em * em) / Km;      // Theorem 5, per-CIS probabilities
            a1 = 1.0;
        }
    } else if (s0) {
        const double e = (K * e4 + Km * em) / (K + Km);
        plug = e;
        const double V1 = fmax(e / K * (1.0 / p - e), 0.0);
        const double V2 = fmax((e * Gm * h / 2.0 - e * e) / Km, 0.0);
        if (V1 + V2 > 0.0) {
            a0 = V2 / (V1 + V2);
            a1 = V1 / (V1 + V2);
            var = V1 * V2 / (V1 + V2);                     // Theorem 1
        } else {
            a0 = a1 = 0.5;
            var = 0.0;
        }
        est = a0 * e4 + a1 * em;
    }
    // classes 4, 5, 6 on every lane: n_2 = Lambda_3 - n_4 - 2 n_5 - 4 n_6 (eq. 2)
    double E[7], Vv[7], P[7], B0[7], B1[7];
    for (int c = 4; c <= 6; ++c) {
        E[c] = __shfl_sync(0xffffffffu, est, c);
        Vv[c] = __shfl_sync(0xffffffffu, var, c);
        P[c] = __shfl_sync(0xffffffffu, p, c);
        B0[c] = __shfl_sync(0xffffffffu, a0 * plug, c);
        B1[c] = __shfl_sync(0xffffffffu, a1 * plug, c);
    }
    const double est2 = u128_to_double(tot->lambda3) - E[4] - 2.0 * E[5] - 4.0 * E[6];
    const double coef[7] = {0, 0, 0, 0, 1.0, 2.0, 4.0};
    double v2 = 0.0;
    if (!mix) {
        if (av0) {
            const double s = E[4] + 2.0 * E[5] + 4.0 * E[6];
            v2 = (E[4] / P[4] + 4.0 * E[5] / P[5] + 16.0 * E[6] / P[6] - s * s) / K;
        }
    } else if (av0 || av1) {
        for (int r = 4; r <= 6; ++r)
            for (int c = 4; c <= 6; ++c) {
                double cv = Vv[r];
                if (r != c) {
                    cv = 0.0;
                    if (av0) cv -= B0[r] * B0[c] / K;
                    if (av1) cv -= B1[r] * B1[c] / Km;
                }
                v2 += coef[r] * coef[c] * cv;
            }
    }
    if (i == 2) {
        est = est2;
        var = v2;
    }
    const double t = warp_sum_d(cls ? est : 0.0);          // concentrations (Sec. 6.3)
    if (i < kSlots) {
        out->hits[0][i] = h0;
        out->hits[1][i] = h1;
        out->est[i] = est;
        out->var[i] = var;
        out->lambda[0][i] = mix ? a0 : 0.0;
        out->lambda[1][i] = mix ? a1 : 0.0;
        out->conc[i] = (cls && t != 0.0) ? est / t : 0.0;
    }
    if (i == 0) {
        out->k = 4;
        out->n_classes = 6;
        out->K[0] = mix ? (av0 ? in.K[0] : 0) : in.K[0];
        out->K[1] = mix ? (av1 ? in.K[1] : 0) : in.K[1];
        out->triangles = av0 ? (double)h0 * G / (6.0 * K) : 0.0;
        out->triangles_var = av0 ? out->triangles / K * (G / 6.0 - out->triangles) : 0.0;
    }
    if (cov) {
        // lane j fills column j: Cov(n_i, n_j) = -sum_l b_i b_j / K_l off the
        // diagonal (b = a^(l) plug; -n_i n_j / K for MOSS-4 alone), row and
        // column 2 from the linear identity
        for (int r = 0; r < kSlots; ++r)
            if (i < kSlots) cov[r * kSlots + i] = 0.0;
        __syncwarp();
        const bool colj = cls && i != 2 && (mix || av0);
        const double b0 = mix ? a0 * plug : est, b1 = a1 * plug;
        double c2 = 0.0;
        for (int r = 1; r <= 6; ++r) {
            const double b0r = __shfl_sync(0xffffffffu, b0, r), b1r = __shfl_sync(0xffffffffu, b1, r);
            if (r == 2 || !colj) continue;
            double c = 0.0;
            if (r == i) {
                c = var;
            } else if (mix) {
                if (av0) c -= b0r * b0 / K;
                if (av1) c -= b1r * b1 / Km;
            } else {
                c = -b0r * b0 / K;
            }
            cov[r * kSlots + i] = c;
            if (r >= 4) {
                if (mix) c2 -= coef[r] * c;
                else c2 += coef[r] * c;
            }
        }
        __syncwarp();
        if (colj) {
            if (!mix) c2 = -c2;
            cov[2 * kSlots + i] = c2;
            cov[i * kSlots + 2] = c2;
        } else if (i == 2 && (mix || av0)) {
            cov[2 * kSlots + 2] = v2;
        }
    }
}

// called by a whole warp: a lane per class
__device__ void finalize_any(const FinalizeIn &in, const uint64_t *hits0, const uint64_t *hits1,
                             const DevTotals *tot, moss_result *out, double *cov = nullptr) {
    if (in.k == 5 && !in.mix) finalize5_warp(in, hits0, hits1, tot, out, cov);
    else finalize4_warp(in, hits0, hits1, tot, out, cov);
}

// one warp
__global__ void k_covariance(FinalizeIn in, const uint64_t *hits, const DevTotals *tot, moss_result *out,
                             double *cov) {
    finalize_any(in, hits, hits + kSlots, tot, out, cov);
}

// one warp
__global__ void k_finalize(FinalizeIn in, const uint64_t *hits, const DevTotals *tot, moss_result *out) {
    finalize_any(in, hits, hits + kSlots, tot, out);
}

// one warp per request of a batch
constexpr int kFinalizeWarps = 4;
__global__ void k_finalize_batch(const BatchRequest *reqs, int nreq, const uint64_t *task_counts,
                                 moss_result *out) {
    const int r = blockIdx.x * kFinalizeWarps + (threadIdx.x >> 5);
    if (r >= nreq) return;   // warp-uniform
    const BatchRequest q = reqs[r];
    const uint64_t *h0 = q.task[0] >= 0 ? task_counts + (uint64_t)q.task[0] * kSlots : nullptr;
    const uint64_t *h1 = q.task[1] >= 0 ? task_counts + (uint64_t)q.task[1] * kSlots : nullptr;
    finalize_any(q.in, h0, h1, q.tot, out + r);
}

}  // namespace

cudaError_t launch_finalize(const FinalizeIn &in, const uint64_t *hits_dev, const DevTotals *tot, void *result_dev,
                            cudaStream_t s) {
    k_finalize<<<1, 32, 0, s>>>(in, hits_dev, tot, static_cast<moss_result *>(result_dev));
    return cudaGetLastError();
}

cudaError_t launch_covariance(const FinalizeIn &in, const uint64_t *hits_dev, const DevTotals *tot, void *result_dev,
                              double *cov_dev, cudaStream_t s) {
    k_covariance<<<1, 32, 0, s>>>(in, hits_dev, tot, static_cast<moss_result *>(result_dev), cov_dev);
    return cudaGetLastError();
}

cudaError_t launch_finalize_batch(const BatchRequest *reqs, int nreq, const uint64_t *task_counts, void *results,
                                  cudaStream_t s) {
    if (nreq <= 0) return cudaSuccess;
    k_finalize_batch<<<(nreq + kFinalizeWarps - 1) / kFinalizeWarps, 32 * kFinalizeWarps, 0, s>>>(
        reqs, nreq, task_counts, static_cast<moss_result *>(results));
    return cudaGetLastError();
}

}  // namespace moss
