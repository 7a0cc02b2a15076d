/*
 * FP64 oracle for Fuzzy C-Means image segmentation — TEST INFRASTRUCTURE.
 *
 * Only the test suite, the smoke check and the benchmark's CPU-baseline leg
 * may load this file's library. The product (the CUDA library) never links,
 * calls or includes it, and this file includes nothing from the product.
 *
 * What it computes (paper: "GPU-Based Fuzzy C-Means Clustering Algorithm for
 * Image Segmentation", arXiv:1601.00072):
 *   - membership u_ij from centers, Eq. 4, written literally with
 *     d_ij = |x_i - v_j| (Sec. 2.1: Euclidean distance; the feature is the
 *     grey level, a scalar);
 *   - centers v_j from memberships, Eq. 3;
 *   - objective J_m, Eq. 1;
 *   - the loop of Algorithm 1: V from U, then U from V, until the change in
 *     U between iterations is below epsilon (Sec. 2.1, Algorithm 1 step 3).
 *
 * Readings where the paper is silent (each also listed in the design notes):
 *   - d = 0: Eq. 4 divides by zero when a pixel equals a center. Bezdek's rule
 *     is used: the clusters at zero distance share the membership equally,
 *     every other cluster gets 0. "Zero" means exactly equal in FP64.
 *   - The "overall difference" of the stopping test is the L-infinity norm
 *     max_{i,j} |u^k_ij - u^{k-1}_ij|, compared with a strict "<".
 *   - An empty cluster (sum_i u_ij^m == 0, only reachable through underflow)
 *     keeps its previous center and raises a flag.
 *   - Iteration k computes U^k from V^k, its change delta_k against U^{k-1},
 *     J_k = J(U^k, V^k); if delta_k < eps it stops and returns (U^k, V^k);
 *     otherwise V^{k+1} = centers(U^k). V^1 comes from the initial U^0
 *     (random, Algorithm 1 step 2) or, with a given V^0, from U^0 = f(x, V^0).
 *
 * Every sum runs sequentially in pixel order; nothing is blocked or fused.
 */
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>

#define ORACLE_INIT_U 0
#define ORACLE_INIT_V 1

#define ORACLE_CONVERGED 0
#define ORACLE_NOT_CONVERGED 1
#define ORACLE_BAD_ARG (-1)
#define ORACLE_NO_MEMORY (-3)

/* Eq. 4 for one pixel, with the zero-distance rule. u[j] for j < C. */
static void membership_of_pixel(double xi, int C, double m, const double* V,
                                double* u) {
    int nzero = 0;
    for (int j = 0; j < C; ++j)
        if (xi == V[j]) ++nzero;
    if (nzero > 0) {
        for (int j = 0; j < C; ++j) u[j] = (xi == V[j]) ? 1.0 / nzero : 0.0;
        return;
    }
    const double e = 2.0 / (m - 1.0);
    for (int j = 0; j < C; ++j) {
        const double dij = fabs(xi - V[j]);
        double s = 0.0;
        for (int k = 0; k < C; ++k) {
            const double dik = fabs(xi - V[k]);
            s += pow(dij / dik, e);
        }
        u[j] = 1.0 / s;
    }
}

/* Eq. 4 over all pixels. U is cluster-major: U[j*n + i]. */
void oracle_memberships(const double* x, int64_t n, int C, double m,
                        const double* V, double* U) {
    double u[64];
    for (int64_t i = 0; i < n; ++i) {
        membership_of_pixel(x[i], C, m, V, u);
        for (int j = 0; j < C; ++j) U[(int64_t)j * n + i] = u[j];
    }
}

/* Eq. 3: v_j = sum_i u_ij^m x_i / sum_i u_ij^m. Writes the numerators and
 * denominators too (nullable). A cluster with a zero denominator keeps
 * Vprev[j]; the return value counts such clusters. */
int oracle_centers(const double* x, int64_t n, int C, double m,
                   const double* U, const double* Vprev, double* V,
                   double* num_out, double* den_out) {
    int empty = 0;
    for (int j = 0; j < C; ++j) {
        double num = 0.0, den = 0.0;
        const double* Uj = U + (int64_t)j * n;
        for (int64_t i = 0; i < n; ++i) {
            const double w = pow(Uj[i], m);
            num += w * x[i];
            den += w;
        }
        if (num_out) num_out[j] = num;
        if (den_out) den_out[j] = den;
        if (den > 0.0) {
            V[j] = num / den;
        } else {
            V[j] = Vprev ? Vprev[j] : 0.0;
            ++empty;
        }
    }
    return empty;
}

/* Eq. 1: J_m = sum_i sum_j u_ij^m ||x_i - v_j||^2. */
double oracle_objective(const double* x, int64_t n, int C, double m,
                        const double* U, const double* V) {
    double J = 0.0;
    for (int64_t i = 0; i < n; ++i)
        for (int j = 0; j < C; ++j) {
            const double d = x[i] - V[j];
            J += pow(U[(int64_t)j * n + i], m) * d * d;
        }
    return J;
}

double oracle_max_abs_diff(const double* a, const double* b, int64_t len) {
    double mx = 0.0;
    for (int64_t t = 0; t < len; ++t) {
        const double d = fabs(a[t] - b[t]);
        if (d > mx || d != d) mx = d;
    }
    return mx;
}

/* Defuzzification (Sec. 2.1): label = argmax_j u_ij, ties to the lowest j. */
void oracle_labels(const double* U, int64_t n, int C, int32_t* labels) {
    for (int64_t i = 0; i < n; ++i) {
        int best = 0;
        double bu = U[i];
        for (int j = 1; j < C; ++j) {
            const double u = U[(int64_t)j * n + i];
            if (u > bu) { bu = u; best = j; }
        }
        labels[i] = best;
    }
}

static int check_args(int64_t n, int C, double m, double eps, int max_iter) {
    if (n < 1 || C < 1 || C > 64 || !(m > 1.0) || !(eps >= 0.0) || max_iter < 1)
        return ORACLE_BAD_ARG;
    return 0;
}

/*
 * Algorithm 1 on every pixel. init_mode ORACLE_INIT_U: init = U^0 [C*n];
 * ORACLE_INIT_V: init = V^0 [C]. Outputs U^k [C*n] (nullable), V^k [C],
 * iters = k. Traces (nullable, length max_iter and max_iter*C) receive
 * delta_k, J_k and V^k. *empty_out (nullable) counts empty-cluster events.
 * Returns ORACLE_CONVERGED, ORACLE_NOT_CONVERGED or a negative error.
 */
int oracle_fcm(const double* x, int64_t n, int C, double m, double eps,
               int max_iter, int init_mode, const double* init,
               double* U_out, double* V_out, int* iters,
               double* trace_delta, double* trace_J, double* trace_V,
               int* empty_out) {
    if (check_args(n, C, m, eps, max_iter)) return ORACLE_BAD_ARG;
    if (!x || !init || !V_out || !iters) return ORACLE_BAD_ARG;
    const int64_t cn = (int64_t)C * n;
    double* Uprev = (double*)malloc(sizeof(double) * cn);
    double* Ucur = (double*)malloc(sizeof(double) * cn);
    if (!Uprev || !Ucur) { free(Uprev); free(Ucur); return ORACLE_NO_MEMORY; }
    double V[64], Vnext[64];
    int empty = 0;

    if (init_mode == ORACLE_INIT_U) {
        memcpy(Uprev, init, sizeof(double) * cn);
    } else if (init_mode == ORACLE_INIT_V) {
        oracle_memberships(x, n, C, m, init, Uprev);
    } else {
        free(Uprev); free(Ucur);
        return ORACLE_BAD_ARG;
    }
    {   /* V^1 from U^0 (Eq. 3); a cluster that is empty keeps 0 or V^0 */
        double zero[64] = {0};
        empty += oracle_centers(x, n, C, m, Uprev,
                                init_mode == ORACLE_INIT_V ? init : zero, V,
                                NULL, NULL);
    }
    int status = ORACLE_NOT_CONVERGED;
    int k;
    for (k = 1; k <= max_iter; ++k) {
        oracle_memberships(x, n, C, m, V, Ucur);                 /* Eq. 4 */
        const double delta = oracle_max_abs_diff(Ucur, Uprev, cn);
        if (trace_delta) trace_delta[k - 1] = delta;
        if (trace_J) trace_J[k - 1] = oracle_objective(x, n, C, m, Ucur, V);
        if (trace_V) memcpy(trace_V + (int64_t)(k - 1) * C, V, sizeof(double) * C);
        if (delta < eps) { status = ORACLE_CONVERGED; break; }
        if (k == max_iter) break;
        empty += oracle_centers(x, n, C, m, Ucur, V, Vnext, NULL, NULL);  /* Eq. 3 */
        memcpy(V, Vnext, sizeof(double) * C);
        double* t = Uprev; Uprev = Ucur; Ucur = t;
    }
    if (k > max_iter) k = max_iter;
    *iters = k;
    memcpy(V_out, V, sizeof(double) * C);
    if (U_out) memcpy(U_out, Ucur, sizeof(double) * cn);
    if (empty_out) *empty_out = empty;
    free(Uprev); free(Ucur);
    return status;
}

/*
 * The same loop for integer grey levels 0..255 (uint8 data), run on the
 * 256-bin histogram: the brFCM reduction the paper cites (Sec. 3). From
 * iteration 1 on, u_ij depends on pixel i only through x_i, so every sum over
 * pixels equals the sum over grey levels b weighted by the count h_b. Only two
 * steps touch individual pixels: V^1 from a per-pixel U^0 (Eq. 3), and
 * delta_1 = max_i max_j |u^1_ij - u^0_ij|. Everything else runs on bins, and
 * the change delta_k for k >= 2 is the maximum over the occupied bins.
 * Arguments and outputs as for oracle_fcm; U_out (nullable) is per pixel.
 */
int oracle_fcm_quantized(const uint8_t* xq, int64_t n, int C, double m,
                         double eps, int max_iter, int init_mode,
                         const double* init, double* U_out, double* V_out,
                         int* iters, double* trace_delta, double* trace_J,
                         double* trace_V, int* empty_out) {
    if (check_args(n, C, m, eps, max_iter)) return ORACLE_BAD_ARG;
    if (!xq || !init || !V_out || !iters) return ORACLE_BAD_ARG;
    double h[256] = {0}, val[256];
    for (int b = 0; b < 256; ++b) val[b] = (double)b;
    for (int64_t i = 0; i < n; ++i) h[xq[i]] += 1.0;

    double Ub_prev[256 * 64], Ub[256 * 64]; /* bin-major here: [b*C + j] */
    double V[64], Vnext[64];
    int empty = 0;
    int first_per_pixel = (init_mode == ORACLE_INIT_U);

    if (init_mode == ORACLE_INIT_U) {
        /* V^1 from the per-pixel U^0 (Eq. 3) */
        for (int j = 0; j < C; ++j) {
            double num = 0.0, den = 0.0;
            const double* Uj = init + (int64_t)j * n;
            for (int64_t i = 0; i < n; ++i) {
                const double w = pow(Uj[i], m);
                num += w * (double)xq[i];
                den += w;
            }
            if (den > 0.0) V[j] = num / den; else { V[j] = 0.0; ++empty; }
        }
    } else if (init_mode == ORACLE_INIT_V) {
        for (int b = 0; b < 256; ++b) membership_of_pixel(val[b], C, m, init, Ub_prev + b * C);
        for (int j = 0; j < C; ++j) {
            double num = 0.0, den = 0.0;
            for (int b = 0; b < 256; ++b) {
                if (h[b] == 0.0) continue;
                const double w = pow(Ub_prev[b * C + j], m);
                num += h[b] * w * val[b];
                den += h[b] * w;
            }
            if (den > 0.0) V[j] = num / den; else { V[j] = init[j]; ++empty; }
        }
    } else {
        return ORACLE_BAD_ARG;
    }

    int status = ORACLE_NOT_CONVERGED;
    int k;
    for (k = 1; k <= max_iter; ++k) {
        for (int b = 0; b < 256; ++b) membership_of_pixel(val[b], C, m, V, Ub + b * C);
        double delta = 0.0;
        if (k == 1 && first_per_pixel) {
            for (int64_t i = 0; i < n; ++i)
                for (int j = 0; j < C; ++j) {
                    const double d = fabs(Ub[xq[i] * C + j] - init[(int64_t)j * n + i]);
                    if (d > delta || d != d) delta = d;
                }
        } else {
            for (int b = 0; b < 256; ++b) {
                if (h[b] == 0.0) continue;
                for (int j = 0; j < C; ++j) {
                    const double d = fabs(Ub[b * C + j] - Ub_prev[b * C + j]);
                    if (d > delta || d != d) delta = d;
                }
            }
        }
        double J = 0.0;
        for (int b = 0; b < 256; ++b) {
            if (h[b] == 0.0) continue;
            for (int j = 0; j < C; ++j) {
                const double d = val[b] - V[j];
                J += h[b] * pow(Ub[b * C + j], m) * d * d;
            }
        }
        if (trace_delta) trace_delta[k - 1] = delta;
        if (trace_J) trace_J[k - 1] = J;
        if (trace_V) memcpy(trace_V + (int64_t)(k - 1) * C, V, sizeof(double) * C);
        if (delta < eps) { status = ORACLE_CONVERGED; break; }
        if (k == max_iter) break;
        for (int j = 0; j < C; ++j) {
            double num = 0.0, den = 0.0;
            for (int b = 0; b < 256; ++b) {
                if (h[b] == 0.0) continue;
                const double w = pow(Ub[b * C + j], m);
                num += h[b] * w * val[b];
                den += h[b] * w;
            }
            if (den > 0.0) Vnext[j] = num / den; else { Vnext[j] = V[j]; ++empty; }
        }
        memcpy(V, Vnext, sizeof(double) * C);
        memcpy(Ub_prev, Ub, sizeof(double) * 256 * C);
    }
    if (k > max_iter) k = max_iter;
    *iters = k;
    memcpy(V_out, V, sizeof(double) * C);
    if (U_out)
        for (int64_t i = 0; i < n; ++i)
            for (int j = 0; j < C; ++j) U_out[(int64_t)j * n + i] = Ub[xq[i] * C + j];
    if (empty_out) *empty_out = empty;
    return status;
}

/* Dice similarity coefficient of a segmentation against ground truth, per
 * class (Sec. 5.2, Eq. 5: DSC = 2 |PR n GT| / (|PR| + |GT|)). The segmented
 * class of pixel i is class_of_label[labels[i]]; truth[i] is its true class.
 * counts (3 * n_classes, nullable) receives |PR_c|, |GT_c|, |PR_c n GT_c|.
 * A class absent from both gets DSC 1 (the two agree that it is empty). */
int oracle_dsc(const int32_t* labels, const uint8_t* truth, int64_t n, const int32_t* class_of_label,
               int n_labels, int n_classes, int64_t* counts, double* dsc) {
    if (!labels || !truth || !class_of_label || !dsc || n < 1 || n_labels < 1 || n_classes < 1)
        return ORACLE_BAD_ARG;
    int64_t pr[256] = {0}, gt[256] = {0}, both[256] = {0};
    if (n_classes > 256) return ORACLE_BAD_ARG;
    for (int64_t i = 0; i < n; ++i) {
        if (labels[i] < 0 || labels[i] >= n_labels || truth[i] >= n_classes) return ORACLE_BAD_ARG;
        const int p = class_of_label[labels[i]], g = truth[i];
        if (p < 0 || p >= n_classes) return ORACLE_BAD_ARG;
        pr[p] += 1;
        gt[g] += 1;
        if (p == g) both[p] += 1;
    }
    for (int c = 0; c < n_classes; ++c) {
        dsc[c] = (pr[c] + gt[c]) == 0 ? 1.0 : 2.0 * (double)both[c] / (double)(pr[c] + gt[c]);
        if (counts) {
            counts[3 * c] = pr[c];
            counts[3 * c + 1] = gt[c];
            counts[3 * c + 2] = both[c];
        }
    }
    return 0;
}

/*
 * Multi-feature FCM: each pixel is a vector x_i of D channels (Sec. 2.1
 * defines d_ij as a norm of x_i - v_j; here the Euclidean norm), each center
 * a vector v_j. Eq. 4 with d_ij = ||x_i - v_j||, Eq. 3 per channel, Eq. 1 with
 * ||x_i - v_j||^2, and the loop and readings of oracle_fcm. x is channel-major
 * (x[d*n + i]); V and V^0 are cluster-major (V[j*D + d]); U is [C][n].
 */
static void membership_of_vector(const double* x, int64_t n, int64_t i, int D, int C, double m,
                                 const double* V, double* u) {
    double dist[64];
    int nzero = 0;
    for (int j = 0; j < C; ++j) {
        double s = 0.0;
        for (int d = 0; d < D; ++d) {
            const double t = x[(int64_t)d * n + i] - V[j * D + d];
            s += t * t;
        }
        dist[j] = sqrt(s);
        if (dist[j] == 0.0) ++nzero;
    }
    if (nzero > 0) {
        for (int j = 0; j < C; ++j) u[j] = dist[j] == 0.0 ? 1.0 / nzero : 0.0;
        return;
    }
    const double e = 2.0 / (m - 1.0);
    for (int j = 0; j < C; ++j) {
        double s = 0.0;
        for (int k = 0; k < C; ++k) s += pow(dist[j] / dist[k], e);
        u[j] = 1.0 / s;
    }
}

void oracle_memberships_multi(const double* x, int64_t n, int D, int C, double m, const double* V,
                              double* U) {
    double u[64];
    for (int64_t i = 0; i < n; ++i) {
        membership_of_vector(x, n, i, D, C, m, V, u);
        for (int j = 0; j < C; ++j) U[(int64_t)j * n + i] = u[j];
    }
}

/* Eq. 3 per channel; an empty cluster keeps Vprev (or 0). Returns the count
 * of empty clusters. */
static int centers_multi(const double* x, int64_t n, int D, int C, double m, const double* U,
                         const double* Vprev, double* V) {
    int empty = 0;
    for (int j = 0; j < C; ++j) {
        double den = 0.0, num[16] = {0};
        const double* Uj = U + (int64_t)j * n;
        for (int64_t i = 0; i < n; ++i) {
            const double w = pow(Uj[i], m);
            den += w;
            for (int d = 0; d < D; ++d) num[d] += w * x[(int64_t)d * n + i];
        }
        for (int d = 0; d < D; ++d) {
            if (den > 0.0) V[j * D + d] = num[d] / den;
            else V[j * D + d] = Vprev ? Vprev[j * D + d] : 0.0;
        }
        if (!(den > 0.0)) ++empty;
    }
    return empty;
}

double oracle_objective_multi(const double* x, int64_t n, int D, int C, double m, const double* U,
                              const double* V) {
    double J = 0.0;
    for (int64_t i = 0; i < n; ++i)
        for (int j = 0; j < C; ++j) {
            double s = 0.0;
            for (int d = 0; d < D; ++d) {
                const double t = x[(int64_t)d * n + i] - V[j * D + d];
                s += t * t;
            }
            J += pow(U[(int64_t)j * n + i], m) * s;
        }
    return J;
}

int oracle_fcm_multi(const double* x, int64_t n, int D, int C, double m, double eps, int max_iter,
                     int init_mode, const double* init, double* U_out, double* V_out, int* iters,
                     double* trace_delta, double* trace_J, int* empty_out) {
    if (check_args(n, C, m, eps, max_iter) || D < 1 || D > 16) return ORACLE_BAD_ARG;
    if (!x || !init || !V_out || !iters) return ORACLE_BAD_ARG;
    const int64_t cn = (int64_t)C * n;
    double* Uprev = (double*)malloc(sizeof(double) * cn);
    double* Ucur = (double*)malloc(sizeof(double) * cn);
    if (!Uprev || !Ucur) { free(Uprev); free(Ucur); return ORACLE_NO_MEMORY; }
    double V[64 * 16], Vnext[64 * 16];
    int empty = 0;
    if (init_mode == ORACLE_INIT_U) {
        memcpy(Uprev, init, sizeof(double) * cn);
    } else if (init_mode == ORACLE_INIT_V) {
        oracle_memberships_multi(x, n, D, C, m, init, Uprev);
    } else {
        free(Uprev); free(Ucur);
        return ORACLE_BAD_ARG;
    }
    {
        double zero[64 * 16] = {0};
        empty += centers_multi(x, n, D, C, m, Uprev, init_mode == ORACLE_INIT_V ? init : zero, V);
    }
    int status = ORACLE_NOT_CONVERGED;
    int k;
    for (k = 1; k <= max_iter; ++k) {
        oracle_memberships_multi(x, n, D, C, m, V, Ucur);
        const double delta = oracle_max_abs_diff(Ucur, Uprev, cn);
        if (trace_delta) trace_delta[k - 1] = delta;
        if (trace_J) trace_J[k - 1] = oracle_objective_multi(x, n, D, C, m, Ucur, V);
        if (delta < eps) { status = ORACLE_CONVERGED; break; }
        if (k == max_iter) break;
        empty += centers_multi(x, n, D, C, m, Ucur, V, Vnext);
        memcpy(V, Vnext, sizeof(double) * C * D);
        double* t = Uprev; Uprev = Ucur; Ucur = t;
    }
    if (k > max_iter) k = max_iter;
    *iters = k;
    memcpy(V_out, V, sizeof(double) * C * D);
    if (U_out) memcpy(U_out, Ucur, sizeof(double) * cn);
    if (empty_out) *empty_out = empty;
    free(Uprev); free(Ucur);
    return status;
}
