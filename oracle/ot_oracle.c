/*
 * FP64 CPU oracle for entropic-OT device association.
 *
 * TEST INFRASTRUCTURE ONLY.  Nothing in the product path may call, link or load
 * this file; only the test-suite, the package entry point's smoke check and the
 * benchmark's CPU-baseline leg use it.  It shares no code, header, table or
 * helper with the CUDA library: it is a plain, slow, loop-by-loop restatement
 * of the paper in double precision, written to be checked by eye.
 *
 * Paper: Paschos, Liakopoulos, Debbah, Wen, "Computational Optimal Transport
 * for 5G Massive C-RAN Device Association" (arXiv 1805.01559).
 *
 * Index convention: i = device (row, I of them), j = RRH (column, J of them).
 * Matrices are I x J, row-major.  The paper swaps m and n between Eq. (1) and
 * Eqs. (2)-(4); here the row marginal p is the device traffic and the column
 * marginal q belongs to the RRHs throughout.
 *
 * Parity status of each function (see the tests for the pins):
 *   oracle_rates      pinned (single-RRH closed form, symmetric two-RRH case,
 *                     low-SINR limit)
 *   oracle_rates_total pinned (equal to oracle_rates on random and dominant-link rows)
 *   oracle_cost       pinned (closed form)
 *   oracle_median     pinned (arange closed form, library select)
 *   oracle_sinkhorn   pinned (J = 1, separable cost, 2x2 closed form, scaling-
 *                     domain brute force, LP limit, Lemma 1 bounds, invariants)
 *   oracle_finalize   pinned (marginals of closed-form plans; residuals per unit
 *                     mass on a perturbed product plan of mass 3)
 *   oracle_maxsinr    pinned (brute-force argmax, Lemma 1)
 *   oracle_adaptive   pinned (one outer step by hand, mass conservation)
 *   oracle_completion pinned (hand-worked two-device cases, overload -> inf)
 *   oracle_euclid_cost pinned (3-4-5 triangles, symmetry)
 */
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>

#ifdef _OPENMP
#include <omp.h>
#endif

#define ORC_OK 0
#define ORC_EINVAL -1
#define ORC_ENOMEM -2

int oracle_num_threads(void) {
#ifdef _OPENMP
    return omp_get_max_threads();
#else
    return 1;
#endif
}

void oracle_set_threads(int n) {
#ifdef _OPENMP
    if (n > 0) omp_set_num_threads(n);
#else
    (void)n;
#endif
}

/*
 * Downlink exclusive-service rate, Sec. II-A:
 *   SINR_ji = P_j G_ji / (sum_{k != j} P_k G_ki + N_0),  R_ij = W log2(1 + SINR_ji).
 * G is I x J with G[i*J + j] the gain from RRH j to device i.  The log base is 2
 * (rate in bit/s for W in Hz).  The interference sum is formed directly over
 * k != j, which is O(I J^2) and slow on purpose: no "total minus own" shortcut.
 */
int oracle_rates(const double* G, const double* P, int64_t I, int64_t J, double N0, double W,
                 double* R_out) {
    if (I <= 0 || J <= 0 || !(N0 >= 0.0) || !(W > 0.0)) return ORC_EINVAL;
#pragma omp parallel for schedule(static)
    for (int64_t i = 0; i < I; ++i) {
        const double* g = G + i * J;
        for (int64_t j = 0; j < J; ++j) {
            double interference = N0;
            for (int64_t k = 0; k < J; ++k)
                if (k != j) interference += P[k] * g[k];
            double sinr = P[j] * g[j] / interference;
            R_out[i * J + j] = W * log1p(sinr) / log(2.0);
        }
    }
    return ORC_OK;
}

/*
 * The same rates with the interference formed as the row total minus the own term:
 *   I_ij = sum_k P_k G_ik - P_j G_ij + N_0,
 * O(I J) instead of O(I J^2), for instances too large for the direct sum.  The row total
 * is a compensated (Neumaier) sum, so T - P_j G_ij loses no more than the rounding of T
 * itself; both formulations agree to FP64 rounding wherever the own term does not carry
 * all but ~1e-10 of the row total.
 */
int oracle_rates_total(const double* G, const double* P, int64_t I, int64_t J, double N0, double W,
                       double* R_out) {
    if (I <= 0 || J <= 0 || !(N0 >= 0.0) || !(W > 0.0)) return ORC_EINVAL;
#pragma omp parallel for schedule(static)
    for (int64_t i = 0; i < I; ++i) {
        const double* g = G + i * J;
        double t = 0.0, c = 0.0;
        for (int64_t k = 0; k < J; ++k) {
            const double x = P[k] * g[k];
            const double u = t + x;
            c += fabs(t) >= fabs(x) ? (t - u) + x : (x - u) + t;
            t = u;
        }
        for (int64_t j = 0; j < J; ++j) {
            const double own = P[j] * g[j];
            const double interference = ((t - own) + c) + N0;
            R_out[i * J + j] = W * log1p(own / interference) / log(2.0);
        }
    }
    return ORC_OK;
}

/* OT cost per unit traffic, Sec. IV choice (ii): C_ij = 1 / (mu R_ij). */
int oracle_cost(const double* R, int64_t n, double mu, double* C_out) {
    if (n <= 0 || !(mu > 0.0)) return ORC_EINVAL;
    for (int64_t t = 0; t < n; ++t) {
        if (!(R[t] > 0.0)) return ORC_EINVAL;
        C_out[t] = 1.0 / (mu * R[t]);
    }
    return ORC_OK;
}

/* Hoare quickselect on a private copy: the k-th smallest (0-based). */
static double select_kth(double* a, int64_t n, int64_t k) {
    int64_t lo = 0, hi = n - 1;
    while (lo < hi) {
        double pivot = a[lo + (hi - lo) / 2];
        int64_t i = lo, j = hi;
        while (i <= j) {
            while (a[i] < pivot) ++i;
            while (a[j] > pivot) --j;
            if (i <= j) {
                double t = a[i]; a[i] = a[j]; a[j] = t;
                ++i; --j;
            }
        }
        if (k <= j) hi = j;
        else if (k >= i) lo = i;
        else return a[k];
    }
    return a[k];
}

/*
 * Median of n values: the middle order statistic, or the mean of the two middle
 * ones when n is even.  Used for eps = c * median(C); the paper only asks for a
 * regularization strength eps > 0 (Eq. 5), the median rule is the reading used
 * by the benchmark configurations.
 */
int oracle_median(const double* x, int64_t n, double* out) {
    if (n <= 0) return ORC_EINVAL;
    for (int64_t t = 0; t < n; ++t)
        if (x[t] != x[t]) return ORC_EINVAL; /* NaN has no rank */
    double* a = (double*)malloc((size_t)n * sizeof(double));
    if (!a) return ORC_ENOMEM;
    memcpy(a, x, (size_t)n * sizeof(double));
    double m;
    if (n % 2 == 1) {
        m = select_kth(a, n, n / 2);
    } else {
        double lo = select_kth(a, n, n / 2 - 1);
        /* after selection every element right of n/2-1 is >= lo: the next order statistic
           is the minimum of that right part */
        double hi = a[n / 2];
        for (int64_t t = n / 2; t < n; ++t)
            if (a[t] < hi) hi = a[t];
        m = 0.5 * (lo + hi);
    }
    free(a);
    *out = m;
    return ORC_OK;
}

/* log(sum_t exp(y_t)) with the maximum factored out. */
static double lse_row(const double* y, int64_t n) {
    double m = -INFINITY;
    for (int64_t t = 0; t < n; ++t)
        if (y[t] > m) m = y[t];
    if (m == -INFINITY) return -INFINITY;
    double s = 0.0;
    for (int64_t t = 0; t < n; ++t) s += exp(y[t] - m);
    return m + log(s);
}

/*
 * a-update of Algorithm 1 (the projection onto C_p), in log form.  With
 * a_i = exp(f_i / eps), b_j = exp(g_j / eps) and xi_ij = exp(-C_ij / eps):
 *   a_i = p_i / sum_j b_j xi_ij   <=>   f_i = eps log p_i - eps LSE_j((g_j - C_ij) / eps).
 */
static void row_update(const double* C, const double* p, const double* g, int64_t I, int64_t J,
                       double eps, double* f) {
#pragma omp parallel
    {
        double* y = (double*)malloc((size_t)J * sizeof(double));
#pragma omp for schedule(static)
        for (int64_t i = 0; i < I; ++i) {
            for (int64_t j = 0; j < J; ++j) y[j] = (g[j] - C[i * J + j]) / eps;
            f[i] = eps * log(p[i]) - eps * lse_row(y, J);
        }
        free(y);
    }
}

/*
 * b-update of Algorithm 1 (the projection onto C_q), in log form:
 *   b_j = q_j / sum_i a_i xi_ij   <=>   g_j = eps log q_j - eps LSE_i((f_i - C_ij) / eps).
 * Two plain passes over the rows: column maxima, then the shifted sums.
 */
static void col_update(const double* C, const double* q, const double* f, int64_t I, int64_t J,
                       double eps, double* g) {
#pragma omp parallel for schedule(static)
    for (int64_t j = 0; j < J; ++j) {
        double m = -INFINITY;
        for (int64_t i = 0; i < I; ++i) {
            double y = (f[i] - C[i * J + j]) / eps;
            if (y > m) m = y;
        }
        double s = 0.0;
        for (int64_t i = 0; i < I; ++i) s += exp((f[i] - C[i * J + j]) / eps - m);
        g[j] = eps * log(q[j]) - eps * (m + log(s));
    }
}

/* Transport plan of Algorithm 1's last step: pi_ij = a_i xi_ij b_j = exp((f_i + g_j - C_ij)/eps). */
static double plan_entry(const double* C, const double* f, const double* g, int64_t J, double eps,
                         int64_t i, int64_t j) {
    return exp((f[i] + g[j] - C[i * J + j]) / eps);
}

/* "Total absolute residual" of the row marginal (Sec. III-C):  sum_i | sum_j pi_ij - p_i |. */
static double row_residual(const double* C, const double* p, const double* f, const double* g,
                           int64_t I, int64_t J, double eps) {
    double* r = (double*)malloc((size_t)I * sizeof(double));
#pragma omp parallel for schedule(static)
    for (int64_t i = 0; i < I; ++i) {
        double s = 0.0;
        for (int64_t j = 0; j < J; ++j) s += plan_entry(C, f, g, J, eps, i, j);
        r[i] = fabs(s - p[i]);
    }
    double err = 0.0;
    for (int64_t i = 0; i < I; ++i) err += r[i];
    free(r);
    return err;
}

/*
 * Algorithm 1 (Sinkhorn), log domain, FP64.
 *
 * Inputs: cost C (I x J), marginals p (I) and q (J) with sum p == sum q up to
 * rounding, eps > 0, tolerance tol >= 0 and an iteration cap max_iter >= 1.
 * Start: b^(0) = 1, i.e. g = 0, unless g0 (J) is given (warm start).
 * The marginals are each divided by their own sum before iterating, so the
 * residual and tol refer to a plan of unit mass; the returned f is shifted by
 * eps * log(sum p) so that exp((f + g - C)/eps) carries the caller's mass.
 *
 * One iteration k = an a-update followed by a b-update.  The loop test
 * ("while accuracy") is made after every completed iteration on the plan
 * pi^(k) = exp((f^k + g^k - C)/eps): its columns are exact, so the residual is
 * that of the rows; stop when it is <= tol, or when k == max_iter.
 * Outputs: f (I), g (J), the iteration count and the final residual.
 */
int oracle_sinkhorn(const double* C, const double* p_in, const double* q_in, int64_t I, int64_t J,
                    double eps, double tol, int32_t max_iter, const double* g0, double* f,
                    double* g, int32_t* iters_out, double* err_out) {
    if (I <= 0 || J <= 0 || !(eps > 0.0) || !(tol >= 0.0) || max_iter < 1) return ORC_EINVAL;
    double sp = 0.0, sq = 0.0;
    for (int64_t i = 0; i < I; ++i) {
        if (!(p_in[i] > 0.0)) return ORC_EINVAL;
        sp += p_in[i];
    }
    for (int64_t j = 0; j < J; ++j) {
        if (!(q_in[j] > 0.0)) return ORC_EINVAL;
        sq += q_in[j];
    }
    double* p = (double*)malloc((size_t)I * sizeof(double));
    double* q = (double*)malloc((size_t)J * sizeof(double));
    if (!p || !q) { free(p); free(q); return ORC_ENOMEM; }
    for (int64_t i = 0; i < I; ++i) p[i] = p_in[i] / sp;
    for (int64_t j = 0; j < J; ++j) q[j] = q_in[j] / sq;

    for (int64_t j = 0; j < J; ++j) g[j] = g0 ? g0[j] : 0.0;
    int32_t k = 0;
    double err = INFINITY;
    for (;;) {
        ++k;
        row_update(C, p, g, I, J, eps, f);
        col_update(C, q, f, I, J, eps, g);
        err = row_residual(C, p, f, g, I, J, eps);
        if (err <= tol || k >= max_iter) break;
    }
    double shift = eps * log(sp);
    for (int64_t i = 0; i < I; ++i) f[i] += shift;
    *iters_out = k;
    *err_out = err;
    free(p);
    free(q);
    return ORC_OK;
}

/* Dense plan pi_ij = exp((f_i + g_j - C_ij)/eps) (Algorithm 1, last step). */
int oracle_plan(const double* C, const double* f, const double* g, int64_t I, int64_t J,
                double eps, double* pi_out) {
    if (I <= 0 || J <= 0 || !(eps > 0.0)) return ORC_EINVAL;
#pragma omp parallel for schedule(static)
    for (int64_t i = 0; i < I; ++i)
        for (int64_t j = 0; j < J; ++j) pi_out[i * J + j] = plan_entry(C, f, g, J, eps, i, j);
    return ORC_OK;
}

/*
 * Summary of a plan given by its potentials:
 *   transport cost  sum_ij C_ij pi_ij  (Eq. 2's objective),
 *   RRH load        rho_j = sum_i C_ij x_ij with the plan mass x = pi (Sec. II-B:
 *                   x_ij = lambda_i pi^assoc_ij, C_ij = 1/(mu R_ij)),
 *   L1 marginal errors  sum_i |sum_j pi_ij - p_i|  and  sum_j |sum_i pi_ij - q_j|.
 * Errors are reported relative to the total mass sum p (unit-mass plan).
 */
int oracle_finalize(const double* C, const double* f, const double* g, const double* p,
                    const double* q, int64_t I, int64_t J, double eps, double* cost_out,
                    double* rho_out, double* err_row_out, double* err_col_out) {
    if (I <= 0 || J <= 0 || !(eps > 0.0)) return ORC_EINVAL;
    double* rowsum = (double*)malloc((size_t)I * sizeof(double));
    double* rowcost = (double*)malloc((size_t)I * sizeof(double));
    double* colsum = (double*)malloc((size_t)J * sizeof(double));
    if (!rowsum || !rowcost || !colsum) {
        free(rowsum); free(rowcost); free(colsum);
        return ORC_ENOMEM;
    }
#pragma omp parallel for schedule(static)
    for (int64_t i = 0; i < I; ++i) {
        double s = 0.0, c = 0.0;
        for (int64_t j = 0; j < J; ++j) {
            double pij = plan_entry(C, f, g, J, eps, i, j);
            s += pij;
            c += C[i * J + j] * pij;
        }
        rowsum[i] = s;
        rowcost[i] = c;
    }
#pragma omp parallel for schedule(static)
    for (int64_t j = 0; j < J; ++j) {
        double s = 0.0, c = 0.0;
        for (int64_t i = 0; i < I; ++i) {
            double pij = plan_entry(C, f, g, J, eps, i, j);
            s += pij;
            c += C[i * J + j] * pij;
        }
        colsum[j] = s;
        rho_out[j] = c;
    }
    double mass = 0.0, cost = 0.0, er = 0.0, ec = 0.0;
    for (int64_t i = 0; i < I; ++i) {
        mass += p[i];
        cost += rowcost[i];
        er += fabs(rowsum[i] - p[i]);
    }
    for (int64_t j = 0; j < J; ++j) ec += fabs(colsum[j] - q[j]);
    *cost_out = cost;
    *err_row_out = er / mass;
    *err_col_out = ec / mass;
    free(rowsum);
    free(rowcost);
    free(colsum);
    return ORC_OK;
}

/*
 * maxSINR association (Sec. II-C; Lemma 1): each device picks the RRH with the
 * largest R_ij (lowest index on ties).  With every other RRH interfering and a
 * common noise floor this is also the strongest-signal rule.  Outputs the
 * choice per device, the RRH traffic Lambda_j = sum_{i: j*(i) = j} lambda_i and
 * the total load sum_i lambda_i C_{i j*(i)} (the quantity Lemma 1 says the OT
 * plan with q = Lambda reproduces).
 */
int oracle_maxsinr(const double* R, const double* C, const double* lam, int64_t I, int64_t J,
                   int32_t* assoc_out, double* Lambda_out, double* total_load_out) {
    if (I <= 0 || J <= 0) return ORC_EINVAL;
    for (int64_t j = 0; j < J; ++j) Lambda_out[j] = 0.0;
    double total = 0.0;
    for (int64_t i = 0; i < I; ++i) {
        int64_t best = 0;
        for (int64_t j = 1; j < J; ++j)
            if (R[i * J + j] > R[i * J + best]) best = j;
        assoc_out[i] = (int32_t)best;
        Lambda_out[best] += lam[i];
        total += lam[i] * C[i * J + best];
    }
    *total_load_out = total;
    return ORC_OK;
}

/*
 * Adaptive Sinkhorn association (Algorithm 2), outer loop.
 * Start from the equal split q_j = sum(lambda) / J (line 1).  Each outer step
 * solves Algorithm 1 with the current q (warm-started from the previous step's
 * g), evaluates the RRH loads rho_j of that plan (Sec. II-B), picks the most
 * loaded RRH j* (lowest index on ties) and moves delta of its target traffic to
 * the other J-1 RRHs in equal parts.  The paper states no stopping rule for the
 * outer loop: it runs `outer` steps and returns the plan of the last solve
 * together with the q that solve used (the update after it is not applied).
 * A q_j* that delta would drive to zero or below moves half of itself instead,
 * so every marginal stays positive.  Optional traces (NULL = not wanted): the
 * per-step maximum load (outer entries), the chosen RRH j* per step (outer
 * entries) and every step's loads rho (outer x J).
 */
int oracle_adaptive(const double* C, const double* lam, int64_t I, int64_t J, double eps,
                    double tol, int32_t max_iter, int32_t outer, double delta, double* f,
                    double* g, double* q_out, double* maxload_out, int32_t* jstar_out,
                    double* rho_out) {
    if (I <= 0 || J <= 1 || outer < 1 || !(delta >= 0.0)) return ORC_EINVAL;
    double total = 0.0;
    for (int64_t i = 0; i < I; ++i) total += lam[i];
    double* q = q_out;
    for (int64_t j = 0; j < J; ++j) q[j] = total / (double)J;
    double* rho = (double*)malloc((size_t)J * sizeof(double));
    double* gw = (double*)malloc((size_t)J * sizeof(double));
    if (!rho || !gw) { free(rho); free(gw); return ORC_ENOMEM; }
    int rc = ORC_OK;
    for (int32_t s = 0; s < outer; ++s) {
        int32_t it;
        double err, cost, er, ec;
        rc = oracle_sinkhorn(C, lam, q, I, J, eps, tol, max_iter, s ? gw : NULL, f, g, &it, &err);
        if (rc) break;
        memcpy(gw, g, (size_t)J * sizeof(double));
        rc = oracle_finalize(C, f, g, lam, q, I, J, eps, &cost, rho, &er, &ec);
        if (rc) break;
        int64_t js = 0;
        for (int64_t j = 1; j < J; ++j)
            if (rho[j] > rho[js]) js = j;
        if (maxload_out) maxload_out[s] = rho[js];
        if (jstar_out) jstar_out[s] = (int32_t)js;
        if (rho_out) memcpy(rho_out + (int64_t)s * J, rho, (size_t)J * sizeof(double));
        if (s == outer - 1) break;
        double d = delta < q[js] ? delta : 0.5 * q[js];
        for (int64_t j = 0; j < J; ++j)
            q[j] = (j == js) ? q[j] - d : q[j] + d / (double)(J - 1);
    }
    free(rho);
    free(gw);
    return rc;
}

/*
 * Average job completion time of an association, Sec. II-B.
 * x is a transport plan in mass units (I x J, x_ij = lambda_i pi_ij with pi_ij the
 * fraction of time device i uses RRH j), C the load cost C_ij = 1/(mu R_ij).
 *   rho_j = sum_i C_ij x_ij                   (RRH load, Sec. II-B with x = lambda pi)
 *   T_i   = sum_j pi_ij C_ij / (1 - rho_j)   (processor sharing: E[N_j] + 1 = 1/(1 - rho_j))
 *   T     = (1/I) sum_i T_i                   (the mean over devices of Eq. (1)'s terms)
 * An RRH with rho_j >= 1 that carries any of a device's traffic makes that device's time
 * infinite (the queue is unstable), and T is +inf.  rho_out (J) is optional.
 */
int oracle_completion(const double* C, const double* x, const double* lam, int64_t I, int64_t J,
                      double* T_out, double* rho_out) {
    if (I <= 0 || J <= 0) return ORC_EINVAL;
    double* rho = (double*)calloc((size_t)J, sizeof(double));
    if (!rho) return ORC_ENOMEM;
    for (int64_t i = 0; i < I; ++i)
        for (int64_t j = 0; j < J; ++j) rho[j] += C[i * J + j] * x[i * J + j];
    double T = 0.0;
    for (int64_t i = 0; i < I; ++i) {
        if (!(lam[i] > 0.0)) {
            free(rho);
            return ORC_EINVAL;
        }
        double Ti = 0.0;
        for (int64_t j = 0; j < J; ++j) {
            const double pij = x[i * J + j] / lam[i];
            if (pij == 0.0) continue;
            if (rho[j] >= 1.0) {
                Ti = INFINITY;
                break;
            }
            Ti += pij * C[i * J + j] / (1.0 - rho[j]);
        }
        T += Ti;
    }
    *T_out = T / (double)I;
    if (rho_out) memcpy(rho_out, rho, (size_t)J * sizeof(double));
    free(rho);
    return ORC_OK;
}

/*
 * Euclidean cost, Sec. IV choice (i): C_ij = || x_i - x_j || between device i at
 * dev_xy[2i], dev_xy[2i+1] and RRH j at rrh_xy[2j], rrh_xy[2j+1] (metres).
 */
int oracle_euclid_cost(const double* dev_xy, const double* rrh_xy, int64_t I, int64_t J, double* C_out) {
    if (I <= 0 || J <= 0) return ORC_EINVAL;
    for (int64_t i = 0; i < I; ++i)
        for (int64_t j = 0; j < J; ++j) {
            const double dx = dev_xy[2 * i] - rrh_xy[2 * j];
            const double dy = dev_xy[2 * i + 1] - rrh_xy[2 * j + 1];
            C_out[i * J + j] = sqrt(dx * dx + dy * dy);
        }
    return ORC_OK;
}
