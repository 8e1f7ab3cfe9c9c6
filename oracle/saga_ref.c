/*
 * Serial float64 Sparse SAGA -- the CPU checker for the ASAGA solver.
 *
 * TEST INFRASTRUCTURE ONLY.  This file is the slow, plain reference that the
 * CUDA path is compared against.  Only the tests, the smoke check and the
 * benchmark's CPU-baseline leg may load it; the solver library never does.
 * It shares no code, header or constant with the CUDA sources.
 *
 * What it computes (arXiv:1606.04809):
 *   - the Sparse SAGA update, Sec. 2 "Sparse SAGA Algorithm" (Eq. SparseSAGA):
 *       x+ = x - gamma (f'_i(x) - alpha_i + D_i abar),  D_i = P_{S_i} D,
 *     with D = diag(1/p_v) and p_v = |{i : v in S_i}| / n;
 *   - with the l2 term projected the same way, Sec. 4.2 "Exact
 *     regularization":  x+ = x - gamma (f'_i(x) - alpha_i + D_i abar + lambda D_i x);
 *   - for linear models f_i(x) = phi_i(a_i.x) the memory alpha_i is the scalar
 *     phi'_i at the last visit (App. G.2 "Efficient storage of the alpha_i"),
 *     so the vector gradient memory is alpha_i a_i and
 *     abar = (1/n) sum_i alpha_i a_i (Sec. 2, definition after Eq. SAGAupdate);
 *   - abar is kept up to date online (Algorithm 2): after the x update,
 *     abar_v += (phi'_i - alpha_i) a_iv / n on the support of row i, and the
 *     memory takes the new derivative, alpha_i <- phi'_i.
 * Within one iteration every coordinate of x and abar on S_i is read before
 * any of them is written (the right-hand side of Eq. SparseSAGA is evaluated
 * at the pre-update x and abar).
 *
 * Losses: logistic phi_i(z) = log(1 + exp(-b_i z)) with b_i in {-1,+1}
 * (Sec. 4.1 "Models"), and squared phi_i(z) = (z - y_i)^2 / 2.
 */
#include <math.h>
#include <stddef.h>
#include <stdint.h>

#define ORACLE_LOSS_LOGISTIC 0
#define ORACLE_LOSS_SQUARED 1

/* phi'_i(z).  Logistic: d/dz log(1+exp(-b z)) = -b / (1 + exp(b z)),
 * evaluated without overflow on either side of 0. */
static double phi_prime(int loss, double z, double b)
{
    if (loss == ORACLE_LOSS_LOGISTIC) {
        double t = b * z;
        if (t >= 0.0) {
            double e = exp(-t);
            return -b * e / (1.0 + e);
        }
        return -b / (1.0 + exp(t));
    }
    return z - b;
}

/*
 * Runs T serial Sparse SAGA iterations in place.  Iteration t visits row
 * idx[t] (the caller supplies the sampled indices; the paper samples them
 * uniformly with replacement).  Returns 0, or -1 on an out-of-range index.
 *
 * row_ptr[n+1], col_idx[nnz], val[nnz]: the CSR matrix (float64 values);
 * labels[n]; D[d]: the reweighting 1/p_v (0 for columns no row touches);
 * x[d], alpha[n], abar[d]: the shared state, updated in place.
 */
int oracle_sparse_saga(int64_t n, int64_t d, const int64_t *row_ptr, const int32_t *col_idx,
                       const double *val, const double *labels, int loss, double lambda,
                       double gamma, const double *D, double *x, double *alpha, double *abar,
                       const int64_t *idx, int64_t T)
{
    for (int64_t t = 0; t < T; ++t) {
        int64_t i = idx[t];
        if (i < 0 || i >= n)
            return -1;
        int64_t lo = row_ptr[i], hi = row_ptr[i + 1];
        double z = 0.0;
        for (int64_t k = lo; k < hi; ++k) {
            int32_t v = col_idx[k];
            if (v < 0 || v >= d)
                return -1;
            z += val[k] * x[v];
        }
        double g = phi_prime(loss, z, labels[i]);
        double delta = g - alpha[i];
        for (int64_t k = lo; k < hi; ++k) {
            int32_t v = col_idx[k];
            double a = val[k];
            double step = delta * a + D[v] * abar[v] + lambda * D[v] * x[v];
            x[v] -= gamma * step;
            abar[v] += delta * a / (double)n;
        }
        alpha[i] = g;
    }
    return 0;
}

/* phi'_i(a_i.x) for every row (used to recompute abar from scratch and to
 * evaluate gradients in float64). */
void oracle_row_derivatives(int64_t n, const int64_t *row_ptr, const int32_t *col_idx,
                            const double *val, const double *labels, int loss, const double *x,
                            double *out)
{
    for (int64_t i = 0; i < n; ++i) {
        double z = 0.0;
        for (int64_t k = row_ptr[i]; k < row_ptr[i + 1]; ++k)
            z += val[k] * x[col_idx[k]];
        out[i] = phi_prime(loss, z, labels[i]);
    }
}

/*
 * Serial SAGA with lagged updates (App. F.1 and F.2, the "just-in-time"
 * scheme of the SAG/SAGA literature that the paper compares Sparse SAGA with).
 * It computes the dense SAGA iteration (Eq. SAGAupdate with the l2 term's
 * gradient lambda x taken exactly):
 *     x+ = x - gamma (delta a_i + abar + lambda x),  delta = phi'_i - alpha_i,
 * but touches only S_i per step.  A coordinate v outside S_i receives
 * x_v <- (1 - gamma lambda) x_v - gamma abar_v, and abar_v cannot change
 * until v is in a sampled support again, so those steps are deferred and
 * applied in closed form when v is next read:
 *     m steps:  x_v <- c^m x_v - gamma abar_v (1 + c + ... + c^(m-1)),
 *     c = 1 - gamma lambda,  the sum = (1 - c^m) / (gamma lambda)  (m if lambda = 0).
 * last[v] is the number of steps already applied to x_v.  In exact
 * arithmetic the iterate equals dense SAGA's after oracle_lagged_catch_up.
 * Returns 0, or -1 on an out-of-range index.  Steps are numbered t0 .. t0+T-1.
 */
static double lagged_x(double xv, double abar_v, double gamma, double lambda, int64_t m)
{
    if (m <= 0)
        return xv;
    if (lambda == 0.0)
        return xv - gamma * abar_v * (double)m;
    double log_c = log1p(-gamma * lambda);
    double cm = exp((double)m * log_c);
    double one_minus_cm = -expm1((double)m * log_c);
    return cm * xv - abar_v * one_minus_cm / lambda;
}

int oracle_lagged_saga(int64_t n, int64_t d, const int64_t *row_ptr, const int32_t *col_idx,
                       const double *val, const double *labels, int loss, double lambda,
                       double gamma, double *x, double *alpha, double *abar, int64_t *last,
                       const int64_t *idx, int64_t T, int64_t t0)
{
    for (int64_t s = 0; s < T; ++s) {
        int64_t t = t0 + s;
        int64_t i = idx[s];
        if (i < 0 || i >= n)
            return -1;
        int64_t lo = row_ptr[i], hi = row_ptr[i + 1];
        double z = 0.0;
        for (int64_t k = lo; k < hi; ++k) {
            int32_t v = col_idx[k];
            if (v < 0 || v >= d)
                return -1;
            x[v] = lagged_x(x[v], abar[v], gamma, lambda, t - last[v]);
            last[v] = t;
            z += val[k] * x[v];
        }
        double g = phi_prime(loss, z, labels[i]);
        double delta = g - alpha[i];
        for (int64_t k = lo; k < hi; ++k) {
            int32_t v = col_idx[k];
            double a = val[k];
            x[v] -= gamma * (delta * a + abar[v] + lambda * x[v]);
            last[v] = t + 1;
            abar[v] += delta * a / (double)n;
        }
        alpha[i] = g;
    }
    return 0;
}

/* Applies every deferred step up to step t_end (the end of a run). */
void oracle_lagged_catch_up(int64_t d, double lambda, double gamma, double *x, const double *abar,
                            int64_t *last, int64_t t_end)
{
    for (int64_t v = 0; v < d; ++v) {
        x[v] = lagged_x(x[v], abar[v], gamma, lambda, t_end - last[v]);
        last[v] = t_end;
    }
}
