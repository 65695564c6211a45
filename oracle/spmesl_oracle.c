/*
 * FP64 CPU oracle for SPMESL (sparse precision matrix estimation via scaled
 * lasso) solved by cyclic coordinate descent.
 *
 * TEST INFRASTRUCTURE ONLY.  Only the test suite, the smoke check and the
 * CPU-baseline leg of the benchmark may build, load or call this file.  It
 * shares no code, header, table or helper with the CUDA library and never
 * includes anything from it.
 *
 * What it computes (paper section / equation / algorithm):
 *   oracle_gram      S = X'X/n (optionally of the column-centred X),
 *                    Section 2.2 (sample covariance; centring, Section 2.2).
 *   oracle_spmesl    Algorithm 2: for every column k, the scaled lasso of
 *                    Eq. (5) solved by Algorithm 1 (cyclic ascending CD with
 *                    warm start, sigma update of Eq. (14)), then
 *                    Omega_1 = -B D (Eq. (4)), the min-magnitude
 *                    symmetrisation of Eq. (9), and, when the fit ran on the
 *                    standardised covariance, the unscaling
 *                    Omega^o = C Omega^C C of Proposition 1.
 *
 * Everything is written on the covariance S rather than on X:
 *   (1/n) x_k' (x_j - X beta) = S_kj - sum_l S_kl beta_l,
 *   (1/n) ||x_j - X beta||^2  = S_jj - 2 beta'S_.j + beta'S beta,
 * which is the definition of S, nothing more.  The coordinate value
 * c = S_kj - sum_{l != k} S_kl beta_l is recomputed from S at every step;
 * no gradient is maintained, so this file does not share the GPU path's
 * formulation.
 *
 * Readings of points where the paper is silent:
 *   - delta (tol) is used for both stopping tests of Algorithm 1;
 *   - maxit caps the inner sweeps of one lasso subproblem and, separately,
 *     the outer sigma iterations; hitting either marks the column
 *     not-converged and the last iterate is kept;
 *   - sigma^2 is floored at 1e-12 * S_jj; a column that hits the floor is
 *     marked degenerate;
 *   - with standardize = 0 the update is beta_k = Soft(c, lambda)/S_kk with
 *     the unweighted penalty lambda0 * sigma_j.
 */
#include <math.h>
#include <stdlib.h>
#include <string.h>
#ifdef _OPENMP
#include <omp.h>
#endif

#define ORACLE_COL_OK 0
#define ORACLE_COL_NOT_CONVERGED 1
#define ORACLE_COL_DEGENERATE 2

/* S = (1/n) X'X, X row-major n x p.  With center != 0 the column means are
 * removed first (Section 2.2 centres the columns). */
void oracle_gram(const double* X, int n, int p, int center, double* S)
{
    double* mu = (double*)calloc((size_t)p, sizeof(double));
    if (center) {
        for (int i = 0; i < n; ++i)
            for (int k = 0; k < p; ++k) mu[k] += X[(size_t)i * p + k];
        for (int k = 0; k < p; ++k) mu[k] /= (double)n;
    }
#ifdef _OPENMP
#pragma omp parallel for schedule(dynamic, 16)
#endif
    for (int k = 0; k < p; ++k) {
        for (int l = k; l < p; ++l) {
            double acc = 0.0;
            for (int i = 0; i < n; ++i)
                acc += (X[(size_t)i * p + k] - mu[k]) * (X[(size_t)i * p + l] - mu[l]);
            acc /= (double)n;
            S[(size_t)k * p + l] = acc;
            S[(size_t)l * p + k] = acc;
        }
    }
    free(mu);
}

static double soft_threshold(double x, double lam)
{
    /* Soft_lambda(x) = sign(x) (|x| - lambda)_+  (Section 3.1) */
    if (x > lam) return x - lam;
    if (x < -lam) return x + lam;
    return 0.0;
}

/* sigma^2 = S_jj - 2 beta'S_.j + beta'S beta over the support of beta
 * (Eq. (14) written on S). */
static double residual_quadratic_form(const double* S, int p, int j, const double* beta,
                                      const int* supp, int nsupp)
{
    double lin = 0.0, quad = 0.0;
    for (int a = 0; a < nsupp; ++a) {
        int k = supp[a];
        lin += beta[k] * S[(size_t)k * p + j];
        double row = 0.0;
        for (int b = 0; b < nsupp; ++b) {
            int l = supp[b];
            row += S[(size_t)k * p + l] * beta[l];
        }
        quad += beta[k] * row;
    }
    return S[(size_t)j * p + j] - 2.0 * lin + quad;
}

/*
 * Algorithm 1 for response column j of S (the regression of x_j on the other
 * columns, beta_j fixed at 0).  beta is a length-p output (beta[j] = 0).
 * Returns a column status; *outer and *sweeps count the sigma iterations and
 * the total inner sweeps.
 */
int oracle_scaled_lasso_column(const double* S, int p, int j, double lambda0, double tol,
                               int maxit, double* beta, double* sigma_out, int* outer_out,
                               int* sweeps_out)
{
    int* supp = (int*)malloc(sizeof(int) * (size_t)p);
    int* where = (int*)malloc(sizeof(int) * (size_t)p);
    int nsupp = 0;
    for (int k = 0; k < p; ++k) { beta[k] = 0.0; where[k] = -1; }

    int status = ORACLE_COL_OK;
    double sigma = 1.0;               /* sigma^(0) = 1, beta^(0) = 0 */
    const double floor2 = 1e-12 * S[(size_t)j * p + j];
    int r = 0, total_sweeps = 0;
    for (r = 0; r < maxit; ++r) {
        const double lam = sigma * lambda0;
        int m, inner_done = 0;
        for (m = 0; m < maxit; ++m) {
            double maxd = 0.0;
            for (int k = 0; k < p; ++k) {
                if (k == j) continue;
                /* c = S_kj - sum_{l != k} S_kl beta_l  (beta_j = 0) */
                double c = S[(size_t)k * p + j];
                for (int a = 0; a < nsupp; ++a) {
                    int l = supp[a];
                    if (l != k) c -= S[(size_t)k * p + l] * beta[l];
                }
                double nb = soft_threshold(c, lam) / S[(size_t)k * p + k];
                double d = fabs(nb - beta[k]);
                if (d > maxd) maxd = d;
                /* maintain the support list of nonzero beta */
                if (nb != 0.0 && where[k] < 0) {
                    where[k] = nsupp; supp[nsupp++] = k;
                } else if (nb == 0.0 && where[k] >= 0) {
                    int pos = where[k], last = supp[--nsupp];
                    supp[pos] = last; where[last] = pos; where[k] = -1;
                }
                beta[k] = nb;
            }
            ++total_sweeps;
            if (maxd < tol) { inner_done = 1; break; }
        }
        if (!inner_done) status = ORACLE_COL_NOT_CONVERGED;
        double q = residual_quadratic_form(S, p, j, beta, supp, nsupp);
        if (q <= floor2) { q = floor2; if (status == ORACLE_COL_OK) status = ORACLE_COL_DEGENERATE; }
        double sigma_new = sqrt(q);
        double ds = fabs(sigma_new - sigma);
        sigma = sigma_new;
        if (ds < tol) break;
    }
    if (r == maxit) { r = maxit - 1; if (status == ORACLE_COL_OK) status = ORACLE_COL_NOT_CONVERGED; }
    *sigma_out = sigma;
    if (outer_out) *outer_out = r + 1;
    if (sweeps_out) *sweeps_out = total_sweeps;
    free(supp);
    free(where);
    return status;
}

/* Standardised covariance S^C = C S C, C = diag(S_jj^{-1/2}) (Section 2.2,
 * Proposition 1).  c_out receives the diagonal of C. */
void oracle_standardize(const double* S, int p, double* SC, double* c_out)
{
    for (int k = 0; k < p; ++k) c_out[k] = 1.0 / sqrt(S[(size_t)k * p + k]);
    for (int k = 0; k < p; ++k)
        for (int l = 0; l < p; ++l)
            SC[(size_t)k * p + l] = S[(size_t)k * p + l] * c_out[k] * c_out[l];
}

/*
 * Scaled lasso for a chosen subset of response columns, on the standardised
 * (standardize != 0) or raw covariance.  B_cols is ncols x p row-major: row t
 * holds the coefficient vector of regression cols[t], sigma_cols the matching
 * sigma.  With unscale != 0 both are returned in the ORIGINAL scale
 * (proof of Proposition 1: b^o_jk = sqrt(s_kk / s_jj) b^C_jk,
 * sigma^o = sqrt(s_kk) sigma^C); otherwise on the scale the fit ran on.
 */
int oracle_columns(const double* S, int p, const int* cols, int ncols, double lambda0,
                   double tol, int maxit, int standardize, int unscale, int nthreads,
                   double* B_cols, double* sigma_cols, int* col_outer, int* col_sweeps,
                   int* col_status)
{
    const double* W = S;
    double* SC = NULL;
    double* c = (double*)malloc(sizeof(double) * (size_t)p);
    if (!c) return -2;
    for (int k = 0; k < p; ++k) c[k] = 1.0;
    if (standardize) {
        SC = (double*)malloc(sizeof(double) * (size_t)p * (size_t)p);
        if (!SC) { free(c); return -2; }
        oracle_standardize(S, p, SC, c);
        W = SC;
    }
    int worst = 0;
#ifdef _OPENMP
    if (nthreads > 0) omp_set_num_threads(nthreads);
#pragma omp parallel for schedule(dynamic, 1) reduction(max : worst)
#endif
    for (int t = 0; t < ncols; ++t) {
        int k = cols[t];
        double* b = B_cols + (size_t)t * p;
        double sg = 0.0;
        int st = oracle_scaled_lasso_column(W, p, k, lambda0, tol, maxit, b, &sg,
                                            col_outer ? &col_outer[t] : NULL,
                                            col_sweeps ? &col_sweeps[t] : NULL);
        if (unscale) {
            for (int j = 0; j < p; ++j) b[j] = b[j] * c[j] / c[k];
            sg = sg / c[k];
        }
        sigma_cols[t] = sg;
        if (col_status) col_status[t] = st;
        if (st > worst) worst = st;
    }
    (void)nthreads;
    free(SC);
    free(c);
    return worst;
}

/*
 * Algorithm 2 end to end on covariance S (p x p row-major, FP64).
 * With standardize != 0 the p scaled lassos run on S^C = C S C, Omega is
 * assembled and symmetrised on that scale, and the result is mapped back by
 * Omega^o = C Omega^C C (Proposition 1).
 * Outputs (all caller-allocated):
 *   Theta  p x p, Theta[j*p+k] = omega_jk after symmetrisation, original scale
 *   sigma  p, error standard deviations in the original scale
 *   B      p x p or NULL; B[j*p+k] = b_jk = coefficient of x_j in regression k
 *          (original scale)
 * Returns the worst column status (0 ok, 1 not converged, 2 degenerate).
 */
int oracle_spmesl(const double* S, int p, double lambda0, double tol, int maxit,
                  int standardize, int nthreads, double* Theta, double* sigma, double* B,
                  int* col_outer, int* col_sweeps, int* col_status)
{
    int* cols = (int*)malloc(sizeof(int) * (size_t)p);
    double* Bc = (double*)malloc(sizeof(double) * (size_t)p * (size_t)p); /* row k = regression k */
    double* c = (double*)malloc(sizeof(double) * (size_t)p);
    if (!cols || !Bc || !c) { free(cols); free(Bc); free(c); return -2; }
    for (int k = 0; k < p; ++k) {
        cols[k] = k;
        c[k] = standardize ? 1.0 / sqrt(S[(size_t)k * p + k]) : 1.0;
    }
    /* the p scaled lassos on the working scale (S^C when standardising) */
    int worst = oracle_columns(S, p, cols, p, lambda0, tol, maxit, standardize, 0, nthreads,
                               Bc, sigma, col_outer, col_sweeps, col_status);
    if (worst < 0) { free(cols); free(Bc); free(c); return worst; }

    /* Omega_1: omega_kk = sigma_k^-2, omega_jk = -b_jk sigma_k^-2 (Eq. (4),
     * Algorithm 2).  Column k of Omega_1 comes from regression k. */
    for (int j = 0; j < p; ++j) {
        for (int k = 0; k < p; ++k) {
            double okk = 1.0 / (sigma[k] * sigma[k]);
            Theta[(size_t)j * p + k] = (j == k) ? okk : -Bc[(size_t)k * p + j] * okk;
        }
    }
    /* Symmetrisation, Eq. (9) as ordered in Algorithm 2: for j < k keep the
     * entry of smaller magnitude; on a tie omega_jk wins. */
    for (int j = 0; j < p - 1; ++j) {
        for (int k = j + 1; k < p; ++k) {
            double* ojk = &Theta[(size_t)j * p + k];
            double* okj = &Theta[(size_t)k * p + j];
            if (fabs(*ojk) > fabs(*okj)) *ojk = *okj;
            else *okj = *ojk;
        }
    }
    /* Omega^o = C Omega^C C (Proposition 1); C = I when not standardising */
    for (int j = 0; j < p; ++j)
        for (int k = 0; k < p; ++k) Theta[(size_t)j * p + k] *= c[j] * c[k];
    for (int k = 0; k < p; ++k) sigma[k] = sigma[k] / c[k];
    if (B) {
        for (int j = 0; j < p; ++j)
            for (int k = 0; k < p; ++k)
                B[(size_t)j * p + k] = Bc[(size_t)k * p + j] * c[j] / c[k];
    }
    free(cols);
    free(Bc);
    free(c);
    return worst;
}
