/*
 * Oracle: sparse linear algebra for the CLS system (Sec. III.B): scalar
 * ILU(0) on CSR and restarted GMRES with right preconditioning and modified
 * Gram-Schmidt (Saad & Schultz 1986; Saad, "Iterative Methods for Sparse
 * Linear Systems", 2003, Alg. 6.10 and Sec. 10.3.2).  Also a dense LU with
 * partial pivoting used to pin GMRES on tiny meshes.
 * TEST INFRASTRUCTURE ONLY (see or_internal.h).
 */
#include <math.h>
#include <stdlib.h>
#include <string.h>

#include "or_internal.h"

void or_csr_free(or_csr *a)
{
    free(a->rowptr); free(a->col); free(a->val);
    a->rowptr = NULL; a->col = NULL; a->val = NULL; a->n = a->nnz = 0;
}

void or_csr_matvec(const or_csr *a, const double *x, double *y)
{
    for (int r = 0; r < a->n; ++r) {
        double s = 0.0;
        for (int e = a->rowptr[r]; e < a->rowptr[r + 1]; ++e) s += a->val[e] * x[a->col[e]];
        y[r] = s;
    }
}

/* ILU(0): same sparsity as A (columns sorted); L unit lower, U upper, stored
 * in one CSR. */
int or_ilu0(const or_csr *a, or_csr *lu, int **diag_pos)
{
    const int n = a->n;
    lu->n = n; lu->nnz = a->nnz;
    lu->rowptr = malloc(sizeof(int) * (size_t)(n + 1));
    lu->col = malloc(sizeof(int) * (size_t)a->nnz);
    lu->val = malloc(sizeof(double) * (size_t)a->nnz);
    int *dp = malloc(sizeof(int) * (size_t)n);
    int *pos = malloc(sizeof(int) * (size_t)n);
    if (!lu->rowptr || !lu->col || !lu->val || !dp || !pos) return -1;
    memcpy(lu->rowptr, a->rowptr, sizeof(int) * (size_t)(n + 1));
    memcpy(lu->col, a->col, sizeof(int) * (size_t)a->nnz);
    memcpy(lu->val, a->val, sizeof(double) * (size_t)a->nnz);
    for (int i = 0; i < n; ++i) pos[i] = -1;
    for (int i = 0; i < n; ++i) {
        dp[i] = -1;
        for (int e = lu->rowptr[i]; e < lu->rowptr[i + 1]; ++e) {
            pos[lu->col[e]] = e;
            if (lu->col[e] == i) dp[i] = e;
        }
        if (dp[i] < 0) return -2;
        for (int e = lu->rowptr[i]; e < lu->rowptr[i + 1]; ++e) {
            int k = lu->col[e];
            if (k >= i) break;
            double piv = lu->val[dp[k]];
            if (piv == 0.0) return -3;
            lu->val[e] /= piv;
            double lik = lu->val[e];
            for (int g = dp[k] + 1; g < lu->rowptr[k + 1]; ++g) {
                int j = lu->col[g];
                if (pos[j] >= 0) lu->val[pos[j]] -= lik * lu->val[g];
            }
        }
        for (int e = lu->rowptr[i]; e < lu->rowptr[i + 1]; ++e) pos[lu->col[e]] = -1;
        if (lu->val[dp[i]] == 0.0) return -3;
    }
    free(pos);
    *diag_pos = dp;
    return 0;
}

/* z = (LU)^{-1} r by forward then backward substitution. */
void or_ilu0_apply(const or_csr *lu, const int *dp, const double *r, double *z)
{
    const int n = lu->n;
    for (int i = 0; i < n; ++i) {
        double s = r[i];
        for (int e = lu->rowptr[i]; e < dp[i]; ++e) s -= lu->val[e] * z[lu->col[e]];
        z[i] = s;
    }
    for (int i = n - 1; i >= 0; --i) {
        double s = z[i];
        for (int e = dp[i] + 1; e < lu->rowptr[i + 1]; ++e) s -= lu->val[e] * z[lu->col[e]];
        z[i] = s / lu->val[dp[i]];
    }
}

static double nrm2(int n, const double *x)
{
    double s = 0.0;
    for (int i = 0; i < n; ++i) s += x[i] * x[i];
    return sqrt(s);
}

/* Restarted GMRES(m), right-preconditioned by the ILU(0) factors: solves
 * A x = b from the initial guess in x until ||b - A x||_2 <= rtol ||b||_2, the
 * iteration cap, or stagnation of the true residual over a whole cycle.
 * Returns 0 if converged, 1 otherwise. */
int or_gmres(const or_csr *a, const or_csr *lu, const int *dp, const double *b,
             double *x, int m, int maxit, double rtol, int *iters, double *relres)
{
    const int n = a->n;
    double bnorm = nrm2(n, b);
    *iters = 0;
    if (bnorm == 0.0) {
        for (int i = 0; i < n; ++i) x[i] = 0.0;
        *relres = 0.0;
        return 0;
    }
    double *V = malloc(sizeof(double) * (size_t)n * (size_t)(m + 1));
    double *H = calloc((size_t)(m + 1) * (size_t)m, sizeof(double));
    double *cs = malloc(sizeof(double) * (size_t)m), *sn = malloc(sizeof(double) * (size_t)m);
    double *g = malloc(sizeof(double) * (size_t)(m + 1)), *y = malloc(sizeof(double) * (size_t)m);
    double *w = malloc(sizeof(double) * (size_t)n), *z = malloc(sizeof(double) * (size_t)n);
    double *r = malloc(sizeof(double) * (size_t)n);
    int status = 1;
    or_csr_matvec(a, x, r);
    for (int i = 0; i < n; ++i) r[i] = b[i] - r[i];
    double beta = nrm2(n, r);
    double tol = rtol * bnorm;
    while (beta > tol && *iters < maxit) {
        double beta_prev = beta;
        for (int i = 0; i < n; ++i) V[i] = r[i] / beta;
        for (int k = 0; k <= m; ++k) g[k] = 0.0;
        g[0] = beta;
        int j, jused = 0;
        for (j = 0; j < m; ++j) {
            double *vj = V + (size_t)j * n, *vn = V + (size_t)(j + 1) * n;
            or_ilu0_apply(lu, dp, vj, z);
            or_csr_matvec(a, z, w);
            for (int k = 0; k <= j; ++k) {                 /* modified Gram-Schmidt */
                const double *vk = V + (size_t)k * n;
                double hk = 0.0;
                for (int i = 0; i < n; ++i) hk += w[i] * vk[i];
                H[k * m + j] = hk;
                for (int i = 0; i < n; ++i) w[i] -= hk * vk[i];
            }
            double hn = nrm2(n, w);
            H[(j + 1) * m + j] = hn;
            if (hn > 0.0) for (int i = 0; i < n; ++i) vn[i] = w[i] / hn;
            for (int k = 0; k < j; ++k) {                   /* previous Givens rotations */
                double t0 = H[k * m + j], t1 = H[(k + 1) * m + j];
                H[k * m + j] = cs[k] * t0 + sn[k] * t1;
                H[(k + 1) * m + j] = -sn[k] * t0 + cs[k] * t1;
            }
            double d = hypot(H[j * m + j], H[(j + 1) * m + j]);
            cs[j] = H[j * m + j] / d;
            sn[j] = H[(j + 1) * m + j] / d;
            H[j * m + j] = d;
            H[(j + 1) * m + j] = 0.0;
            g[j + 1] = -sn[j] * g[j];
            g[j] = cs[j] * g[j];
            ++*iters;
            jused = j + 1;
            if (fabs(g[j + 1]) <= tol || *iters >= maxit || hn == 0.0) break;
        }
        for (int k = jused - 1; k >= 0; --k) {                /* H y = g */
            double s = g[k];
            for (int q = k + 1; q < jused; ++q) s -= H[k * m + q] * y[q];
            y[k] = s / H[k * m + k];
        }
        for (int i = 0; i < n; ++i) w[i] = 0.0;
        for (int k = 0; k < jused; ++k) {
            const double *vk = V + (size_t)k * n;
            for (int i = 0; i < n; ++i) w[i] += y[k] * vk[i];
        }
        or_ilu0_apply(lu, dp, w, z);
        for (int i = 0; i < n; ++i) x[i] += z[i];
        or_csr_matvec(a, x, r);
        for (int i = 0; i < n; ++i) r[i] = b[i] - r[i];
        beta = nrm2(n, r);
        if (beta > tol && beta > 0.9 * beta_prev && fabs(g[jused]) <= tol) break;   /* stagnated */
    }
    if (beta <= tol) status = 0;
    *relres = beta / bnorm;
    free(V); free(H); free(cs); free(sn); free(g); free(y); free(w); free(z); free(r);
    return status;
}

/* Dense LU with partial pivoting; a is n x n row-major, b overwritten by x. */
int or_dense_lu_solve(int n, double *a, double *b)
{
    for (int k = 0; k < n; ++k) {
        int p = k;
        for (int i = k + 1; i < n; ++i) if (fabs(a[(size_t)i * n + k]) > fabs(a[(size_t)p * n + k])) p = i;
        if (a[(size_t)p * n + k] == 0.0) return -1;
        if (p != k) {
            for (int c = 0; c < n; ++c) { double t = a[(size_t)k * n + c]; a[(size_t)k * n + c] = a[(size_t)p * n + c]; a[(size_t)p * n + c] = t; }
            double t = b[k]; b[k] = b[p]; b[p] = t;
        }
        for (int i = k + 1; i < n; ++i) {
            double l = a[(size_t)i * n + k] / a[(size_t)k * n + k];
            a[(size_t)i * n + k] = l;
            for (int c = k + 1; c < n; ++c) a[(size_t)i * n + c] -= l * a[(size_t)k * n + c];
            b[i] -= l * b[k];
        }
    }
    for (int k = n - 1; k >= 0; --k) {
        double s = b[k];
        for (int c = k + 1; c < n; ++c) s -= a[(size_t)k * n + c] * b[c];
        b[k] = s / a[(size_t)k * n + k];
    }
    return 0;
}
