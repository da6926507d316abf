/*
 * Oracle: shock detector and DWBAP limiter (Sec. III.C, Eqs. (34)-(38)).
 * TEST INFRASTRUCTURE ONLY (see or_internal.h).
 *
 * Reading of the paper used here (and, independently, by the CUDA library):
 *  - detector, Eq. (37): IS_i = sum_j |u_i(r_i) - u_j(r_i)| /
 *    (J h_i^{(k_i+1)/2} max(ubar_i, ubar_j)) over the J face neighbours, for the
 *    density and the total energy; a cell is limited when either is >= 1
 *    (Eq. (38));
 *  - DWBAP, Eqs. (34)-(36): a derivative of cell i is replaced by
 *    u_0 tan(sum_j omega_j arctan(u_j / u_0)) (0 when u_0 = 0), with u_0 the
 *    cell's own value and u_j the same derivative of the neighbour polynomials
 *    at the cell centroid (the biased average of the ratios, so that equal
 *    candidates are left unchanged); weights beta_j = d_j^{-S(chi)},
 *    d_j = mean distance from the candidate's centroid (the cell's own for
 *    j = 0) to the cell's face midpoints, S(chi) = 1/(sqrt(chi + 1e-8) + 0.05),
 *    chi = std / mean of the neighbours' pressures; second derivatives first,
 *    then first derivatives, all from the unlimited neighbour polynomials;
 *  - robust mode (limiter = 2, not in the paper): a limited cell keeps its
 *    cell average only (first order), for contacts with density ratios near
 *    10, where the DWBAP polynomials let cell averages turn negative;
 *  - positivity (not in the paper): a cell is also limited when its
 *    unlimited polynomial gives rho <= 0 or p <= 0 at one of its face Gauss
 *    points; if the limited polynomial of a limited cell still does, the cell
 *    falls back to its cell average (all coefficients zero).
 */
#include <math.h>
#include <stdlib.h>
#include <string.h>

#include "or_internal.h"

void or_eval_cell(const or_mesh *m, const double *w, const double *coef, int c, double x, double y, double *out);

static double biased(const double *u, const double *om, int n)
{
    if (u[0] == 0.0) return 0.0;
    double acc = 0.0;
    for (int j = 0; j < n; ++j) acc += om[j] * atan(u[j] / u[0]);
    return u[0] * tan(acc);
}

/* Detector of Eq. (37) for variable var of cell i. */
static double detector(const or_mesh *m, const double *w, const double *coef, int i, int var)
{
    const int64_t T = m->n_tri;
    const int J = m->nb_cnt[i];
    if (J == 0) return 0.0;
    double gi[24], gj[24];
    or_eval_cell(m, w, coef, i, m->cx[i], m->cy[i], gi);
    double s = 0.0, umax = w[(size_t)var * T + i];
    for (int k = 0; k < J; ++k) {
        int j = m->nb_cell[3 * i + k];
        or_eval_cell(m, w, coef, j, m->cx[i] - m->nb_dx[3 * i + k], m->cy[i] - m->nb_dy[3 * i + k], gj);
        s += fabs(gi[var] - gj[var]);
        umax = fmax(umax, w[(size_t)var * T + j]);
    }
    return s / (J * pow(m->h[i], 0.5 * (m->korder[i] + 1)) * umax);
}

/* 1 if the polynomial of cell i (coefficients coef) gives rho > 0 and p > 0
 * at all of its face Gauss points. */
static int physical_at_gauss_points(const or_mesh *m, const double *w, const double *coef, int64_t i)
{
    const double gamma = m->prm.gamma;
    for (int s = 0; s < 3; ++s) {
        int f = m->cface[3 * i + s];
        if (f < 0) continue;
        for (int g = 0; g < 2; ++g) {
            double x = m->gx[2 * f + g], y = m->gy[2 * f + g];
            if (m->face[5 * f + 2] != (int)i) { x -= m->shift[2 * f]; y -= m->shift[2 * f + 1]; }
            double e[24];
            or_eval_cell(m, w, coef, (int)i, x, y, e);
            double p = (gamma - 1.0) * (e[3] - 0.5 * (e[1] * e[1] + e[2] * e[2]) / e[0]);
            if (!(e[0] > 0.0) || !(p > 0.0)) return 0;
        }
    }
    return 1;
}

/* Limited coefficients coef_out (same layout as coef) and the detector flags
 * (flag[i] = 1 limited, 2 limited and reset to the average).  Returns the
 * number of flagged cells. */
int or_limit(const or_mesh *m, const double *w, const double *coef, double *coef_out, int32_t *flag)
{
    const int64_t T = m->n_tri;
    const double gamma = m->prm.gamma;
    memcpy(coef_out, coef, sizeof(double) * 20 * (size_t)T);
    int nflag = 0;
    for (int64_t i = 0; i < T; ++i) {
        flag[i] = 0;
        const int J = m->nb_cnt[i];
        if (J == 0) continue;
        if (detector(m, w, coef, (int)i, 0) < 1.0 && detector(m, w, coef, (int)i, 3) < 1.0 &&
            physical_at_gauss_points(m, w, coef, i))
            continue;
        flag[i] = 1;
        ++nflag;
        if (m->prm.limiter == 2) {
            flag[i] = 2;
            for (int q = 0; q < 20; ++q) coef_out[(size_t)q * T + i] = 0.0;
            continue;
        }
        /* weights, Eqs. (35)-(36) */
        double fmx[3], fmy[3];
        int nf = 0;
        for (int s = 0; s < 3; ++s) {
            int f = m->cface[3 * i + s];
            if (f < 0 || m->face[5 * f + 3] < 0) continue;
            double ax = m->nodes[2 * m->face[5 * f]], ay = m->nodes[2 * m->face[5 * f] + 1];
            double bx = m->nodes[2 * m->face[5 * f + 1]], by = m->nodes[2 * m->face[5 * f + 1] + 1];
            double mx = 0.5 * (ax + bx), my = 0.5 * (ay + by);
            if (m->face[5 * f + 2] != (int)i) { mx -= m->shift[2 * f]; my -= m->shift[2 * f + 1]; }
            fmx[nf] = mx; fmy[nf] = my; ++nf;
        }
        double px[4], py[4];
        px[0] = m->cx[i]; py[0] = m->cy[i];
        double X[3], Xbar = 0.0;
        for (int k = 0; k < J; ++k) {
            int j = m->nb_cell[3 * i + k];
            px[k + 1] = m->cx[j] + m->nb_dx[3 * i + k];
            py[k + 1] = m->cy[j] + m->nb_dy[3 * i + k];
            double rho = w[j], u = w[T + j] / rho, v = w[2 * T + j] / rho;
            X[k] = (gamma - 1.0) * (w[3 * T + j] - 0.5 * rho * (u * u + v * v));
            Xbar += X[k] / J;
        }
        double var = 0.0;
        for (int k = 0; k < J; ++k) var += (X[k] - Xbar) * (X[k] - Xbar) / J;
        const double chi = sqrt(var) / Xbar;
        const double S = 1.0 / (sqrt(chi + 1e-8) + 0.05);
        double beta[4], bsum = 0.0;
        for (int j = 0; j <= J; ++j) {
            double d = 0.0;
            for (int q = 0; q < nf; ++q) d += hypot(px[j] - fmx[q], py[j] - fmy[q]) / nf;
            beta[j] = pow(d, -S);
            bsum += beta[j];
        }
        double om[4];
        for (int j = 0; j <= J; ++j) om[j] = beta[j] / bsum;
        const double hi = m->h[i];
        for (int v = 0; v < 4; ++v) {
            /* second derivatives (physical) from the cells with k = 2 */
            if (m->korder[i] == 2) {
                for (int l = 2; l < 5; ++l) {
                    double cand[4], omc[4], os = 0.0;
                    int n = 0;
                    cand[n] = coef[((size_t)v * 5 + l) * T + i] / (hi * hi); omc[n] = om[0]; os += om[0]; ++n;
                    for (int k = 0; k < J; ++k) {
                        int j = m->nb_cell[3 * i + k];
                        if (m->korder[j] != 2) continue;
                        cand[n] = coef[((size_t)v * 5 + l) * T + j] / (m->h[j] * m->h[j]);
                        omc[n] = om[k + 1]; os += om[k + 1]; ++n;
                    }
                    for (int q = 0; q < n; ++q) omc[q] /= os;
                    coef_out[((size_t)v * 5 + l) * T + i] = hi * hi * biased(cand, omc, n);
                }
            }
            /* first derivatives at the centroid: own vs neighbour polynomials at r_i */
            double gi[24];
            or_eval_cell(m, w, coef, (int)i, m->cx[i], m->cy[i], gi);
            double gx[4], gy[4];
            gx[0] = gi[4 + v]; gy[0] = gi[8 + v];
            for (int k = 0; k < J; ++k) {
                int j = m->nb_cell[3 * i + k];
                double gj[24];
                or_eval_cell(m, w, coef, j, m->cx[i] - m->nb_dx[3 * i + k], m->cy[i] - m->nb_dy[3 * i + k], gj);
                gx[k + 1] = gj[4 + v]; gy[k + 1] = gj[8 + v];
            }
            /* own gradient at the centroid is (u1 + u3*0 + u4*0)/h: the centroid has zero offset */
            coef_out[((size_t)v * 5 + 0) * T + i] = hi * biased(gx, om, J + 1);
            coef_out[((size_t)v * 5 + 1) * T + i] = hi * biased(gy, om, J + 1);
        }
        /* safeguard at the cell's face Gauss points */
        const int bad = !physical_at_gauss_points(m, w, coef_out, i);
        if (bad) {
            flag[i] = 2;
            for (int q = 0; q < 20; ++q) coef_out[(size_t)q * T + i] = 0.0;
        }
    }
    return nflag;
}
