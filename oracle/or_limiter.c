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
 *  - characteristic variables (limit_char = 1, Sec. IV.B compares them with
 *    the conservative ones): each derivative row is limited in the
 *    eigenvector basis of the Euler flux Jacobian along a direction (x for
 *    d/dx and d2/dx2, y for d/dy and d2/dy2, the diagonal for d2/dxdy) at the
 *    cell average; candidates are mapped by the left eigenvectors, limited
 *    component by component, and mapped back by the right ones;
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

/* Right (columns) and left (rows) eigenvectors of the Jacobian of the Euler
 * flux along the unit direction (nx, ny) at the conservative state W:
 * eigenvalues q_n - c, q_n, q_n, q_n + c.  R and L are 4x4 row-major. */
void or_char_basis(const double *W, double gamma, double nx, double ny, double *R, double *L)
{
    const double rho = W[0], u = W[1] / rho, v = W[2] / rho;
    const double ke = 0.5 * (u * u + v * v);
    const double p = (gamma - 1.0) * (W[3] - rho * ke);
    const double c = sqrt(gamma * p / rho), H = (W[3] + p) / rho;
    const double qn = u * nx + v * ny, qt = -u * ny + v * nx;
    const double Rm[16] = {1.0, 1.0, 0.0, 1.0,
                           u - c * nx, u, -ny, u + c * nx,
                           v - c * ny, v, nx, v + c * ny,
                           H - qn * c, ke, qt, H + qn * c};
    const double b1 = (gamma - 1.0) / (c * c), b2 = b1 * ke;
    const double Lm[16] = {0.5 * (b2 + qn / c), -0.5 * (b1 * u + nx / c), -0.5 * (b1 * v + ny / c), 0.5 * b1,
                           1.0 - b2, b1 * u, b1 * v, -b1,
                           -qt, -ny, nx, 0.0,
                           0.5 * (b2 - qn / c), -0.5 * (b1 * u - nx / c), -0.5 * (b1 * v - ny / c), 0.5 * b1};
    memcpy(R, Rm, sizeof(Rm));
    memcpy(L, Lm, sizeof(Lm));
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
        /* candidates per derivative row l (physical units), cand[c][v]: the cell's
         * own derivative (c = 0) and the neighbours' at r_i */
        double gi[24], gnb[3][24];
        or_eval_cell(m, w, coef, (int)i, m->cx[i], m->cy[i], gi);
        for (int k = 0; k < J; ++k) {
            int j = m->nb_cell[3 * i + k];
            or_eval_cell(m, w, coef, j, m->cx[i] - m->nb_dx[3 * i + k], m->cy[i] - m->nb_dy[3 * i + k], gnb[k]);
        }
        const double wi[4] = {w[i], w[T + i], w[2 * T + i], w[3 * T + i]};
        for (int l = 0; l < 5; ++l) {
            if (l >= 2 && m->korder[i] != 2) continue;
            double cand[4][4], omc[4], os = 0.0;
            int n = 0;
            for (int v = 0; v < 4; ++v)   /* own: d/dx = u1/h at the centroid, second derivatives u/h^2 */
                cand[0][v] = l < 2 ? gi[4 * (l + 1) + v] : coef[((size_t)v * 5 + l) * T + i] / (hi * hi);
            omc[n] = om[0]; os += om[0]; ++n;
            for (int k = 0; k < J; ++k) {
                int j = m->nb_cell[3 * i + k];
                if (l >= 2 && m->korder[j] != 2) continue;
                for (int v = 0; v < 4; ++v)
                    cand[n][v] = l < 2 ? gnb[k][4 * (l + 1) + v]
                                       : coef[((size_t)v * 5 + l) * T + j] / (m->h[j] * m->h[j]);
                omc[n] = om[k + 1]; os += om[k + 1]; ++n;
            }
            for (int q = 0; q < n; ++q) omc[q] /= os;
            double res[4];
            if (m->prm.limit_char) {
                static const double dir[5][2] = {{1, 0}, {0, 1}, {1, 0}, {0.70710678118654752, 0.70710678118654752},
                                                 {0, 1}};
                double Rm[16], Lm[16], ch[4][4], lim[4];
                or_char_basis(wi, gamma, dir[l][0], dir[l][1], Rm, Lm);
                for (int q = 0; q < n; ++q)
                    for (int a = 0; a < 4; ++a) {
                        ch[a][q] = 0.0;
                        for (int b = 0; b < 4; ++b) ch[a][q] += Lm[4 * a + b] * cand[q][b];
                    }
                for (int a = 0; a < 4; ++a) lim[a] = biased(ch[a], omc, n);
                for (int a = 0; a < 4; ++a) {
                    res[a] = 0.0;
                    for (int b = 0; b < 4; ++b) res[a] += Rm[4 * a + b] * lim[b];
                }
            } else {
                for (int v = 0; v < 4; ++v) {
                    double cv[4];
                    for (int q = 0; q < n; ++q) cv[q] = cand[q][v];
                    res[v] = biased(cv, omc, n);
                }
            }
            const double sc = l < 2 ? hi : hi * hi;
            for (int v = 0; v < 4; ++v) coef_out[((size_t)v * 5 + l) * T + i] = sc * res[v];
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
