// Shock detector and DWBAP limiter on the CLS reconstruction (Sec. III.C).
//
// Reading of Eqs. (34)-(38) used here (the CPU checker of the tests follows the
// same reading, written independently):
//  - detector, Eq. (37): IS_i = sum_j |u_i(r_i) - u_j(r_i)| /
//    (J h_i^{(k_i+1)/2} max(ubar_i, ubar_j)) over the J face neighbours, for the
//    density and for the total energy; the cell is limited unless both are
//    below 1 (Eq. (38));
//  - DWBAP, Eqs. (34)-(36): a derivative of a flagged cell becomes
//    u_0 tan(sum_j omega_j arctan(u_j / u_0)) (0 when u_0 = 0), u_0 the cell's
//    own derivative and u_j the same derivative of neighbour j's polynomial at
//    the cell centroid; omega_j = beta_j / sum beta, beta_j = d_j^{-S(chi)},
//    d_j the mean distance from candidate j's centroid (the cell's own for
//    j = 0) to the cell's interior-face midpoints, S(chi) = 1/(sqrt(chi + 1e-8)
//    + 0.05), chi = standard deviation / mean of the neighbours' pressures;
//    second derivatives (from neighbours with k_j = 2, weights renormalised)
//    and first derivatives, all from the unlimited polynomials;
//  - positivity (not in the paper): a cell is also limited when its unlimited
//    polynomial has rho <= 0 or p <= 0 at one of its face Gauss points; a
//    limited cell whose polynomial still has one keeps its cell average only
//    (all coefficients zero);
//  - characteristic variables (limit_char = 1; Sec. IV.B compares them with the
//    conservative ones): each derivative row is limited in the eigenvector
//    basis of the Euler flux Jacobian at the cell average, along x for d/dx and
//    d2/dx2, y for d/dy and d2/dy2 and the diagonal for d2/dxdy;
//  - robust mode (limiter = 2, not in the paper): a limited cell keeps its
//    cell average only (first order), for contacts with density ratios near
//    10, where the DWBAP polynomials let cell averages turn negative.
//
// One thread per cell, FP64.  The unlimited coefficients stay in x (the warm
// start of the next CLS solve); the limited ones are written to a separate
// array that the flux kernel reads.
#include <cmath>

#include "gks_internal.h"

namespace gks {
namespace {

// Variable v of cell c's polynomial at offset (dx, dy) in c's scaled frame.
__device__ __forceinline__ double poly_value(const DeviceMesh &d, const double *__restrict__ w, const double *x,
                                             int64_t c, int v, double dx, double dy)
{
    const int64_t T = d.T;
    const double qx = dx * dx - d.mxx[c], qxy = dx * dy - d.mxy[c], qy = dy * dy - d.myy[c];
    return w[v * T + c] + x[(v * 5 + 0) * T + c] * dx + x[(v * 5 + 1) * T + c] * dy +
           0.5 * x[(v * 5 + 2) * T + c] * qx + x[(v * 5 + 3) * T + c] * qxy + 0.5 * x[(v * 5 + 4) * T + c] * qy;
}

// Right (columns) and left (rows) eigenvectors, row-major 4x4, of the Jacobian
// of the Euler flux along the unit direction (nx, ny) at the conservative
// state W (eigenvalues q_n - c, q_n, q_n, q_n + c).
__device__ __forceinline__ void char_basis(const double *W, double gamma, double nx, double ny, double *R, double *L)
{
    const double rho = W[0], u = W[1] / rho, v = W[2] / rho;
    const double ke = 0.5 * (u * u + v * v);
    const double p = (gamma - 1.0) * (W[3] - rho * ke);
    const double c = sqrt(gamma * p / rho), H = (W[3] + p) / rho;
    const double qn = u * nx + v * ny, qt = -u * ny + v * nx;
    const double b1 = (gamma - 1.0) / (c * c), b2 = b1 * ke, ic = 1.0 / c;
    R[0] = 1.0;             R[1] = 1.0; R[2] = 0.0; R[3] = 1.0;
    R[4] = u - c * nx;      R[5] = u;   R[6] = -ny; R[7] = u + c * nx;
    R[8] = v - c * ny;      R[9] = v;   R[10] = nx; R[11] = v + c * ny;
    R[12] = H - qn * c;     R[13] = ke; R[14] = qt; R[15] = H + qn * c;
    L[0] = 0.5 * (b2 + qn * ic);  L[1] = -0.5 * (b1 * u + nx * ic); L[2] = -0.5 * (b1 * v + ny * ic); L[3] = 0.5 * b1;
    L[4] = 1.0 - b2;              L[5] = b1 * u;                    L[6] = b1 * v;                    L[7] = -b1;
    L[8] = -qt;                   L[9] = -ny;                       L[10] = nx;                       L[11] = 0.0;
    L[12] = 0.5 * (b2 - qn * ic); L[13] = -0.5 * (b1 * u - nx * ic); L[14] = -0.5 * (b1 * v - ny * ic); L[15] = 0.5 * b1;
}

// u_0 tan(sum_j om_j atan(u_j / u_0)) over the first n of 4 candidates.
__device__ __forceinline__ double biased_mean(const double (&u)[4], const double (&om)[4], int n)
{
    if (u[0] == 0.0) return 0.0;
    double acc = 0.0;
#pragma unroll
    for (int j = 0; j < 4; ++j)
        if (j < n) acc += om[j] * atan(u[j] / u[0]);
    return u[0] * tan(acc);
}

// rho > 0 and p > 0 at all face Gauss points of cell i for the coefficients c.
__device__ __forceinline__ bool physical_gp(const DeviceMesh &d, const double *__restrict__ w, const double *c,
                                            int64_t i, double gamma)
{
    const int64_t T = d.T, F = d.F;
    bool ok = true;
#pragma unroll
    for (int s = 0; s < 3; ++s) {
        const int32_t cf = d.cf[s * T + i];
        if (cf < 0) continue;
        const int64_t f = cf >> 1;
        const double *g = (cf & 1) ? d.gr : d.gl;
#pragma unroll
        for (int k = 0; k < 2; ++k) {
            const double dx = g[(2 * k) * F + f], dy = g[(2 * k + 1) * F + f];
            const double rho = poly_value(d, w, c, i, 0, dx, dy);
            const double mx = poly_value(d, w, c, i, 1, dx, dy), my = poly_value(d, w, c, i, 2, dx, dy);
            const double E = poly_value(d, w, c, i, 3, dx, dy);
            const double p = (gamma - 1.0) * (E - 0.5 * (mx * mx + my * my) / rho);
            ok = ok && rho > 0.0 && p > 0.0;
        }
    }
    return ok;
}

__global__ void __launch_bounds__(kBlock) k_limit(const DeviceMesh d, const double *__restrict__ w,
                                                  const double *__restrict__ x, double *xl,
                                                  int32_t *__restrict__ flag, double gamma, int robust, int charm)
{
    const int64_t T = d.T, F = d.F;
    const int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (i >= T) return;
    int32_t nbj[3];
    double oxj[3], oyj[3];
    int J = 0;
#pragma unroll
    for (int s = 0; s < 3; ++s) {
        nbj[s] = d.nb[s * T + i];      // neighbour slots are filled from slot 0
        oxj[s] = d.ox[s * T + i];
        oyj[s] = d.oy[s * T + i];
        J += nbj[s] >= 0;
    }
    const double hi = d.h[i];
    const int ki = d.kord[i];
    bool flagged = false;
    if (J > 0) {
        // Eq. (37) for rho and E
        const double v0 = poly_value(d, w, x, i, 0, 0.0, 0.0), v3 = poly_value(d, w, x, i, 3, 0.0, 0.0);
        double s0 = 0.0, s3 = 0.0, m0 = w[i], m3 = w[3 * T + i];
#pragma unroll
        for (int s = 0; s < 3; ++s) {
            if (s >= J) continue;
            const int64_t j = nbj[s];
            const double r = hi / d.h[j];
            const double ddx = -oxj[s] * r, ddy = -oyj[s] * r;   // r_i in j's scaled frame
            s0 += fabs(v0 - poly_value(d, w, x, j, 0, ddx, ddy));
            s3 += fabs(v3 - poly_value(d, w, x, j, 3, ddx, ddy));
            m0 = fmax(m0, w[j]);
            m3 = fmax(m3, w[3 * T + j]);
        }
        const double scale = J * pow(hi, 0.5 * (ki + 1));
        flagged = !(s0 / (scale * m0) < 1.0 && s3 / (scale * m3) < 1.0) || !physical_gp(d, w, x, i, gamma);
    }
    if (!flagged) {
#pragma unroll 4
        for (int q = 0; q < 20; ++q) xl[q * T + i] = x[q * T + i];
        flag[i] = 0;
        return;
    }
    if (robust) {
        for (int q = 0; q < 20; ++q) xl[q * T + i] = 0.0;
        flag[i] = 2;
        return;
    }

    // ---- weights, Eqs. (35)-(36); distances in i's scaled frame times h_i
    double fmx[3] = {0.0, 0.0, 0.0}, fmy[3] = {0.0, 0.0, 0.0};
    int nf = 0;
#pragma unroll
    for (int s = 0; s < 3; ++s) {
        const int32_t cf = d.cf[s * T + i];
        if (cf < 0) continue;
        const int64_t f = cf >> 1;
        if (d.fr[f] < 0) continue;
        const double *g = (cf & 1) ? d.gr : d.gl;   // the two Gauss points straddle the midpoint
        const double mx = 0.5 * (g[f] + g[2 * F + f]), my = 0.5 * (g[F + f] + g[3 * F + f]);
        if (nf == 0) { fmx[0] = mx; fmy[0] = my; }
        else if (nf == 1) { fmx[1] = mx; fmy[1] = my; }
        else { fmx[2] = mx; fmy[2] = my; }
        ++nf;
    }
    double X[3] = {0.0, 0.0, 0.0}, Xbar = 0.0;
#pragma unroll
    for (int s = 0; s < 3; ++s) {
        if (s >= J) continue;
        const int64_t j = nbj[s];
        const double rho = w[j], u = w[T + j] / rho, v = w[2 * T + j] / rho;
        X[s] = (gamma - 1.0) * (w[3 * T + j] - 0.5 * rho * (u * u + v * v));
        Xbar += X[s] / J;
    }
    double var = 0.0;
#pragma unroll
    for (int s = 0; s < 3; ++s)
        if (s < J) var += (X[s] - Xbar) * (X[s] - Xbar) / J;
    const double chi = sqrt(var) / Xbar;
    const double S = 1.0 / (sqrt(chi + 1e-8) + 0.05);
    double om[4] = {0.0, 0.0, 0.0, 0.0}, bsum = 0.0;
#pragma unroll
    for (int c = 0; c < 4; ++c) {
        if (c > J) continue;
        const double px = c == 0 ? 0.0 : oxj[c - 1], py = c == 0 ? 0.0 : oyj[c - 1];
        double dist = 0.0;
#pragma unroll
        for (int q = 0; q < 3; ++q)
            if (q < nf) dist += hi * hypot(px - fmx[q], py - fmy[q]) / nf;
        om[c] = pow(dist, -S);
        bsum += om[c];
    }
#pragma unroll
    for (int c = 0; c < 4; ++c) om[c] /= bsum;

    double hj[3] = {1.0, 1.0, 1.0}, ddx[3] = {0.0, 0.0, 0.0}, ddy[3] = {0.0, 0.0, 0.0};
    bool k2[3] = {false, false, false};
#pragma unroll
    for (int s = 0; s < 3; ++s) {
        if (s >= J) continue;
        hj[s] = d.h[nbj[s]];
        ddx[s] = -oxj[s] * hi / hj[s];
        ddy[s] = -oyj[s] * hi / hj[s];
        k2[s] = d.kord[nbj[s]] == 2;
    }
    // candidates of every derivative row l, in physical units: cand[c][v] for the
    // cell's own polynomial (c = 0) and the neighbours' (at r_i; for the second
    // derivatives only neighbours with k = 2, weights renormalised)
    const double Wi[4] = {w[i], w[T + i], w[2 * T + i], w[3 * T + i]};
    for (int l = 0; l < 5; ++l) {
        if (l >= 2 && ki != 2) {
            for (int v = 0; v < 4; ++v) xl[(v * 5 + l) * T + i] = x[(v * 5 + l) * T + i];
            continue;
        }
        double cand[4][4] = {}, omc[4] = {0.0, 0.0, 0.0, 0.0};
        const double sc = l < 2 ? hi : hi * hi;
#pragma unroll
        for (int v = 0; v < 4; ++v) cand[0][v] = x[(v * 5 + l) * T + i] / sc;
        omc[0] = om[0];
        double os = om[0];
        int n = 1;
#pragma unroll
        for (int s = 0; s < 3; ++s) {
            if (s >= J || (l >= 2 && !k2[s])) continue;
            const int64_t j = nbj[s];
#pragma unroll
            for (int v = 0; v < 4; ++v) {
                double c;
                if (l >= 2) {
                    c = x[(v * 5 + l) * T + j] / (hj[s] * hj[s]);
                } else {
                    const double ua = x[(v * 5 + l) * T + j];          // u1 (l = 0) or u2 (l = 1)
                    const double ub = x[(v * 5 + 2 + l) * T + j];      // u3 or u4
                    const double uc = x[(v * 5 + 3 + l) * T + j];      // u4 or u5
                    c = (ua + ub * ddx[s] + uc * ddy[s]) / hj[s];
                }
                if (n == 1) cand[1][v] = c;
                else if (n == 2) cand[2][v] = c;
                else cand[3][v] = c;
            }
            if (n == 1) omc[1] = om[s + 1];
            else if (n == 2) omc[2] = om[s + 1];
            else omc[3] = om[s + 1];
            os += om[s + 1];
            ++n;
        }
#pragma unroll
        for (int q = 0; q < 4; ++q) omc[q] /= os;
        double res[4];
        if (charm) {
            // characteristic variables along x (d/dx, d2/dx2), y (d/dy, d2/dy2), the diagonal (d2/dxdy)
            const double nx = l == 1 || l == 4 ? 0.0 : (l == 3 ? 0.70710678118654752 : 1.0);
            const double ny = l == 0 || l == 2 ? 0.0 : (l == 3 ? 0.70710678118654752 : 1.0);
            double Rm[16], Lm[16];
            char_basis(Wi, gamma, nx, ny, Rm, Lm);
            double lim[4];
#pragma unroll
            for (int a2 = 0; a2 < 4; ++a2) {
                double ch[4];
#pragma unroll
                for (int q = 0; q < 4; ++q)
                    ch[q] = Lm[4 * a2] * cand[q][0] + Lm[4 * a2 + 1] * cand[q][1] + Lm[4 * a2 + 2] * cand[q][2] +
                            Lm[4 * a2 + 3] * cand[q][3];
                lim[a2] = biased_mean(ch, omc, n);
            }
#pragma unroll
            for (int a2 = 0; a2 < 4; ++a2)
                res[a2] = Rm[4 * a2] * lim[0] + Rm[4 * a2 + 1] * lim[1] + Rm[4 * a2 + 2] * lim[2] + Rm[4 * a2 + 3] * lim[3];
        } else {
#pragma unroll
            for (int v = 0; v < 4; ++v) {
                const double cv[4] = {cand[0][v], cand[1][v], cand[2][v], cand[3][v]};
                res[v] = biased_mean(cv, omc, n);
            }
        }
#pragma unroll
        for (int v = 0; v < 4; ++v) xl[(v * 5 + l) * T + i] = sc * res[v];
    }

    // ---- safeguard at the cell's face Gauss points
    const bool bad = !physical_gp(d, w, xl, i, gamma);
    if (bad)
        for (int q = 0; q < 20; ++q) xl[q * T + i] = 0.0;
    flag[i] = bad ? 2 : 1;
}

// caller[perm[i]] = internal[i] for the limiter flags (padding skipped)
__global__ void k_scatter_flags(const int32_t *__restrict__ src, const int32_t *__restrict__ perm,
                                int32_t *__restrict__ dst, int64_t T)
{
    const int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (i >= T) return;
    const int32_t c = perm[i];
    if (c >= 0) dst[c] = src[i];
}

}  // namespace

gks_status launch_limiter(gks_mesh *m, const double *w, const double *x, cudaStream_t s)
{
    const DeviceMesh &d = m->d;
    if (!d.ox || !d.oy || !d.kord || !m->wk.xl || !m->wk.lflag) {
        set_error("the limiter was not enabled when the mesh was created (gks_config.limiter = 1)");
        return GKS_EINVAL;
    }
    if (d.T == 0) return GKS_OK;
    const unsigned nb = (unsigned)((d.T + kBlock - 1) / kBlock);
    k_limit<<<nb, kBlock, 0, s>>>(d, w, x, m->wk.xl, m->wk.lflag, m->cfg.gamma, m->cfg.limiter == 2 ? 1 : 0,
                                  m->cfg.limit_char);
    note_launch();
    GKS_CUDA(cudaGetLastError());
    return GKS_OK;
}

gks_status launch_scatter_flags(gks_mesh *m, int32_t *flags_out, cudaStream_t s)
{
    const DeviceMesh &d = m->d;
    if (d.T == 0) return GKS_OK;
    const unsigned nb = (unsigned)((d.T + kBlock - 1) / kBlock);
    k_scatter_flags<<<nb, kBlock, 0, s>>>(m->wk.lflag, d.perm, flags_out, d.T);
    note_launch();
    GKS_CUDA(cudaGetLastError());
    return GKS_OK;
}

}  // namespace gks
