/*
 * Oracle: the third-order BGK flux at one face Gauss point (Sec. II).
 * TEST INFRASTRUCTURE ONLY (see or_internal.h).
 *
 * Everything is written with a generic polynomial type in the particle
 * velocity (u, v) and zeta = xi . xi, and generic Maxwellian moments:
 *   <u^a v^b zeta^z> = <u^a> <v^b> <zeta^z>
 * with full-space or half-space (u > 0, u < 0) moments in u.  The moment
 * matrix <psi psi^T> is built from those moments and inverted by dense LU,
 * and the time integrals of c1..c8 (Eq. (13)) are taken by composite
 * Gauss-Legendre quadrature.  No closed form of the slope solve or of the
 * time integrals is used here.
 *
 * Face frame: x is the face normal (from the left to the right cell), y the
 * tangent.  A state row-block is W[6][4]: value, d/dn, d/dt, d2/dn2,
 * d2/dndt, d2/dt2 of (rho, rho U, rho V, E).
 */
#include <math.h>
#include <stdlib.h>
#include <string.h>

#include "or_internal.h"

#define PU 10   /* powers of u: 0..9    */
#define PV 10   /* powers of v: 0..9    */
#define PZ 4    /* powers of zeta: 0..3 */

/* Coefficients c[a][b][z] of u^a v^b zeta^z; nu, nv, nz bound the powers in
 * use (every coefficient outside them is zero), so loops stay short. */
typedef struct { int nu, nv, nz; double c[PU][PV][PZ]; } poly;

static __thread int g_overflow;   /* set if a product exceeds the supported degree */

static void p_zero(poly *p) { memset(p, 0, sizeof(*p)); p->nu = p->nv = p->nz = 1; }

static int imax(int a, int b) { return a > b ? a : b; }

static void p_axpy(poly *y, double s, const poly *x)
{
    for (int a = 0; a < x->nu; ++a)
        for (int b = 0; b < x->nv; ++b)
            for (int z = 0; z < x->nz; ++z) y->c[a][b][z] += s * x->c[a][b][z];
    y->nu = imax(y->nu, x->nu); y->nv = imax(y->nv, x->nv); y->nz = imax(y->nz, x->nz);
}

static void p_mul(poly *out, const poly *x, const poly *y)
{
    int ya[PU * PV * PZ], yb[PU * PV * PZ], yz[PU * PV * PZ];
    double yv[PU * PV * PZ];
    int ny = 0;
    for (int a = 0; a < y->nu; ++a)
        for (int b = 0; b < y->nv; ++b)
            for (int z = 0; z < y->nz; ++z)
                if (y->c[a][b][z] != 0.0) { ya[ny] = a; yb[ny] = b; yz[ny] = z; yv[ny] = y->c[a][b][z]; ++ny; }
    poly r;
    p_zero(&r);
    r.nu = x->nu + y->nu - 1; r.nv = x->nv + y->nv - 1; r.nz = x->nz + y->nz - 1;
    if (r.nu > PU) r.nu = PU;
    if (r.nv > PV) r.nv = PV;
    if (r.nz > PZ) r.nz = PZ;
    for (int a = 0; a < x->nu; ++a)
        for (int b = 0; b < x->nv; ++b)
            for (int z = 0; z < x->nz; ++z) {
                double xv = x->c[a][b][z];
                if (xv == 0.0) continue;
                for (int k = 0; k < ny; ++k) {
                    int a2 = a + ya[k], b2 = b + yb[k], z2 = z + yz[k];
                    if (a2 >= PU || b2 >= PV || z2 >= PZ) { g_overflow = 1; continue; }
                    r.c[a2][b2][z2] += xv * yv[k];
                }
            }
    *out = r;
}

static void p_mono(poly *p, double coef, int a, int b, int z)
{
    p_zero(p);
    p->c[a][b][z] = coef;
    p->nu = a + 1; p->nv = b + 1; p->nz = z + 1;
}

/* psi_alpha of Eq. (4): 1, u, v, (u^2 + v^2 + zeta)/2 */
static void p_psi(poly *p, int alpha)
{
    p_zero(p);
    switch (alpha) {
    case 0: p->c[0][0][0] = 1.0; break;
    case 1: p->c[1][0][0] = 1.0; p->nu = 2; break;
    case 2: p->c[0][1][0] = 1.0; p->nv = 2; break;
    default: p->c[2][0][0] = 0.5; p->c[0][2][0] = 0.5; p->c[0][0][1] = 0.5; p->nu = 3; p->nv = 3; p->nz = 2; break;
    }
}

/* a slope "a" of Eq. (12) as the polynomial sum_alpha a_alpha psi_alpha */
static void p_slope(poly *p, const double *s)
{
    poly t;
    p_zero(p);
    for (int al = 0; al < 4; ++al) { p_psi(&t, al); p_axpy(p, s[al], &t); }
}

/* Moment tables, long enough for the shifts by psi and by u psi. */
#define NU (PU + 3)
#define NV (PV + 3)
#define NZ (PZ + 2)
typedef struct {
    double mu[NU];   /* <u^a> for the chosen half or full space */
    double mv[NV];   /* <v^b> full space                         */
    double mz[NZ];   /* <zeta^z>                                 */
} moments;

/* <u^da v^db zeta^dz P> */
static double p_moment_shift(const poly *p, const moments *m, int da, int db, int dz)
{
    double s = 0.0;
    for (int a = 0; a < p->nu; ++a)
        for (int b = 0; b < p->nv; ++b)
            for (int z = 0; z < p->nz; ++z)
                if (p->c[a][b][z] != 0.0) s += p->c[a][b][z] * m->mu[a + da] * m->mv[b + db] * m->mz[z + dz];
    return s;
}

/* <psi_alpha P> for alpha = 0..3 */
static void psi_moment(const poly *P, const moments *m, double *out)
{
    out[0] = p_moment_shift(P, m, 0, 0, 0);
    out[1] = p_moment_shift(P, m, 1, 0, 0);
    out[2] = p_moment_shift(P, m, 0, 1, 0);
    out[3] = 0.5 * (p_moment_shift(P, m, 2, 0, 0) + p_moment_shift(P, m, 0, 2, 0) + p_moment_shift(P, m, 0, 0, 1));
}

/* One-dimensional Maxwellian moments <u^k>, k < n, of
 * sqrt(lam/pi) exp(-lam (u-U)^2): full space (half = 0), u > 0 (half = +1) or
 * u < 0 (half = -1).  Recurrence <u^{k+2}> = U <u^{k+1}> + (k+1)/(2 lam) <u^k>,
 * which holds on either half line because the boundary term at u = 0 vanishes
 * for k + 1 >= 1. */
void or_moments_1d(double U, double lam, int half, int n, double *m)
{
    if (half == 0) { m[0] = 1.0; m[1] = U; }
    else if (half > 0) {
        m[0] = 0.5 * erfc(-sqrt(lam) * U);
        m[1] = U * m[0] + 0.5 * exp(-lam * U * U) / sqrt(M_PI * lam);
    } else {
        m[0] = 0.5 * erfc(sqrt(lam) * U);
        m[1] = U * m[0] - 0.5 * exp(-lam * U * U) / sqrt(M_PI * lam);
    }
    for (int k = 0; k + 2 < n; ++k) m[k + 2] = U * m[k + 1] + (k + 1) / (2.0 * lam) * m[k];
}

/* <zeta^q> for K internal degrees of freedom: Gamma(K/2+q) / (Gamma(K/2) lam^q) */
void or_moments_xi(double lam, double K, int n, double *m)
{
    m[0] = 1.0;
    for (int q = 0; q + 1 < n; ++q) m[q + 1] = m[q] * (0.5 * K + q) / lam;
}

typedef struct {
    double rho, U, V, lam, p;
    moments full, half;   /* half: u > 0 for the left state, u < 0 for the right */
    double M[16];         /* <psi psi^T>, full space                               */
    double a1[4], a2[4], A[4], a11[4], a12[4], a22[4], A1[4], A2[4], At[4];
} kstate;

static __thread double g_K;        /* internal degrees of freedom */

static void state_moments(kstate *s, const double *w, double gamma, int half)
{
    s->rho = w[0];
    s->U = w[1] / w[0];
    s->V = w[2] / w[0];
    double eint = w[3] - 0.5 * s->rho * (s->U * s->U + s->V * s->V);
    s->lam = (g_K + 2.0) * s->rho / (4.0 * eint);                  /* Eq. (3), D = 2 */
    s->p = (gamma - 1.0) * eint;
    or_moments_1d(s->U, s->lam, 0, NU, s->full.mu);
    or_moments_1d(s->V, s->lam, 0, NV, s->full.mv);
    or_moments_xi(s->lam, g_K, NZ, s->full.mz);
    s->half = s->full;
    if (half != 0) or_moments_1d(s->U, s->lam, half, NU, s->half.mu);
    poly pb;
    double col[4];
    for (int be = 0; be < 4; ++be) {             /* M[al][be] = <psi_al psi_be> */
        p_psi(&pb, be);
        psi_moment(&pb, &s->full, col);
        for (int al = 0; al < 4; ++al) s->M[4 * al + be] = col[al];
    }
}

/* a = <psi psi^T>^{-1} b by dense LU */
static void msolve(const kstate *s, const double *b, double *a)
{
    double Mc[16];
    memcpy(Mc, s->M, sizeof(Mc));
    for (int k = 0; k < 4; ++k) a[k] = b[k];
    or_dense_lu_solve(4, Mc, a);
}

/* Slopes of Eq. (12) from the macroscopic derivatives (rows 1..5 of W),
 * using g_x / g = a1, g_xx / g = a11 + a1^2 and the compatibility condition
 * <psi (g_t + u g_x + v g_y)> = 0 and its x, y and t derivatives. */
static void state_slopes(kstate *s, const double *W, int with_At)
{
    poly pa1, pa2, pA, pa11, pa12, pa22, pA1, pA2, t, q, r, un, vn;
    double b[4], mo[4];
    p_mono(&un, 1.0, 1, 0, 0);
    p_mono(&vn, 1.0, 0, 1, 0);
    for (int k = 0; k < 4; ++k) b[k] = W[4 + k] / s->rho;
    msolve(s, b, s->a1);
    for (int k = 0; k < 4; ++k) b[k] = W[8 + k] / s->rho;
    msolve(s, b, s->a2);
    p_slope(&pa1, s->a1);
    p_slope(&pa2, s->a2);
    /* A:  <psi (a1 u + a2 v + A)> = 0 */
    p_mul(&t, &pa1, &un); p_mul(&q, &pa2, &vn); p_axpy(&t, 1.0, &q);
    psi_moment(&t, &s->full, mo);
    for (int k = 0; k < 4; ++k) b[k] = -mo[k];
    msolve(s, b, s->A);
    p_slope(&pA, s->A);
    /* a11, a12, a22:  d2W/rho = <psi (a_ij + a_i a_j)> */
    p_mul(&t, &pa1, &pa1); psi_moment(&t, &s->full, mo);
    for (int k = 0; k < 4; ++k) b[k] = W[12 + k] / s->rho - mo[k];
    msolve(s, b, s->a11);
    p_mul(&t, &pa1, &pa2); psi_moment(&t, &s->full, mo);
    for (int k = 0; k < 4; ++k) b[k] = W[16 + k] / s->rho - mo[k];
    msolve(s, b, s->a12);
    p_mul(&t, &pa2, &pa2); psi_moment(&t, &s->full, mo);
    for (int k = 0; k < 4; ++k) b[k] = W[20 + k] / s->rho - mo[k];
    msolve(s, b, s->a22);
    p_slope(&pa11, s->a11);
    p_slope(&pa12, s->a12);
    p_slope(&pa22, s->a22);
    /* L = a1 u + a2 v + A (the first-order compatibility polynomial) */
    poly L;
    p_mul(&L, &pa1, &un); p_mul(&q, &pa2, &vn); p_axpy(&L, 1.0, &q); p_axpy(&L, 1.0, &pA);
    /* A1: <psi [a1 L + a11 u + a12 v + A1]> = 0 */
    p_mul(&t, &pa1, &L); p_mul(&q, &pa11, &un); p_axpy(&t, 1.0, &q); p_mul(&q, &pa12, &vn); p_axpy(&t, 1.0, &q);
    psi_moment(&t, &s->full, mo);
    for (int k = 0; k < 4; ++k) b[k] = -mo[k];
    msolve(s, b, s->A1);
    /* A2: <psi [a2 L + a12 u + a22 v + A2]> = 0 */
    p_mul(&t, &pa2, &L); p_mul(&q, &pa12, &un); p_axpy(&t, 1.0, &q); p_mul(&q, &pa22, &vn); p_axpy(&t, 1.0, &q);
    psi_moment(&t, &s->full, mo);
    for (int k = 0; k < 4; ++k) b[k] = -mo[k];
    msolve(s, b, s->A2);
    for (int k = 0; k < 4; ++k) s->At[k] = 0.0;
    if (with_At) {
        /* At: <psi [A L + A1 u + A2 v + At]> = 0 */
        p_slope(&pA1, s->A1);
        p_slope(&pA2, s->A2);
        p_mul(&t, &pA, &L); p_mul(&q, &pA1, &un); p_axpy(&t, 1.0, &q); p_mul(&q, &pA2, &vn); p_axpy(&t, 1.0, &q);
        psi_moment(&t, &s->full, mo);
        for (int k = 0; k < 4; ++k) b[k] = -mo[k];
        msolve(s, b, s->At);
    }
    (void)r;
}

/* Gauss-Legendre nodes and weights on [-1, 1] by Newton on P_n. */
void or_gauss_legendre(int n, double *x, double *w)
{
    for (int i = 0; i < n; ++i) {
        double z = cos(M_PI * (i + 0.75) / (n + 0.5)), dp = 0.0;
        for (int it = 0; it < 100; ++it) {
            double p0 = 1.0, p1 = z;
            for (int k = 2; k <= n; ++k) { double p2 = ((2.0 * k - 1.0) * z * p1 - (k - 1.0) * p0) / k; p0 = p1; p1 = p2; }
            if (n == 1) { p1 = z; p0 = 1.0; }
            dp = n * (z * p1 - p0) / (z * z - 1.0);
            double dz = p1 / dp;
            z -= dz;
            if (fabs(dz) < 1e-16) break;
        }
        double p0 = 1.0, p1 = z;
        for (int k = 2; k <= n; ++k) { double p2 = ((2.0 * k - 1.0) * z * p1 - (k - 1.0) * p0) / k; p0 = p1; p1 = p2; }
        dp = n * (z * p1 - p0) / (z * z - 1.0);
        x[i] = z;
        w[i] = 2.0 / ((1.0 - z * z) * dp * dp);
    }
}

/* c1..c8 of Eq. (13) at time t; with tau2_exact the exact kernels of c4, c5,
 * c6 (which carry + 2 tau^2 (1 - e^{-t/tau})) are used instead. */
static void c_of_t(double t, double tau, int tau2_exact, double *c)
{
    double e = exp(-t / tau);
    c[0] = 1.0 - e;
    c[1] = (t + tau) * e - tau;
    c[2] = t - tau + tau * e;
    c[3] = -e * (t * t + 2.0 * t * tau);
    c[4] = t * t - 2.0 * tau * t;
    c[5] = -t * tau - e * t * tau;
    c[6] = e;
    c[7] = -t * e;
    c[8] = t * t * e;                 /* the t^2 c7 factor of the last line of Eq. (11) */
    if (tau2_exact) {
        double k = 2.0 * tau * tau * (1.0 - e);
        c[3] += k; c[4] += k; c[5] += k;
    }
}

/* C_k = int_0^dt c_k(t) dt (k = 1..8) and int_0^dt t^2 c7 dt, by 12-point
 * Gauss-Legendre on sub-intervals [0, tau/16], then doubling up to dt. */
void or_time_integrals(double dt, double tau, int tau2_exact, double *C)
{
    enum { NG = 12 };
    double gx[NG], gw[NG];
    or_gauss_legendre(NG, gx, gw);
    for (int k = 0; k < 9; ++k) C[k] = 0.0;
    double a = 0.0, b = fmin(dt, tau / 16.0);
    while (a < dt) {
        for (int q = 0; q < NG; ++q) {
            double t = 0.5 * (a + b) + 0.5 * (b - a) * gx[q], c[9];
            c_of_t(t, tau, tau2_exact, c);
            for (int k = 0; k < 9; ++k) C[k] += 0.5 * (b - a) * gw[q] * c[k];
        }
        a = b;
        b = fmin(dt, 2.0 * b);
    }
}

/* Build the polynomial multiplying g in the time-integrated distribution:
 *   coefficient of 1, A, (a1 u + a2 v), S2, ((A a1 + A1) u + (A a2 + A2) v) and
 *   (A^2 + At), with S2 = (a1^2+a11) u^2 + 2 (a1 a2 + a12) u v + (a2^2+a22) v^2. */
static void build_q(poly *Q, const kstate *s, double k1, double kA, double kL, double kS2,
                    double kAL, double kAA)
{
    poly pa1, pa2, pA, pa11, pa12, pa22, pA1, pA2, pAt, t, q, un, vn, uu, uv, vv;
    p_mono(&un, 1.0, 1, 0, 0); p_mono(&vn, 1.0, 0, 1, 0);
    p_mono(&uu, 1.0, 2, 0, 0); p_mono(&uv, 1.0, 1, 1, 0); p_mono(&vv, 1.0, 0, 2, 0);
    p_slope(&pa1, s->a1); p_slope(&pa2, s->a2); p_slope(&pA, s->A);
    p_slope(&pa11, s->a11); p_slope(&pa12, s->a12); p_slope(&pa22, s->a22);
    p_slope(&pA1, s->A1); p_slope(&pA2, s->A2); p_slope(&pAt, s->At);
    p_mono(Q, k1, 0, 0, 0);
    p_axpy(Q, kA, &pA);
    p_mul(&t, &pa1, &un); p_axpy(Q, kL, &t);
    p_mul(&t, &pa2, &vn); p_axpy(Q, kL, &t);
    /* S2 */
    p_mul(&q, &pa1, &pa1); p_axpy(&q, 1.0, &pa11); p_mul(&t, &q, &uu); p_axpy(Q, kS2, &t);
    p_mul(&q, &pa1, &pa2); p_axpy(&q, 1.0, &pa12); p_mul(&t, &q, &uv); p_axpy(Q, 2.0 * kS2, &t);
    p_mul(&q, &pa2, &pa2); p_axpy(&q, 1.0, &pa22); p_mul(&t, &q, &vv); p_axpy(Q, kS2, &t);
    /* (A a1 + A1) u + (A a2 + A2) v */
    p_mul(&q, &pA, &pa1); p_axpy(&q, 1.0, &pA1); p_mul(&t, &q, &un); p_axpy(Q, kAL, &t);
    p_mul(&q, &pA, &pa2); p_axpy(&q, 1.0, &pA2); p_mul(&t, &q, &vn); p_axpy(Q, kAL, &t);
    /* A^2 + At */
    p_mul(&q, &pA, &pA); p_axpy(&q, 1.0, &pAt); p_axpy(Q, kAA, &q);
}

/* <u psi_alpha Q> */
static void flux_moment(const poly *Q, const moments *m, double *out)
{
    out[0] = p_moment_shift(Q, m, 1, 0, 0);
    out[1] = p_moment_shift(Q, m, 2, 0, 0);
    out[2] = p_moment_shift(Q, m, 1, 1, 0);
    out[3] = 0.5 * (p_moment_shift(Q, m, 3, 0, 0) + p_moment_shift(Q, m, 1, 2, 0) + p_moment_shift(Q, m, 1, 0, 1));
}

/* Heat flux <(1/2) (u - U) |c|^2 Q>, c = (u - U, v - V, xi), of the time-integrated
 * distribution Q relative to the velocity (U, V): the polynomial
 * (1/2)[(u-U)^3 + (u-U)(v-V)^2 + (u-U) zeta] expanded in monomials, each moment
 * taken directly. */
static double heat_moment(const poly *Q, const moments *m, double U, double V)
{
    const struct { int a, b, z; double c; } t[10] = {
        {3, 0, 0, 0.5}, {2, 0, 0, -1.5 * U}, {1, 0, 0, 0.5 * (3.0 * U * U + V * V)},
        {0, 0, 0, -0.5 * (U * U * U + U * V * V)}, {1, 2, 0, 0.5}, {1, 1, 0, -V}, {0, 2, 0, -0.5 * U},
        {0, 1, 0, U * V}, {1, 0, 1, 0.5}, {0, 0, 1, -0.5 * U}};
    double q = 0.0;
    for (int k = 0; k < 10; ++k) q += t[k].c * p_moment_shift(Q, m, t[k].a, t[k].b, t[k].z);
    return q;
}

/* Interface equilibrium W0 of one Gauss point, rows value, d/dn, d/dt, d2/dn2,
 * d2/dndt, d2/dt2 (face frame), from the left/right states with their slopes.
 * The value is rho_l <psi>_{u>0,l} + rho_r <psi>_{u<0,r}.  The derivative rows:
 *   mode 0: the mean of the left and right rows;
 *   mode 1: the kinetic weighting of the same splitting, the half-space moments
 *     of the derivatives of the two distributions, rho_k <psi g_k'/g_k>_k with
 *     g_n/g = a1.psi, g_t/g = a2.psi, g_nn/g = (a1.psi)^2 + a11.psi,
 *     g_nt/g = (a1.psi)(a2.psi) + a12.psi, g_tt/g = (a2.psi)^2 + a22.psi
 *     (the derivatives of a Maxwellian in the paper's nomenclature); these are
 *     the exact derivatives of the value formula when the two states vary as
 *     their reconstructions do. */
static void interface_w0(const kstate *L, const kstate *R, const double *wl, const double *wr, int mode,
                         double *w0)
{
    double ml[4], mr[4];
    poly one;
    p_mono(&one, 1.0, 0, 0, 0);
    psi_moment(&one, &L->half, ml);
    psi_moment(&one, &R->half, mr);
    for (int k = 0; k < 4; ++k) w0[k] = L->rho * ml[k] + R->rho * mr[k];
    if (mode == 0) {
        for (int k = 4; k < 24; ++k) w0[k] = 0.5 * (wl[k] + wr[k]);
        return;
    }
    for (int k = 4; k < 24; ++k) w0[k] = 0.0;
    const kstate *S[2] = {L, R};
    for (int side = 0; side < 2; ++side) {
        const kstate *s = S[side];
        poly s1, s2, t, u;
        double out[4];
        p_slope(&s1, s->a1);
        p_slope(&s2, s->a2);
        psi_moment(&s1, &s->half, out);
        for (int q = 0; q < 4; ++q) w0[4 + q] += s->rho * out[q];
        psi_moment(&s2, &s->half, out);
        for (int q = 0; q < 4; ++q) w0[8 + q] += s->rho * out[q];
        const poly *fa[3] = {&s1, &s1, &s2}, *fb[3] = {&s1, &s2, &s2};
        const double *sec[3] = {s->a11, s->a12, s->a22};
        for (int r = 0; r < 3; ++r) {
            p_mul(&t, fa[r], fb[r]);
            p_slope(&u, sec[r]);
            p_axpy(&t, 1.0, &u);
            psi_moment(&t, &s->half, out);
            for (int q = 0; q < 4; ++q) w0[12 + 4 * r + q] += s->rho * out[q];
        }
    }
}

/* Time-integrated flux through a unit-length face at one Gauss point, in the
 * face frame, from the left and right states wl[24], wr[24] (rows: value,
 * d/dn, d/dt, d2/dn2, d2/dndt, d2/dt2).  f[4] = int_0^dt F dt.
 * aux (optional, 16): tau, W0[4], C1..C8, C7t, p_l, p_r.
 * Returns nonzero if a state is not physical (rho <= 0 or p <= 0). */
int or_gp_flux(const double *wl, const double *wr, double dt, const or_params *prm, double *f, double *aux)
{
    const double gamma = prm->gamma;
    g_K = 2.0 / (gamma - 1.0) - 2.0;          /* (K + D)/2 = 1/(gamma - 1), D = 2 */
    g_overflow = 0;
    kstate L, R, Z;
    state_moments(&L, wl, gamma, +1);
    state_moments(&R, wr, gamma, -1);
    if (!(L.rho > 0.0) || !(R.rho > 0.0) || !(L.p > 0.0) || !(R.p > 0.0)) return 1;
    state_slopes(&L, wl, 0);
    state_slopes(&R, wr, 0);

    /* interface equilibrium: W0 = rho_l <psi>_{u>0,l} + rho_r <psi>_{u<0,r} */
    double w0[24];
    interface_w0(&L, &R, wl, wr, prm->slope0_mode, w0);
    state_moments(&Z, w0, gamma, 0);
    if (!(Z.rho > 0.0) || !(Z.p > 0.0)) return 1;
    state_slopes(&Z, w0, 1);

    /* collision time, Eqs. (39)-(40); the pressure-jump term is scaled by dt */
    double jump = fabs(L.p - R.p) / fabs(L.p + R.p);
    double tau = (prm->mu > 0.0) ? prm->mu / Z.p + dt * jump : 0.01 * dt + dt * jump;

    double C[9];
    or_time_integrals(dt, tau, prm->tau2_exact, C);
    const double C1 = C[0], C2 = C[1], C3 = C[2], C4 = C[3], C5 = C[4], C6 = C[5];
    const double C7 = C[6], C8 = C[7], C7t = C[8];

    /* equilibrium part, Eq. (15) at the Gauss point (y = 0) */
    poly Q0, Ql, Qr;
    build_q(&Q0, &Z, C1, C3, C2, 0.5 * C4, C6, 0.5 * C5);
    /* non-equilibrium part, Eq. (11) at y = 0 */
    build_q(&Ql, &L, C7, -tau * C7, C8 - tau * C7, 0.5 * C7t - tau * C8, -tau * C8, 0.0);
    build_q(&Qr, &R, C7, -tau * C7, C8 - tau * C7, 0.5 * C7t - tau * C8, -tau * C8, 0.0);
    double f0[4], fl[4], fr[4];
    flux_moment(&Q0, &Z.full, f0);
    flux_moment(&Ql, &L.half, fl);
    flux_moment(&Qr, &R.half, fr);
    for (int k = 0; k < 4; ++k) f[k] = Z.rho * f0[k] + L.rho * fl[k] + R.rho * fr[k];
    /* Prandtl number (not in the paper; the BGK model has Pr = 1): the heat flux
     * relative to the interface equilibrium velocity is rescaled by 1/Pr in the
     * energy flux, F_E += (1/Pr - 1) q (the correction of the BGK-NS scheme,
     * K. Xu, J. Comput. Phys. 171 (2001) 289-335). */
    if (prm->prandtl != 1.0) {
        const double q = Z.rho * heat_moment(&Q0, &Z.full, Z.U, Z.V) + L.rho * heat_moment(&Ql, &L.half, Z.U, Z.V) +
                         R.rho * heat_moment(&Qr, &R.half, Z.U, Z.V);
        f[3] += (1.0 / prm->prandtl - 1.0) * q;
    }
    if (aux) {
        aux[0] = tau;
        for (int k = 0; k < 4; ++k) aux[1 + k] = w0[k];
        for (int k = 0; k < 9; ++k) aux[5 + k] = C[k];
        aux[14] = L.p; aux[15] = R.p;
    }
    return g_overflow ? 2 : 0;
}

/* W0 rows [24] of a Gauss point (exported for tests; see interface_w0).
 * Returns nonzero if a state is not physical. */
int or_interface_w0(const double *wl, const double *wr, double gamma, int mode, double *w0)
{
    g_K = 2.0 / (gamma - 1.0) - 2.0;
    g_overflow = 0;
    kstate L, R;
    state_moments(&L, wl, gamma, +1);
    state_moments(&R, wr, gamma, -1);
    if (!(L.rho > 0.0) || !(R.rho > 0.0) || !(L.p > 0.0) || !(R.p > 0.0)) return 1;
    state_slopes(&L, wl, 0);
    state_slopes(&R, wr, 0);
    interface_w0(&L, &R, wl, wr, mode, w0);
    return g_overflow ? 2 : 0;
}

/* Slopes of one state (exported for tests): out[36] = a1 a2 A a11 a12 a22 A1 A2 At. */
int or_state_slopes(const double *w, double gamma, double *out)
{
    g_K = 2.0 / (gamma - 1.0) - 2.0;
    g_overflow = 0;
    kstate s;
    state_moments(&s, w, gamma, 0);
    state_slopes(&s, w, 1);
    const double *src[9] = {s.a1, s.a2, s.A, s.a11, s.a12, s.a22, s.A1, s.A2, s.At};
    for (int k = 0; k < 9; ++k) for (int q = 0; q < 4; ++q) out[4 * k + q] = src[k][q];
    return g_overflow;
}

/* <u^a v^b zeta^z> of a Maxwellian (exported for tests). */
double or_moment_abz(double U, double V, double lam, double K, int half, int a, int b, int z)
{
    double mu[NU], mv[NV], mz[NZ];
    if (a >= NU || b >= NV || z >= NZ) return NAN;
    or_moments_1d(U, lam, half, NU, mu);
    or_moments_1d(V, lam, 0, NV, mv);
    or_moments_xi(lam, K, NZ, mz);
    return mu[a] * mv[b] * mz[z];
}
