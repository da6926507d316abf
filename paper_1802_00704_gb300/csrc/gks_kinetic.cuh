// Device arithmetic of the third-order BGK flux at one Gauss point (Sec. II.B).
//
// Notation (face frame): u is the particle velocity along the face normal,
// v along the tangent, e = (u^2 + v^2 + xi.xi)/2, psi = (1, u, v, e) (Eq. (4)).
// A slope (Eq. (12)) is a vector s with s.psi = s0 + s1 u + s2 v + s3 e.
// Moments <u^a v^b e^c> of a Maxwellian are formed on the fly from the 1-D
// moments <u^a> (full or half space), <v^b> and <(xi.xi)^c>.
//
// Polynomials in (u, v, e) of total degree <= 4 are kept as 35 coefficients;
// every loop over them has a constant trip count and is unrolled, so the
// coefficients and moment tables live in registers.
#pragma once

#include <cuda_runtime.h>

namespace gks {
namespace kin {

// ---- monomial tables: u^i v^j e^k, i + j + k <= 4, ordered by k, then j, then i
constexpr int kNM = 35;
struct MonoTab {
    int i[kNM], j[kNM], k[kNM];
    int idx[5][5][5];
};
__host__ __device__ constexpr MonoTab make_tab()
{
    MonoTab t{};
    int n = 0;
    for (int a = 0; a < 5; ++a)
        for (int b = 0; b < 5; ++b)
            for (int c = 0; c < 5; ++c) t.idx[a][b][c] = -1;
    for (int k = 0; k <= 4; ++k)
        for (int j = 0; j <= 4 - k; ++j)
            for (int i = 0; i <= 4 - k - j; ++i) {
                t.i[n] = i;
                t.j[n] = j;
                t.k[n] = k;
                t.idx[i][j][k] = n;
                ++n;
            }
    return t;
}
__device__ constexpr MonoTab kTab = make_tab();
// exponent of psi_beta: 1, u, v, e
__device__ constexpr int kPsiI[4] = {0, 1, 0, 0}, kPsiJ[4] = {0, 0, 1, 0}, kPsiK[4] = {0, 0, 0, 1};

template <typename R>
struct Mom {
    R u[10];   // <u^a>, full or half space
    R v[10];   // <v^b>
    R z[4];    // <(xi.xi)^c>
};

template <typename R>
struct Poly {
    R c[kNM];
};

template <typename R>
__device__ __forceinline__ void pzero(Poly<R> &p)
{
#pragma unroll
    for (int n = 0; n < kNM; ++n) p.c[n] = R(0);
}

// <u^a v^b e^c> from the 1-D moments (c <= 3), e = (u^2 + v^2 + z)/2
template <typename R>
__device__ __forceinline__ R E(const Mom<R> &m, int a, int b, int c)
{
    const R *u = m.u, *v = m.v, *z = m.z;
    if (c == 0) return u[a] * v[b];
    if (c == 1) return R(0.5) * (u[a + 2] * v[b] + u[a] * v[b + 2] + u[a] * v[b] * z[1]);
    if (c == 2)
        return R(0.25) * (u[a + 4] * v[b] + u[a] * v[b + 4] + u[a] * v[b] * z[2] +
                          R(2) * (u[a + 2] * v[b + 2] + (u[a + 2] * v[b] + u[a] * v[b + 2]) * z[1]));
    return R(0.125) * (u[a + 6] * v[b] + u[a] * v[b + 6] + u[a] * v[b] * z[3] +
                       R(3) * (u[a + 4] * v[b + 2] + u[a + 2] * v[b + 4] + (u[a + 4] * v[b] + u[a] * v[b + 4]) * z[1] +
                               (u[a + 2] * v[b] + u[a] * v[b + 2]) * z[2]) +
                       R(6) * u[a + 2] * v[b + 2] * z[1]);
}

// out_alpha = <psi_alpha P> (deg P <= 3 so that every moment stays in the tables)
template <typename R, int DEG>
__device__ __forceinline__ void psi_contract(const Poly<R> &p, const Mom<R> &m, R *out)
{
#pragma unroll
    for (int al = 0; al < 4; ++al) out[al] = R(0);
#pragma unroll
    for (int n = 0; n < kNM; ++n) {
        if (kTab.i[n] + kTab.j[n] + kTab.k[n] > DEG || kTab.k[n] > 2) continue;
        const int i = kTab.i[n], j = kTab.j[n], k = kTab.k[n];
        out[0] += p.c[n] * E(m, i, j, k);
        out[1] += p.c[n] * E(m, i + 1, j, k);
        out[2] += p.c[n] * E(m, i, j + 1, k);
        out[3] += p.c[n] * E(m, i, j, k + 1);
    }
}

// out_alpha = <u psi_alpha Q>
template <typename R>
__device__ __forceinline__ void upsi_contract(const Poly<R> &p, const Mom<R> &m, R *out)
{
#pragma unroll
    for (int al = 0; al < 4; ++al) out[al] = R(0);
#pragma unroll
    for (int n = 0; n < kNM; ++n) {
        if (kTab.k[n] > 2) continue;          // products of two slopes carry at most e^2
        const int i = kTab.i[n], j = kTab.j[n], k = kTab.k[n];
        out[0] += p.c[n] * E(m, i + 1, j, k);
        out[1] += p.c[n] * E(m, i + 2, j, k);
        out[2] += p.c[n] * E(m, i + 1, j + 1, k);
        out[3] += p.c[n] * E(m, i + 1, j, k + 1);
    }
}

// P += f (s.psi) u^i0 v^j0
template <typename R>
__device__ __forceinline__ void add_lin(Poly<R> &p, R f, const R *s, int i0, int j0)
{
#pragma unroll
    for (int b = 0; b < 4; ++b) p.c[kTab.idx[i0 + kPsiI[b]][j0 + kPsiJ[b]][kPsiK[b]]] += f * s[b];
}

// P += f (s.psi)(t.psi) u^i0 v^j0
template <typename R>
__device__ __forceinline__ void add_prod(Poly<R> &p, R f, const R *s, const R *t, int i0, int j0)
{
#pragma unroll
    for (int b = 0; b < 4; ++b)
#pragma unroll
        for (int c = 0; c < 4; ++c)
            p.c[kTab.idx[i0 + kPsiI[b] + kPsiI[c]][j0 + kPsiJ[b] + kPsiJ[c]][kPsiK[b] + kPsiK[c]]] += f * s[b] * t[c];
}

template <typename R>
struct KState {
    R rho, U, V, lam, p;
    R a1[4], a2[4], A[4], a11[4], a12[4], a22[4], A1[4], A2[4], At[4];
};

// Full-space 1-D moments <u^k>, k < 10, of sqrt(lam/pi) exp(-lam (u-U)^2)
template <typename R>
__device__ __forceinline__ void mom_full(R U, R lam, R *m)
{
    const R h = R(0.5) / lam;
    m[0] = R(1);
    m[1] = U;
#pragma unroll
    for (int k = 0; k < 8; ++k) m[k + 2] = U * m[k + 1] + R(k + 1) * h * m[k];
}

// Half-space moments (sign = +1: u > 0, -1: u < 0)
template <typename R>
__device__ __forceinline__ void mom_half(R U, R lam, R sign, R *m)
{
    const R h = R(0.5) / lam;
    const R sl = sqrt(lam);
    m[0] = R(0.5) * erfc(-sign * sl * U);
    m[1] = U * m[0] + sign * R(0.5) * exp(-lam * U * U) / (sl * R(1.7724538509055160273));
#pragma unroll
    for (int k = 0; k < 8; ++k) m[k + 2] = U * m[k + 1] + R(k + 1) * h * m[k];
}

template <typename R>
__device__ __forceinline__ void mom_xi(R lam, R K, R *z)
{
    z[0] = R(1);
    z[1] = R(0.5) * K / lam;
    z[2] = z[1] * (R(0.5) * K + R(1)) / lam;
    z[3] = z[2] * (R(0.5) * K + R(2)) / lam;
}

// a = <psi psi^T>^{-1} b for a full-space Maxwellian (closed form).
template <typename R>
__device__ __forceinline__ void minv(const KState<R> &s, R K, const R *b, R *a)
{
    const R B = s.U * s.U + s.V * s.V + (K + R(2)) / (R(2) * s.lam);
    const R R4 = R(2) * b[3] - B * b[0];
    const R R3 = b[2] - s.V * b[0];
    const R R2 = b[1] - s.U * b[0];
    a[3] = R(4) * s.lam * s.lam / (K + R(2)) * (R4 - R(2) * s.U * R2 - R(2) * s.V * R3);
    a[2] = R(2) * s.lam * R3 - s.V * a[3];
    a[1] = R(2) * s.lam * R2 - s.U * a[3];
    a[0] = b[0] - s.U * a[1] - s.V * a[2] - R(0.5) * a[3] * B;
}

// Primitive variables of a state (rho, rho U, rho V, E); lambda from Eq. (3).
template <typename R>
__device__ __forceinline__ bool prim(const R *w, R gamma, R K, KState<R> &s)
{
    s.rho = w[0];
    s.U = w[1] / w[0];
    s.V = w[2] / w[0];
    const R eint = w[3] - R(0.5) * s.rho * (s.U * s.U + s.V * s.V);
    s.p = (gamma - R(1)) * eint;
    s.lam = (K + R(2)) * s.rho / (R(4) * eint);
    return s.rho > R(0) && s.p > R(0);
}

// Slopes from the macroscopic derivatives W[6][4] (rows 1..5 used):
//   g_n/g = a1, g_t/g = a2, g_nn/g = a11 + a1^2, ..., and the time slopes from
//   the compatibility condition <psi (g_t + u g_n + v g_t)> = 0 and its n, t
//   (and, with with_At, time) derivatives.
template <typename R>
__device__ __forceinline__ void slopes(KState<R> &s, const R *W, R K, const Mom<R> &m, bool with_At)
{
    R b[4], mo[4];
    const R ir = R(1) / s.rho;
#pragma unroll
    for (int q = 0; q < 4; ++q) b[q] = W[4 + q] * ir;
    minv(s, K, b, s.a1);
#pragma unroll
    for (int q = 0; q < 4; ++q) b[q] = W[8 + q] * ir;
    minv(s, K, b, s.a2);
    Poly<R> P;
    // A: <psi (a1 u + a2 v + A)> = 0
    pzero(P);
    add_lin(P, R(1), s.a1, 1, 0);
    add_lin(P, R(1), s.a2, 0, 1);
    psi_contract<R, 2>(P, m, mo);
#pragma unroll
    for (int q = 0; q < 4; ++q) b[q] = -mo[q];
    minv(s, K, b, s.A);
    // a11, a12, a22: second derivatives / rho = <psi (a_ij + a_i a_j)>
    pzero(P);
    add_prod(P, R(1), s.a1, s.a1, 0, 0);
    psi_contract<R, 2>(P, m, mo);
#pragma unroll
    for (int q = 0; q < 4; ++q) b[q] = W[12 + q] * ir - mo[q];
    minv(s, K, b, s.a11);
    pzero(P);
    add_prod(P, R(1), s.a1, s.a2, 0, 0);
    psi_contract<R, 2>(P, m, mo);
#pragma unroll
    for (int q = 0; q < 4; ++q) b[q] = W[16 + q] * ir - mo[q];
    minv(s, K, b, s.a12);
    pzero(P);
    add_prod(P, R(1), s.a2, s.a2, 0, 0);
    psi_contract<R, 2>(P, m, mo);
#pragma unroll
    for (int q = 0; q < 4; ++q) b[q] = W[20 + q] * ir - mo[q];
    minv(s, K, b, s.a22);
    // A1: <psi [a1 (a1 u + a2 v + A) + a11 u + a12 v + A1]> = 0
    pzero(P);
    add_prod(P, R(1), s.a1, s.a1, 1, 0);
    add_prod(P, R(1), s.a1, s.a2, 0, 1);
    add_prod(P, R(1), s.a1, s.A, 0, 0);
    add_lin(P, R(1), s.a11, 1, 0);
    add_lin(P, R(1), s.a12, 0, 1);
    psi_contract<R, 3>(P, m, mo);
#pragma unroll
    for (int q = 0; q < 4; ++q) b[q] = -mo[q];
    minv(s, K, b, s.A1);
    // A2: <psi [a2 (a1 u + a2 v + A) + a12 u + a22 v + A2]> = 0
    pzero(P);
    add_prod(P, R(1), s.a2, s.a1, 1, 0);
    add_prod(P, R(1), s.a2, s.a2, 0, 1);
    add_prod(P, R(1), s.a2, s.A, 0, 0);
    add_lin(P, R(1), s.a12, 1, 0);
    add_lin(P, R(1), s.a22, 0, 1);
    psi_contract<R, 3>(P, m, mo);
#pragma unroll
    for (int q = 0; q < 4; ++q) b[q] = -mo[q];
    minv(s, K, b, s.A2);
    if (with_At) {
        // At: <psi [A (a1 u + a2 v + A) + A1 u + A2 v + At]> = 0
        pzero(P);
        add_prod(P, R(1), s.A, s.a1, 1, 0);
        add_prod(P, R(1), s.A, s.a2, 0, 1);
        add_prod(P, R(1), s.A, s.A, 0, 0);
        add_lin(P, R(1), s.A1, 1, 0);
        add_lin(P, R(1), s.A2, 0, 1);
        psi_contract<R, 3>(P, m, mo);
#pragma unroll
        for (int q = 0; q < 4; ++q) b[q] = -mo[q];
        minv(s, K, b, s.At);
    } else {
#pragma unroll
        for (int q = 0; q < 4; ++q) s.At[q] = R(0);
    }
}

// Q = k1 + kA A + kL (a1 u + a2 v) + kS [(a1^2+a11) u^2 + 2 (a1 a2 + a12) u v + (a2^2+a22) v^2]
//     + kAL [(A a1 + A1) u + (A a2 + A2) v] + kAA (A^2 + At)
template <typename R>
__device__ __forceinline__ void build_q(Poly<R> &Q, const KState<R> &s, R k1, R kA, R kL, R kS, R kAL, R kAA)
{
    pzero(Q);
    Q.c[0] += k1;
    add_lin(Q, kA, s.A, 0, 0);
    add_lin(Q, kL, s.a1, 1, 0);
    add_lin(Q, kL, s.a2, 0, 1);
    add_prod(Q, kS, s.a1, s.a1, 2, 0);
    add_lin(Q, kS, s.a11, 2, 0);
    add_prod(Q, R(2) * kS, s.a1, s.a2, 1, 1);
    add_lin(Q, R(2) * kS, s.a12, 1, 1);
    add_prod(Q, kS, s.a2, s.a2, 0, 2);
    add_lin(Q, kS, s.a22, 0, 2);
    add_prod(Q, kAL, s.A, s.a1, 1, 0);
    add_lin(Q, kAL, s.A1, 1, 0);
    add_prod(Q, kAL, s.A, s.a2, 0, 1);
    add_lin(Q, kAL, s.A2, 0, 1);
    add_prod(Q, kAA, s.A, s.A, 0, 0);
    add_lin(Q, kAA, s.At, 0, 0);
}

// Time integrals over [0, dt] of c1..c8 of Eq. (13) and of t^2 c7, with
// x = dt / tau: closed forms for x >= 1/2, power series where they cancel.
template <typename R>
__device__ __forceinline__ void time_integrals(R dt, R tau, int tau2_exact, R *C)
{
    const R x = dt / tau;
    R t0, t1, t2, c1, c2, c3;   // t_n = int_0^x s^n e^{-s} ds; c* the scaled C1, C2, C3
    if (x >= R(0.5)) {
        const R e = exp(-x);
        t0 = -expm1(-x);
        t1 = t0 - x * e;
        t2 = R(2) * t1 - x * x * e;
        c1 = x - t0;
        c2 = t1 + t0 - x;
        c3 = R(0.5) * x * x - x + t0;
    } else {
        // t_n = sum_k (-1)^k x^{n+k+1} / (k! (n+k+1)); c1 = sum_{p>=2} (-1)^p x^p / p!;
        // c2 = sum_{p>=3} (-1)^p (p-2) x^p / p!;  c3 = sum_{p>=3} (-1)^{p+1} x^p / p!
        t0 = t1 = t2 = c1 = c2 = c3 = R(0);
        R xp = x;                              // x^{k+1} / k!
        R sg = R(1);
#pragma unroll
        for (int k = 0; k < 18; ++k) {         // term k: (-1)^k x^{k+1} / k!
            const R base = sg * xp;            // (-1)^k x^{k+1} / k!
            t0 += base / R(k + 1);
            t1 += base * x / R(k + 2);
            t2 += base * x * x / R(k + 3);
            xp *= x / R(k + 1);
            sg = -sg;
        }
        R pw = x * x / R(2);                   // x^p / p! starting at p = 2
        R s2 = R(1);                           // (-1)^p at p = 2
#pragma unroll
        for (int p = 2; p < 20; ++p) {
            c1 += s2 * pw;
            if (p >= 3) {
                c2 += s2 * R(p - 2) * pw;
                c3 -= s2 * pw;
            }
            pw *= x / R(p + 1);
            s2 = -s2;
        }
    }
    const R tau2 = tau * tau, tau3 = tau2 * tau;
    C[0] = tau * c1;                                   // int c1
    C[1] = tau2 * c2;                                  // int c2
    C[2] = tau2 * c3;                                  // int c3
    C[3] = -tau3 * (t2 + R(2) * t1);                   // int c4 (as printed)
    C[4] = tau3 * (x * x * x / R(3) - x * x);          // int c5 (as printed)
    C[5] = -tau3 * (R(0.5) * x * x + t1);              // int c6 (as printed)
    C[6] = tau * t0;                                   // int c7
    C[7] = -tau2 * t1;                                 // int c8
    C[8] = tau3 * t2;                                  // int t^2 c7
    if (tau2_exact) {
        const R k = R(2) * tau3 * c1;                  // 2 tau^2 int (1 - e^{-t/tau}) dt
        C[3] += k;
        C[4] += k;
        C[5] += k;
    }
}

// Interface data of one Gauss point: primitive left/right states, the
// interface equilibrium W0 = rho_l <psi>_{u>0} + rho_r <psi>_{u<0} with the
// mean of the left/right derivatives, its primitive state, the collision time
// (Eqs. (39)-(40), pressure-jump term scaled by dt) and the time integrals.
template <typename R>
struct Iface {
    KState<R> L, Rs, Z;
    R w0[24];
    R tau;
    R C[9];
};

template <typename R>
__device__ __forceinline__ bool interface_state(const R *wl, const R *wr, R dt, R gamma, R mu, int tau2_exact,
                                                Iface<R> &I)
{
    const R K = R(2) / (gamma - R(1)) - R(2);
    bool ok = prim(wl, gamma, K, I.L) & prim(wr, gamma, K, I.Rs);
    if (!ok) return false;
    {
        R ml[10], mr[10], mvl[10], mvr[10], zl[4], zr[4];
        mom_half(I.L.U, I.L.lam, R(1), ml);
        mom_half(I.Rs.U, I.Rs.lam, R(-1), mr);
        mom_full(I.L.V, I.L.lam, mvl);
        mom_full(I.Rs.V, I.Rs.lam, mvr);
        mom_xi(I.L.lam, K, zl);
        mom_xi(I.Rs.lam, K, zr);
        I.w0[0] = I.L.rho * ml[0] + I.Rs.rho * mr[0];
        I.w0[1] = I.L.rho * ml[1] + I.Rs.rho * mr[1];
        I.w0[2] = I.L.rho * ml[0] * mvl[1] + I.Rs.rho * mr[0] * mvr[1];
        I.w0[3] = I.L.rho * R(0.5) * (ml[2] + ml[0] * mvl[2] + ml[0] * zl[1]) +
                  I.Rs.rho * R(0.5) * (mr[2] + mr[0] * mvr[2] + mr[0] * zr[1]);
#pragma unroll
        for (int q = 4; q < 24; ++q) I.w0[q] = R(0.5) * (wl[q] + wr[q]);
    }
    if (!prim(I.w0, gamma, K, I.Z)) return false;
    const R jump = fabs(I.L.p - I.Rs.p) / fabs(I.L.p + I.Rs.p);
    I.tau = mu > R(0) ? mu / I.Z.p + dt * jump : R(0.01) * dt + dt * jump;
    time_integrals(dt, I.tau, tau2_exact, I.C);
    return true;
}

// Kinetic weighting of the interface derivatives (slope0_mode 1): the
// derivative rows of W0 become the half-space moments of the derivatives of
// the left and right distributions, rho_k <psi g_k'/g_k>_k (u > 0 left, u < 0
// right) with g_n/g = a1.psi, g_t/g = a2.psi, g_nn/g = (a1.psi)^2 + a11.psi,
// g_nt/g = (a1.psi)(a2.psi) + a12.psi, g_tt/g = (a2.psi)^2 + a22.psi: the
// derivatives of the value rho_l <psi>_{u>0} + rho_r <psi>_{u<0} when the two
// states vary as their reconstructions do.  Needs the slopes of I.L and I.Rs.
template <typename R>
__device__ __forceinline__ void kinetic_w0(Iface<R> &I, R K)
{
#pragma unroll
    for (int q = 4; q < 24; ++q) I.w0[q] = R(0);
    Mom<R> m;
    Poly<R> P;
    R out[4];
#pragma unroll
    for (int side = 0; side < 2; ++side) {
        const KState<R> &s = side ? I.Rs : I.L;
        mom_half(s.U, s.lam, side ? R(-1) : R(1), m.u);
        mom_full(s.V, s.lam, m.v);
        mom_xi(s.lam, K, m.z);
        const R *lin[5] = {s.a1, s.a2, s.a11, s.a12, s.a22};
        const R *pa[5] = {nullptr, nullptr, s.a1, s.a1, s.a2}, *pb[5] = {nullptr, nullptr, s.a1, s.a2, s.a2};
#pragma unroll
        for (int r = 0; r < 5; ++r) {
            pzero(P);
            if (r >= 2) add_prod(P, R(1), pa[r], pb[r], 0, 0);
            add_lin(P, R(1), lin[r], 0, 0);
            psi_contract<R, 2>(P, m, out);
#pragma unroll
            for (int q = 0; q < 4; ++q) I.w0[4 + 4 * r + q] += s.rho * out[q];
        }
    }
}

// Flux terms of Eqs. (11) and (15) at y = 0, from the slopes of the three
// states.  with_const = false leaves out the zeroth-order terms C1 g0 and
// C7 g_k (see lead_flux).
//
// HEAT: also d_alpha = <psi_alpha f> (the time-integrated moments without the
// factor u), for the heat flux of the Prandtl correction.
// KIN: interface derivatives by kinetic weighting (kinetic_w0) instead of the
// mean of the left and right rows held in I.w0.
template <typename R, bool HEAT = false, bool KIN = false>
__device__ __forceinline__ void body_flux(const R *wl, const R *wr, Iface<R> &I, R gamma, bool with_const, R *f,
                                          R *d = nullptr)
{
    const R K = R(2) / (gamma - R(1)) - R(2);
    const R tau = I.tau;
    const R *C = I.C;
#pragma unroll
    for (int q = 0; q < 4; ++q) f[q] = R(0);
    R out[4];
    Poly<R> Q;
    Mom<R> m;
    if (KIN) {
        // the left and right slopes first: the interface derivatives are built from them
        mom_full(I.L.U, I.L.lam, m.u);
        mom_full(I.L.V, I.L.lam, m.v);
        mom_xi(I.L.lam, K, m.z);
        slopes(I.L, wl, K, m, false);
        mom_full(I.Rs.U, I.Rs.lam, m.u);
        mom_full(I.Rs.V, I.Rs.lam, m.v);
        mom_xi(I.Rs.lam, K, m.z);
        slopes(I.Rs, wr, K, m, false);
        kinetic_w0(I, K);
    }
    // equilibrium part, Eq. (15)
    mom_full(I.Z.U, I.Z.lam, m.u);
    mom_full(I.Z.V, I.Z.lam, m.v);
    mom_xi(I.Z.lam, K, m.z);
    slopes(I.Z, I.w0, K, m, true);
    build_q(Q, I.Z, with_const ? C[0] : R(0), C[2], C[1], R(0.5) * C[3], C[5], R(0.5) * C[4]);
    upsi_contract(Q, m, out);
#pragma unroll
    for (int q = 0; q < 4; ++q) f[q] += I.Z.rho * out[q];
    if (HEAT) {
        psi_contract<R, 4>(Q, m, out);
#pragma unroll
        for (int q = 0; q < 4; ++q) d[q] = I.Z.rho * out[q];
    }
    // non-equilibrium part, Eq. (11), left (u > 0) and right (u < 0): one copy
    // of the code for both sides (the flux kernels are long enough for
    // instruction fetch to stall them), the side's state and rows copied in
    const R kA = -tau * C[6], kL = C[7] - tau * C[6], kS = R(0.5) * C[8] - tau * C[7], kAL = -tau * C[7];
    const R k7 = with_const ? C[6] : R(0);
#pragma unroll 1
    for (int side = 0; side < 2; ++side) {
        KState<R> st = side ? I.Rs : I.L;
        mom_full(st.U, st.lam, m.u);
        mom_full(st.V, st.lam, m.v);
        mom_xi(st.lam, K, m.z);
        if (!KIN) {
            R rows[24];
#pragma unroll
            for (int q = 0; q < 24; ++q) rows[q] = side ? wr[q] : wl[q];
            slopes(st, rows, K, m, false);
        }
        build_q(Q, st, k7, kA, kL, kS, kAL, R(0));
        mom_half(st.U, st.lam, side ? R(-1) : R(1), m.u);
        upsi_contract(Q, m, out);
#pragma unroll
        for (int q = 0; q < 4; ++q) f[q] += st.rho * out[q];
        if (HEAT) {
            psi_contract<R, 4>(Q, m, out);
#pragma unroll
            for (int q = 0; q < 4; ++q) d[q] += st.rho * out[q];
        }
    }
}

// Heat flux relative to the velocity (U, V) from the flux moments F = <u psi f>
// and the moments D = <psi f>: <(1/2)(u - U)|c|^2 f>, c = (u - U, v - V, xi),
// expanded in the moments u e, u^2, u v, u, e, v, 1.
template <typename R>
__device__ __forceinline__ R heat_flux(const R *F, const R *D, R U, R V)
{
    const R q2 = U * U + V * V;
    return F[3] - U * F[1] - V * F[2] + (R(0.5) * q2 + U * U) * F[0] - U * D[3] + U * V * D[2] -
           R(0.5) * U * q2 * D[0];
}

// Zeroth-order (leading) terms: C1 rho0 <u psi>_0 + C7 (rho_l <u psi>_{u>0,l} +
// rho_r <u psi>_{u<0,r}); all other terms carry a slope and are smaller by a
// factor of order dt |grad W| / |W|.
template <typename R>
__device__ __forceinline__ void lead_flux(const Iface<R> &I, R gamma, R *f)
{
    const R K = R(2) / (gamma - R(1)) - R(2);
    R mu[4], mv[3], mz[2];
    // equilibrium: <u psi> of the full Maxwellian of W0
    {
        const R h = R(0.5) / I.Z.lam;
        mu[0] = R(1); mu[1] = I.Z.U; mu[2] = I.Z.U * mu[1] + h; mu[3] = I.Z.U * mu[2] + R(2) * h * mu[1];
        mv[0] = R(1); mv[1] = I.Z.V; mv[2] = I.Z.V * I.Z.V + h;
        mz[1] = R(0.5) * K / I.Z.lam;
        const R s = I.C[0] * I.Z.rho;
        f[0] = s * mu[1];
        f[1] = s * mu[2];
        f[2] = s * mu[1] * mv[1];
        f[3] = s * R(0.5) * (mu[3] + mu[1] * mv[2] + mu[1] * mz[1]);
    }
    const KState<R> *S[2] = {&I.L, &I.Rs};
#pragma unroll
    for (int side = 0; side < 2; ++side) {
        const KState<R> &k = *S[side];
        R m[10];
        mom_half(k.U, k.lam, side == 0 ? R(1) : R(-1), m);
        const R h = R(0.5) / k.lam;
        const R v2 = k.V * k.V + h, z1 = R(0.5) * K / k.lam;
        const R s = I.C[6] * k.rho;
        f[0] += s * m[1];
        f[1] += s * m[2];
        f[2] += s * m[1] * k.V;
        f[3] += s * R(0.5) * (m[3] + m[1] * v2 + m[1] * z1);
    }
}

// Time-integrated flux through a unit-length face at one Gauss point, all in
// precision R.  wl, wr: [6][4] face-frame rows (value, d/dn, d/dt, d2/dn2,
// d2/dndt, d2/dt2).  Returns false if a state is not physical (f is zero).
// HEAT: Prandtl correction F_E += (1/Pr - 1) q, q the heat flux relative to the
// interface equilibrium velocity (not in the paper; the BGK model has Pr = 1;
// the correction of the BGK-NS scheme, K. Xu, J. Comput. Phys. 171 (2001)).
template <typename R, bool HEAT = false, bool KIN = false>
__device__ __forceinline__ bool gp_flux(const R *wl, const R *wr, R dt, R gamma, R mu, int tau2_exact, R *f,
                                        R prandtl = R(1))
{
    Iface<R> I;
    if (!interface_state(wl, wr, dt, gamma, mu, tau2_exact, I)) {
#pragma unroll
        for (int q = 0; q < 4; ++q) f[q] = R(0);
        return false;
    }
    R d[4];
    body_flux<R, HEAT, KIN>(wl, wr, I, gamma, true, f, d);
    if (HEAT) f[3] += (R(1) / prandtl - R(1)) * heat_flux(f, d, I.Z.U, I.Z.V);
    return true;
}

// Primitive state from the FP64 values with two reciprocals (correctly rounded
// reciprocal instructions times the numerators: within 1.5 ulp, no IEEE
// division); h = 1/(2 lam) comes out of the same quantities.
__device__ __forceinline__ bool prim64(const double *w, double gamma, double K, KState<double> &s, double &h)
{
    s.rho = w[0];
    const double ir = __drcp_rn(w[0]);
    s.U = w[1] * ir;
    s.V = w[2] * ir;
    const double eint = w[3] - 0.5 * s.rho * (s.U * s.U + s.V * s.V);
    s.p = (gamma - 1.0) * eint;
    s.lam = 0.25 * (K + 2.0) * s.rho * __drcp_rn(eint);
    h = 2.0 / (K + 2.0) * eint * ir;                 // (K + 2) rho / (4 eint) = lam
    return s.rho > 0.0 && s.p > 0.0;
}

// Half-space moments <u^k>, k = 0..3, in FP64 (sign = +1: u > 0, -1: u < 0);
// h = 1/(2 lam).
__device__ __forceinline__ void mom_half4(double U, double lam, double h, double sign, double *m)
{
    const double rs = rsqrt(lam);                    // 1/sqrt(lam); sqrt(lam) = lam rs
    m[0] = 0.5 * erfc(-sign * (lam * rs) * U);
    m[1] = U * m[0] + sign * (0.5 / 1.7724538509055160273) * exp(-lam * U * U) * rs;
    m[2] = U * m[1] + h * m[0];
    m[3] = U * m[2] + 2.0 * h * m[1];
}

// FP64 time integrals of c1 and c7 (Eq. (13)) over [0, dt], the coefficients of
// the zeroth-order terms: int c1 = dt - T0, int c7 = T0, T0 = tau (1 - e^{-dt/tau});
// power series where the closed form cancels (x = dt/tau < 1/2).
__device__ __forceinline__ void lead_integrals(double dt, double tau, double &c0, double &c6)
{
    const double x = dt * __drcp_rn(tau);
    double t0, c1;
    if (x >= 0.5) {
        t0 = -expm1(-x);
        c1 = x - t0;
    } else {
        // t0 = sum_{p>=1} (-1)^{p+1} x^p / p!,  c1 = x - t0 = sum_{p>=2} (-1)^p x^p / p!
        double pw = x, sg = 1.0;
        t0 = 0.0;
        c1 = 0.0;
#pragma unroll
        for (int p = 1; p < 20; ++p) {
            t0 += sg * pw;
            if (p >= 2) c1 -= sg * pw;
            pw *= x * (1.0 / double(p + 1));
            sg = -sg;
        }
    }
    c0 = tau * c1;
    c6 = tau * t0;
}

// Mixed precision Gauss-point flux in two parts.  vl, vr: FP64 face-frame
// values (rho, rho U, rho V, E); dl, dr: FP32 face-frame derivative rows [5][4]
// (d/dn, d/dt, d2/dn2, d2/dndt, d2/dt2); K = 2/(gamma - 1) - 2.  The interface
// state W0, the collision time, the time integrals and the zeroth-order terms
// C1 rho0 <u psi>_0 + C7 (rho_l <u psi>_{u>0} + rho_r <u psi>_{u<0}) are FP64
// (gp_lead_mixed); every slope-carrying term is FP32 (gp_body_mixed), formed
// from the FP32 roundings of the FP64 values, W0 and tau.
struct MixedLead {
    double f[4];      // zeroth-order terms of the flux
    double w0[4];     // interface state
    double tau;       // collision time
    double dlead[4];  // HEAT: <psi f> of the zeroth-order terms
    double zu, zv;    // HEAT: interface velocity
};

template <bool HEAT = false>
__device__ __forceinline__ bool gp_lead_mixed(const double *vl, const double *vr, double dt, double gamma, double K,
                                              double mu, MixedLead &o)
{
    KState<double> L, Rs, Z;
    double hl, hr, hz;
    if (!(prim64(vl, gamma, K, L, hl) & prim64(vr, gamma, K, Rs, hr))) return false;
    double ml[4], mr[4];
    mom_half4(L.U, L.lam, hl, 1.0, ml);
    mom_half4(Rs.U, Rs.lam, hr, -1.0, mr);
    const double v2l = L.V * L.V + hl, v2r = Rs.V * Rs.V + hr;
    const double zl = K * hl, zr = K * hr;           // <xi.xi> / 2 = K / (4 lam)
    double *w0 = o.w0;
    w0[0] = L.rho * ml[0] + Rs.rho * mr[0];
    w0[1] = L.rho * ml[1] + Rs.rho * mr[1];
    w0[2] = L.rho * ml[0] * L.V + Rs.rho * mr[0] * Rs.V;
    w0[3] = L.rho * 0.5 * (ml[2] + ml[0] * (v2l + zl)) + Rs.rho * 0.5 * (mr[2] + mr[0] * (v2r + zr));
    if (!prim64(w0, gamma, K, Z, hz)) return false;
    const double jump = fabs(L.p - Rs.p) * __drcp_rn(fabs(L.p + Rs.p));
    o.tau = mu > 0.0 ? mu * __drcp_rn(Z.p) + dt * jump : 0.01 * dt + dt * jump;
    double C0, C6;
    lead_integrals(dt, o.tau, C0, C6);
    double *f = o.f;
    {
        const double m2 = Z.U * Z.U + hz, m3 = Z.U * m2 + 2.0 * hz * Z.U;
        const double v2 = Z.V * Z.V + hz, z1 = K * hz;
        const double s0 = C0 * Z.rho;
        f[0] = s0 * Z.U;
        f[1] = s0 * m2;
        f[2] = s0 * Z.U * Z.V;
        f[3] = s0 * 0.5 * (m3 + Z.U * (v2 + z1));
        const double sl = C6 * L.rho, sr = C6 * Rs.rho;
        f[0] += sl * ml[1] + sr * mr[1];
        f[1] += sl * ml[2] + sr * mr[2];
        f[2] += sl * ml[1] * L.V + sr * mr[1] * Rs.V;
        f[3] += sl * 0.5 * (ml[3] + ml[1] * (v2l + zl)) + sr * 0.5 * (mr[3] + mr[1] * (v2r + zr));
    }
    if constexpr (HEAT) {
        const double sl = C6 * L.rho, sr = C6 * Rs.rho;
        o.dlead[0] = C0 * w0[0] + sl * ml[0] + sr * mr[0];
        o.dlead[1] = C0 * w0[1] + sl * ml[1] + sr * mr[1];
        o.dlead[2] = C0 * w0[2] + sl * ml[0] * L.V + sr * mr[0] * Rs.V;
        o.dlead[3] = C0 * w0[3] + sl * 0.5 * (ml[2] + ml[0] * (v2l + zl)) + sr * 0.5 * (mr[2] + mr[0] * (v2r + zr));
        o.zu = Z.U;
        o.zv = Z.V;
    }
    return true;
}

// The slope-carrying terms in FP32: vl4, vr4, w0f, tauf are the FP32 roundings
// of the FP64 values, interface state and collision time; g the flux part, dg
// (HEAT) its <psi f> part.
template <bool HEAT = false, bool KIN = false>
__device__ __forceinline__ void gp_body_mixed(const float *vl4, const float *vr4, const float *dl, const float *dr,
                                              const float *w0f, float tauf, float dtf, float gf, float Kf,
                                              int tau2_exact, float *g, float *dg)
{
    Iface<float> J;
    float fl[24], fr[24];
#pragma unroll
    for (int q = 0; q < 4; ++q) {
        J.w0[q] = w0f[q];
        fl[q] = vl4[q];
        fr[q] = vr4[q];
    }
#pragma unroll
    for (int q = 0; q < 20; ++q) {
        fl[4 + q] = dl[q];
        fr[4 + q] = dr[q];
        J.w0[4 + q] = 0.5f * (dl[q] + dr[q]);
    }
    prim(fl, gf, Kf, J.L);
    prim(fr, gf, Kf, J.Rs);
    prim(J.w0, gf, Kf, J.Z);
    J.tau = tauf;
    time_integrals(dtf, J.tau, tau2_exact, J.C);
    body_flux<float, HEAT, KIN>(fl, fr, J, gf, false, g, dg);
}

// Both parts at one Gauss point.  Returns false (f zero) if a state is not physical.
template <bool HEAT = false, bool KIN = false>
__device__ __forceinline__ bool gp_flux_mixed_split(const double *vl, const double *vr, const float *dl, const float *dr,
                                                    double dt, double gamma, double K, double mu, int tau2_exact,
                                                    double *f, double prandtl = 1.0)
{
#pragma unroll
    for (int q = 0; q < 4; ++q) f[q] = 0.0;
    MixedLead o;
    if (!gp_lead_mixed<HEAT>(vl, vr, dt, gamma, K, mu, o)) return false;
    float vl4[4], vr4[4], w0f[4], g[4], dg[4];
#pragma unroll
    for (int q = 0; q < 4; ++q) {
        vl4[q] = float(vl[q]);
        vr4[q] = float(vr[q]);
        w0f[q] = float(o.w0[q]);
    }
    gp_body_mixed<HEAT, KIN>(vl4, vr4, dl, dr, w0f, float(o.tau), float(dt), float(gamma), float(K), tau2_exact, g,
                             dg);
#pragma unroll
    for (int q = 0; q < 4; ++q) f[q] = o.f[q] + double(g[q]);
    if (HEAT) {
        double D[4];
#pragma unroll
        for (int q = 0; q < 4; ++q) D[q] = o.dlead[q] + double(dg[q]);
        f[3] += (1.0 / prandtl - 1.0) * heat_flux(f, D, o.zu, o.zv);
    }
    return true;
}

// Mixed precision flux from FP64 rows [6][4] (used by the point-flux entry point).
template <bool HEAT = false, bool KIN = false>
__device__ __forceinline__ bool gp_flux_mixed(const double *wl, const double *wr, double dt, double gamma, double mu,
                                              int tau2_exact, double *f, double prandtl = 1.0)
{
    float dl[20], dr[20];
#pragma unroll
    for (int q = 0; q < 20; ++q) {
        dl[q] = float(wl[4 + q]);
        dr[q] = float(wr[4 + q]);
    }
    return gp_flux_mixed_split<HEAT, KIN>(wl, wr, dl, dr, dt, gamma, 2.0 / (gamma - 1.0) - 2.0, mu, tau2_exact, f,
                                          prandtl);
}

}  // namespace kin
}  // namespace gks
