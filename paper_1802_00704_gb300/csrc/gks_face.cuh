// Device helpers shared by the face-flux translation units: the polynomial
// reconstruction at a Gauss point (Eq. (19)) in FP64 and as FP32 derivative
// rows, the rotation to the face frame, and the ghost states of boundary faces.
#pragma once

#include "gks_internal.h"

namespace gks {
namespace {

constexpr int kFluxBlock = 128;

// Value and derivatives (global frame) of cell c's reconstruction (Eq. (19))
// at the point whose scaled offsets from the centroid are (dx, dy).
// o[6][4]: W, W_x, W_y, W_xx, W_xy, W_yy.
__device__ __forceinline__ void recon(const DeviceMesh &d, const double *__restrict__ w,
                                      const double *__restrict__ x, int c, double dx, double dy, double *o)
{
    const int64_t T = d.T;
    const double ih = 1.0 / d.h[c];
    const double qx = dx * dx - d.mxx[c], qxy = dx * dy - d.mxy[c], qy = dy * dy - d.myy[c];
#pragma unroll
    for (int v = 0; v < 4; ++v) {
        const double u1 = x[(v * 5 + 0) * T + c], u2 = x[(v * 5 + 1) * T + c], u3 = x[(v * 5 + 2) * T + c];
        const double u4 = x[(v * 5 + 3) * T + c], u5 = x[(v * 5 + 4) * T + c];
        o[v] = w[v * T + c] + u1 * dx + u2 * dy + 0.5 * u3 * qx + u4 * qxy + 0.5 * u5 * qy;
        o[4 + v] = (u1 + u3 * dx + u4 * dy) * ih;
        o[8 + v] = (u2 + u4 * dx + u5 * dy) * ih;
        o[12 + v] = u3 * ih * ih;
        o[16 + v] = u4 * ih * ih;
        o[20 + v] = u5 * ih * ih;
    }
}

// Global rows -> face frame (n = (nx, ny), t = (-ny, nx)): directions of the
// derivatives and the momentum components of every row.
__device__ __forceinline__ void to_face(const double *g, double nx, double ny, double *f)
{
    const double tx = -ny, ty = nx;
#pragma unroll
    for (int v = 0; v < 4; ++v) {
        const double gx = g[4 + v], gy = g[8 + v], gxx = g[12 + v], gxy = g[16 + v], gyy = g[20 + v];
        f[v] = g[v];
        f[4 + v] = nx * gx + ny * gy;
        f[8 + v] = tx * gx + ty * gy;
        f[12 + v] = nx * nx * gxx + 2.0 * nx * ny * gxy + ny * ny * gyy;
        f[16 + v] = nx * tx * gxx + (nx * ty + ny * tx) * gxy + ny * ty * gyy;
        f[20 + v] = tx * tx * gxx + 2.0 * tx * ty * gxy + ty * ty * gyy;
    }
#pragma unroll
    for (int r = 0; r < 6; ++r) {
        const double mx = f[4 * r + 1], my = f[4 * r + 2];
        f[4 * r + 1] = nx * mx + ny * my;
        f[4 * r + 2] = tx * mx + ty * my;
    }
}

// Mixed precision reconstruction: FP64 values (recon_val) and FP32 derivative
// rows in the global frame (recon_der, from the FP32 copy of the coefficients;
// fx, fy the FP32 roundings of the scaled offsets dx, dy).
__device__ __forceinline__ void recon_val(const DeviceMesh &d, const double *__restrict__ w,
                                          const double *__restrict__ x, int c, double dx, double dy, double *val)
{
    const int64_t T = d.T;
    const double qx = dx * dx - d.mxx[c], qxy = dx * dy - d.mxy[c], qy = dy * dy - d.myy[c];
#pragma unroll
    for (int v = 0; v < 4; ++v) {
        const double u1 = x[(v * 5 + 0) * T + c], u2 = x[(v * 5 + 1) * T + c], u3 = x[(v * 5 + 2) * T + c];
        const double u4 = x[(v * 5 + 3) * T + c], u5 = x[(v * 5 + 4) * T + c];
        val[v] = w[v * T + c] + u1 * dx + u2 * dy + 0.5 * u3 * qx + u4 * qxy + 0.5 * u5 * qy;
    }
}

__device__ __forceinline__ void recon_der(const DeviceMesh &d, const float *__restrict__ x32, int c, float fx,
                                          float fy, float *der)
{
    const int64_t T = d.T;
    const float ih = d.ih32[c];
#pragma unroll
    for (int v = 0; v < 4; ++v) {
        const float f1 = x32[(v * 5 + 0) * T + c], f2 = x32[(v * 5 + 1) * T + c], f3 = x32[(v * 5 + 2) * T + c];
        const float f4 = x32[(v * 5 + 3) * T + c], f5 = x32[(v * 5 + 4) * T + c];
        der[v] = (f1 + f3 * fx + f4 * fy) * ih;
        der[4 + v] = (f2 + f4 * fx + f5 * fy) * ih;
        der[8 + v] = f3 * ih * ih;
        der[12 + v] = f4 * ih * ih;
        der[16 + v] = f5 * ih * ih;
    }
}

// Face frame (n = (nx, ny), t = (-ny, nx)) of the FP64 values (momentum) ...
__device__ __forceinline__ void to_face_val(double *val, double nx, double ny)
{
    const double mx = val[1], my = val[2];
    val[1] = nx * mx + ny * my;
    val[2] = -ny * mx + nx * my;
}

// ... and of the FP32 derivative rows (directions and momentum); fnx, fny the
// FP32 roundings of the normal
__device__ __forceinline__ void to_face_der(float *der, float fnx, float fny)
{
    const float tx = -fny, ty = fnx;
    float o[20];
#pragma unroll
    for (int v = 0; v < 4; ++v) {
        const float gx = der[v], gy = der[4 + v], gxx = der[8 + v], gxy = der[12 + v], gyy = der[16 + v];
        o[v] = fnx * gx + fny * gy;
        o[4 + v] = tx * gx + ty * gy;
        o[8 + v] = fnx * fnx * gxx + 2.0f * fnx * fny * gxy + fny * fny * gyy;
        o[12 + v] = fnx * tx * gxx + (fnx * ty + fny * tx) * gxy + fny * ty * gyy;
        o[16 + v] = tx * tx * gxx + 2.0f * tx * ty * gxy + ty * ty * gyy;
    }
#pragma unroll
    for (int r = 0; r < 5; ++r) {
        const float a = o[4 * r + 1], b = o[4 * r + 2];
        der[4 * r + 0] = o[4 * r + 0];
        der[4 * r + 1] = fnx * a + fny * b;
        der[4 * r + 2] = tx * a + ty * b;
        der[4 * r + 3] = o[4 * r + 3];
    }
}

// Isothermal no-slip wall as the mirror image of the primitive fields:
// pressure even in the normal coordinate n, velocity odd about the wall
// velocity, temperature T = p / rho odd about the wall temperature.  Fields with
// that symmetry (a linear shear, a linear temperature profile at uniform
// pressure) continue across the wall unchanged, so the kinetic flux through the
// wall carries their viscous stress and Fourier conduction.
//
// A field near the Gauss point is a second-order jet j[6] in the face frame
// (value, d/dn, d/dt, d2/dn2, d2/dndt, d2/dt2: the entries of one variable in
// the face-frame rows).  q = a / b is formed by the recursive quotient rule
// b q = a differentiated term by term.
template <typename R>
__device__ __forceinline__ void jet_quot(const R *a, const R *b, R *q)
{
    const R ib = R(1) / b[0];
    q[0] = a[0] * ib;
    q[1] = (a[1] - q[0] * b[1]) * ib;
    q[2] = (a[2] - q[0] * b[2]) * ib;
    q[3] = (a[3] - R(2) * q[1] * b[1] - q[0] * b[3]) * ib;
    q[4] = (a[4] - q[1] * b[2] - q[2] * b[1] - q[0] * b[4]) * ib;
    q[5] = (a[5] - R(2) * q[2] * b[2] - q[0] * b[5]) * ib;
}

template <typename R>
__device__ __forceinline__ void jet_prod(const R *a, const R *b, R *c)
{
    c[0] = a[0] * b[0];
    c[1] = a[1] * b[0] + a[0] * b[1];
    c[2] = a[2] * b[0] + a[0] * b[2];
    c[3] = a[3] * b[0] + R(2) * a[1] * b[1] + a[0] * b[3];
    c[4] = a[4] * b[0] + a[1] * b[2] + a[2] * b[1] + a[0] * b[4];
    c[5] = a[5] * b[0] + R(2) * a[2] * b[2] + a[0] * b[5];
}

// Ghost state of the no-slip wall.  v0: the interior values (rho, rho u_n,
// rho u_t, E), der: its five face-frame derivative rows (entry (r, v) of row
// r = d/dn .. d2/dt2 at der[4 r + v]); uwn, uwt the wall velocity along n and
// t, tw the wall temperature.  Out: the ghost values vg (skipped if NULL) and
// derivative rows dg, same layouts.
template <typename R>
__device__ __forceinline__ void noslip_jets(const R *v0, const R *der, R uwn, R uwt, R tw, R gamma, R *vg, R *dg)
{
    // interior jets: entry 0 from v0, entries 1..5 from the derivative rows der[4 (r - 1) + v]
    R rho[6], mn[6], mt[6], en[6];
    rho[0] = v0[0];
    mn[0] = v0[1];
    mt[0] = v0[2];
    en[0] = v0[3];
#pragma unroll
    for (int r = 1; r < 6; ++r) {
        rho[r] = der[4 * (r - 1) + 0];
        mn[r] = der[4 * (r - 1) + 1];
        mt[r] = der[4 * (r - 1) + 2];
        en[r] = der[4 * (r - 1) + 3];
    }
    R un[6], ut[6], kin[6], a[6], b[6], p[6], T[6];
    jet_quot(mn, rho, un);
    jet_quot(mt, rho, ut);
    jet_prod(mn, un, a);
    jet_prod(mt, ut, b);
#pragma unroll
    for (int r = 0; r < 6; ++r) p[r] = (gamma - R(1)) * (en[r] - R(0.5) * (a[r] + b[r]));
    jet_quot(p, rho, T);
    // mirror image: an entry of order k in n gets (-1)^k (pressure), the
    // reflection about a wall value c negates that: 2 c - q, (-1)^{k+1} d^k q
    const R ev[6] = {R(1), R(-1), R(1), R(1), R(-1), R(1)};
    R pg[6], ung[6], utg[6], Tg[6];
#pragma unroll
    for (int r = 0; r < 6; ++r) {
        pg[r] = ev[r] * p[r];
        ung[r] = -ev[r] * un[r];
        utg[r] = -ev[r] * ut[r];
        Tg[r] = -ev[r] * T[r];
    }
    ung[0] += R(2) * uwn;
    utg[0] += R(2) * uwt;
    Tg[0] += R(2) * tw;
    R rg[6], mng[6], mtg[6];
    jet_quot(pg, Tg, rg);
    jet_prod(rg, ung, mng);
    jet_prod(rg, utg, mtg);
    jet_prod(mng, ung, a);
    jet_prod(mtg, utg, b);
    const R ig = R(1) / (gamma - R(1));
    if (vg) {
        vg[0] = rg[0];
        vg[1] = mng[0];
        vg[2] = mtg[0];
        vg[3] = pg[0] * ig + R(0.5) * (a[0] + b[0]);
    }
#pragma unroll
    for (int r = 1; r < 6; ++r) {
        dg[4 * (r - 1) + 0] = rg[r];
        dg[4 * (r - 1) + 1] = mng[r];
        dg[4 * (r - 1) + 2] = mtg[r];
        dg[4 * (r - 1) + 3] = pg[r] * ig + R(0.5) * (a[r] + b[r]);
    }
}

// Ghost state of a boundary face, FP64 values (face frame) ...
__device__ __forceinline__ void ghost_val(int tag, const double *bc, double nx, double ny, double gamma,
                                          const double *vl, double *vr)
{
    if (tag == GKS_BC_DIRICHLET) {
        vr[0] = bc[0];
        vr[1] = nx * bc[1] + ny * bc[2];
        vr[2] = -ny * bc[1] + nx * bc[2];
        vr[3] = bc[3];
        return;
    }
    if (tag == GKS_BC_OUTFLOW) {
#pragma unroll
        for (int q = 0; q < 4; ++q) vr[q] = vl[q];
        return;
    }
    if (tag == GKS_BC_NOSLIP) {
        // same pressure, velocity 2 u_w - u, temperature 2 T_w - T
        const double rho = vl[0], un = vl[1] / rho, ut = vl[2] / rho;
        const double p = (gamma - 1.0) * (vl[3] - 0.5 * rho * (un * un + ut * ut));
        const double uwn = nx * bc[0] + ny * bc[1], uwt = -ny * bc[0] + nx * bc[1];
        const double tg = 2.0 * bc[2] - p / rho;
        const double gn = 2.0 * uwn - un, gt = 2.0 * uwt - ut;
        const double rg = p / tg;
        vr[0] = rg;
        vr[1] = rg * gn;
        vr[2] = rg * gt;
        vr[3] = p / (gamma - 1.0) + 0.5 * rg * (gn * gn + gt * gt);
    } else {
        vr[0] = vl[0];
        vr[1] = -vl[1];
        vr[2] = vl[2];
        vr[3] = vl[3];
    }
}

// ... and FP32 derivative rows: zero (Dirichlet), copied (outflow), the mirror
// image with (-1)^p for a derivative of order p in n (slip wall), or the
// derivatives of the reflected primitive fields (no-slip wall; vl the FP32
// roundings of the interior values, face frame)
__device__ __forceinline__ void ghost_der(int tag, const double *bc, float fnx, float fny, float gamma,
                                          const float *vl, const float *dl, float *dr)
{
    if (tag == GKS_BC_DIRICHLET || tag == GKS_BC_OUTFLOW) {
#pragma unroll
        for (int q = 0; q < 20; ++q) dr[q] = tag == GKS_BC_OUTFLOW ? dl[q] : 0.0f;
        return;
    }
    if (tag == GKS_BC_NOSLIP) {
        const float bx = float(bc[0]), by = float(bc[1]);
        noslip_jets<float>(vl, dl, fnx * bx + fny * by, -fny * bx + fnx * by, float(bc[2]), gamma, nullptr, dr);
        return;
    }
    const int npar[5] = {1, 0, 0, 1, 0};   // parity of the n-order of rows d/dn .. d2/dt2
#pragma unroll
    for (int r = 0; r < 5; ++r)
#pragma unroll
        for (int v = 0; v < 4; ++v) {
            float sg = v == 1 ? -1.0f : 1.0f;
            if (npar[r]) sg = -sg;
            dr[4 * r + v] = sg * dl[4 * r + v];
        }
}

// Ghost right state of a boundary face (face frame).
__device__ __forceinline__ void ghost(int tag, const double *bc, double nx, double ny, double gamma,
                                      const double *wl, double *wr)
{
    if (tag == GKS_BC_DIRICHLET) {
#pragma unroll
        for (int q = 0; q < 24; ++q) wr[q] = 0.0;
        wr[0] = bc[0];
        wr[1] = nx * bc[1] + ny * bc[2];
        wr[2] = -ny * bc[1] + nx * bc[2];
        wr[3] = bc[3];
        return;
    }
    if (tag == GKS_BC_OUTFLOW) {
#pragma unroll
        for (int q = 0; q < 24; ++q) wr[q] = wl[q];
        return;
    }
    if (tag == GKS_BC_NOSLIP) {
        noslip_jets<double>(wl, wl + 4, nx * bc[0] + ny * bc[1], -ny * bc[0] + nx * bc[1], bc[2], gamma, wr, wr + 4);
        return;
    }
    // slip wall, mirror image: q_R(n, t) = s_q q_L(-n, t); a derivative of order p in n gets (-1)^p
    const int npar[6] = {0, 1, 0, 0, 1, 0};   // parity of the n-order of each row
#pragma unroll
    for (int r = 0; r < 6; ++r)
#pragma unroll
        for (int v = 0; v < 4; ++v) {
            double s = v == 1 ? -1.0 : 1.0;
            if (npar[r]) s = -s;
            wr[4 * r + v] = s * wl[4 * r + v];
        }
}

}  // namespace
}  // namespace gks
