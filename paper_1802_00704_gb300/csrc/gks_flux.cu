// Face fluxes (Eqs. (7), (11), (15)): reconstruction at the Gauss points,
// ghost states, and the kinetic flux; one thread per face Gauss point, the two
// points of a face in neighbouring lanes summed with one shuffle, so each face
// flux is written once, without atomics.
#include <algorithm>
#include <cfloat>

#include <type_traits>

#include "gks_internal.h"
#include "gks_kinetic.cuh"
#include "gks_lead_df.cuh"

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

// y = float(x), n values
__global__ void k_to_f32(const double *__restrict__ x, float *__restrict__ y, int64_t n)
{
    const int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (i < n) y[i] = float(x[i]);
}

// ---- double-FP32 mixed flux (flux_lead = 1)

using dfm::df;

// Gauss-point values of cell c's reconstruction (Eq. (19)) in double-FP32:
// w + sum_k u_k phi_k with the basis values phi = (dx, dy, (dx^2 - <dx^2>)/2,
// dx dy - <dx dy>, (dy^2 - <dy^2>)/2) at the scaled offsets (dx, dy).
__device__ __forceinline__ void recon_val_df(const DeviceMesh &d, const float *__restrict__ w2,
                                             const float *__restrict__ x2, int c, df dx, df dy, df *val)
{
    const int64_t T = d.T;
    const df mxx = {d.m2[c], d.m2[3 * T + c]}, mxy = {d.m2[T + c], d.m2[4 * T + c]};
    const df myy = {d.m2[2 * T + c], d.m2[5 * T + c]};
    const df phi[5] = {dx, dy, dfm::scale2(dfm::sub(dfm::mul(dx, dx), mxx), 0.5f), dfm::sub(dfm::mul(dx, dy), mxy),
                       dfm::scale2(dfm::sub(dfm::mul(dy, dy), myy), 0.5f)};
#pragma unroll
    for (int v = 0; v < 4; ++v) {
        dfm::Acc a = dfm::acc_start(df{w2[v * T + c], w2[(4 + v) * T + c]});
#pragma unroll
        for (int q = 0; q < 5; ++q)
            dfm::acc_prod(a, df{x2[(v * 5 + q) * T + c], x2[(20 + v * 5 + q) * T + c]}, phi[q]);
        val[v] = dfm::acc_end(a);
    }
}

// momentum of the values to the face frame (n, t = (-ny, nx))
__device__ __forceinline__ void to_face_val_df(df *val, df nx, df ny)
{
    const df mx = val[1], my = val[2];
    val[1] = dfm::add(dfm::mul(nx, mx), dfm::mul(ny, my));
    val[2] = dfm::sub(dfm::mul(nx, my), dfm::mul(ny, mx));
}

// Ghost values of a boundary face in pairs (face frame): the rules of ghost_val.
__device__ __forceinline__ void ghost_val_df(int tag, const double *bc, df nx, df ny, const lead::LeadConst &c,
                                             const df *vl, df *vr)
{
    if (tag == GKS_BC_DIRICHLET) {
        const df b1 = dfm::split_double(bc[1]), b2 = dfm::split_double(bc[2]);
        vr[0] = dfm::split_double(bc[0]);
        vr[1] = dfm::add(dfm::mul(nx, b1), dfm::mul(ny, b2));
        vr[2] = dfm::sub(dfm::mul(nx, b2), dfm::mul(ny, b1));
        vr[3] = dfm::split_double(bc[3]);
        return;
    }
    if (tag == GKS_BC_OUTFLOW) {
#pragma unroll
        for (int q = 0; q < 4; ++q) vr[q] = vl[q];
        return;
    }
    if (tag == GKS_BC_NOSLIP) {
        // same pressure, velocity 2 u_w - u, temperature 2 T_w - T
        const df ir = dfm::recip(vl[0]);
        const df un = dfm::mul(vl[1], ir), ut = dfm::mul(vl[2], ir);
        const df ke = dfm::scale2(dfm::add(dfm::mul(vl[1], un), dfm::mul(vl[2], ut)), 0.5f);
        const df p = dfm::mul(dfm::sub(vl[3], ke), c.gm1);
        const df bx = dfm::split_double(bc[0]), by = dfm::split_double(bc[1]);
        const df uwn = dfm::add(dfm::mul(nx, bx), dfm::mul(ny, by));
        const df uwt = dfm::sub(dfm::mul(nx, by), dfm::mul(ny, bx));
        const df tg = dfm::sub(dfm::scale2(dfm::split_double(bc[2]), 2.0f), dfm::mul(p, ir));
        const df gn = dfm::sub(dfm::scale2(uwn, 2.0f), un), gt = dfm::sub(dfm::scale2(uwt, 2.0f), ut);
        const df rg = dfm::div(p, tg);
        vr[0] = rg;
        vr[1] = dfm::mul(rg, gn);
        vr[2] = dfm::mul(rg, gt);
        vr[3] = dfm::add(dfm::mul(p, c.igm1),
                         dfm::scale2(dfm::mul(rg, dfm::add(dfm::mul(gn, gn), dfm::mul(gt, gt))), 0.5f));
        return;
    }
    vr[0] = vl[0];
    vr[1] = dfm::neg(vl[1]);
    vr[2] = vl[2];
    vr[3] = vl[3];
}

// y = (hi, lo) pairs of x: w2 [8][T] from w [4][T], x2 [40][T] from x [20][T]
// (high parts of all rows first), by integer operations
__global__ void k_to_df(const double *__restrict__ w, const double *__restrict__ x, float *__restrict__ w2,
                        float *__restrict__ x2, int64_t T)
{
    const int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (i >= T) return;
#pragma unroll
    for (int v = 0; v < 4; ++v) {
        const df p = dfm::split_double(w[v * T + i]);
        w2[v * T + i] = p.hi;
        w2[(4 + v) * T + i] = p.lo;
    }
#pragma unroll 4
    for (int q = 0; q < 20; ++q) {
        const df p = dfm::split_double(x[q * T + i]);
        x2[q * T + i] = p.hi;
        x2[(20 + q) * T + i] = p.lo;
    }
}

// Mixed flux, one thread per Gauss point: values, interface state, collision
// time and zeroth-order terms in double-FP32 (gks_lead_df.cuh), slope-carrying
// terms in FP32 (kin::gp_body_mixed), both on the FP32 pipe; the two points of
// a face in neighbouring lanes, summed in pairs and written once in FP64.
// HEAT: Prandtl correction (pr_fac = 1/Pr - 1); KIN: kinetic interface slopes.
template <bool HEAT, bool KIN>
__global__ void __launch_bounds__(kFluxBlock, 4)
    k_face_flux_df(DeviceMesh d, const float *__restrict__ w2, const float *__restrict__ x2, double dt_const,
                   const double *__restrict__ dt_dev, lead::LeadConst lc, float gamma_f, float K_f, int tau2,
                   df pr_fac, double *__restrict__ flux, int32_t *status)
{
    const int64_t F = d.F;
    const int64_t g = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    const int64_t f = g >> 1;
    const int k = (int)(g & 1);
    const int cs = f < F ? d.face_case[f] : 0;
    const double dt = f < F ? (dt_dev ? dt_dev[cs] : dt_const) : 0.0;
    const bool valid = f < F && dt > 0.0;       // cases with dt = 0 are not advanced
    df out[4] = {{0.0f, 0.0f}, {0.0f, 0.0f}, {0.0f, 0.0f}, {0.0f, 0.0f}};
    if (valid) {
        const df dtd = dfm::split_double(dt);
        const df nx = {d.fn2[f], d.fn2[2 * F + f]}, ny = {d.fn2[F + f], d.fn2[3 * F + f]};
        const int l = d.fl[f], r = d.fr[f];
        df vl[4], vr[4];
        float dl[20], dr[20];
        {
            const df lx = {d.gl2[(2 * k) * F + f], d.gl2[(4 + 2 * k) * F + f]};
            const df ly = {d.gl2[(2 * k + 1) * F + f], d.gl2[(5 + 2 * k) * F + f]};
            recon_val_df(d, w2, x2, l, lx, ly, vl);
            recon_der(d, x2, l, lx.hi, ly.hi, dl);
        }
        to_face_val_df(vl, nx, ny);
        to_face_der(dl, nx.hi, ny.hi);
        if (r >= 0) {
            const df rx = {d.gr2[(2 * k) * F + f], d.gr2[(4 + 2 * k) * F + f]};
            const df ry = {d.gr2[(2 * k + 1) * F + f], d.gr2[(5 + 2 * k) * F + f]};
            recon_val_df(d, w2, x2, r, rx, ry, vr);
            recon_der(d, x2, r, rx.hi, ry.hi, dr);
            to_face_val_df(vr, nx, ny);
            to_face_der(dr, nx.hi, ny.hi);
        } else {
            const double bc[4] = {d.bc[f], d.bc[F + f], d.bc[2 * F + f], d.bc[3 * F + f]};
            const float vlf[4] = {vl[0].hi, vl[1].hi, vl[2].hi, vl[3].hi};
            ghost_val_df(d.ftag[f], bc, nx, ny, lc, vl, vr);
            ghost_der(d.ftag[f], bc, nx.hi, ny.hi, gamma_f, vlf, dl, dr);
        }
        lead::Lead o;
        if (lead::gp_lead(vl, vr, dtd, lc, o)) {
            float vl4[4], vr4[4], w0f[4], gq[4], dg[4];
#pragma unroll
            for (int q = 0; q < 4; ++q) {
                vl4[q] = vl[q].hi;
                vr4[q] = vr[q].hi;
                w0f[q] = o.w0[q].hi;
            }
            kin::gp_body_mixed<HEAT, KIN>(vl4, vr4, dl, dr, w0f, o.tau.hi, dtd.hi, gamma_f, K_f, tau2, gq, dg);
            df fk[4];
#pragma unroll
            for (int q = 0; q < 4; ++q) fk[q] = dfm::add(o.f[q], gq[q]);
            if (HEAT) {
                df D[4];
#pragma unroll
                for (int q = 0; q < 4; ++q) D[q] = dfm::add(dfm::mul(o.c0c6, o.w0[q]), dg[q]);
                fk[3] = dfm::add(fk[3], dfm::mul(pr_fac, lead::heat_flux(fk, D, o.zu, o.zv)));
            }
            const df s = {d.flen2[f], d.flen2[F + f]};      // Gauss weight 1/2 times the face length
            out[0] = dfm::mul(s, fk[0]);
            out[1] = dfm::mul(s, dfm::sub(dfm::mul(nx, fk[1]), dfm::mul(ny, fk[2])));
            out[2] = dfm::mul(s, dfm::add(dfm::mul(ny, fk[1]), dfm::mul(nx, fk[2])));
            out[3] = dfm::mul(s, fk[3]);
        } else {
            atomicOr(&status[cs], kStatusNonPhys);
        }
    }
#pragma unroll
    for (int q = 0; q < 4; ++q) {
        const df o2 = {__shfl_xor_sync(0xffffffffu, out[q].hi, 1), __shfl_xor_sync(0xffffffffu, out[q].lo, 1)};
        out[q] = dfm::add(out[q], o2);
    }
    if (f < F && k == 0)
#pragma unroll
        for (int q = 0; q < 4; ++q) flux[q * F + f] = dfm::to_double(out[q]);
}

// MIXED: interface state and leading terms in FP64, slope-carrying terms in FP32.
// HEAT: Prandtl correction of the energy flux (prandtl != 1).
// KIN: interface derivatives by kinetic weighting (slope0_mode 1).
template <bool MIXED, bool HEAT, bool KIN>
__global__ void __launch_bounds__(kFluxBlock, MIXED ? 4 : 1) k_face_flux(DeviceMesh d, const double *__restrict__ w,
                                                          const double *__restrict__ x,
                                                          const float *__restrict__ x32, double dt_const,
                                                          const double *__restrict__ dt_dev, double gamma, double K,
                                                          double mu, int tau2, double prandtl,
                                                          double *__restrict__ flux, int32_t *status)
{
    const int64_t F = d.F;
    const int64_t g = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    const int64_t f = g >> 1;
    const int k = (int)(g & 1);
    const int cs = f < F ? d.face_case[f] : 0;
    const double dt = f < F ? (dt_dev ? dt_dev[cs] : dt_const) : 0.0;
    const bool valid = f < F && dt > 0.0;       // cases with dt = 0 are not advanced
    double out[4] = {0.0, 0.0, 0.0, 0.0};
    if (valid) {
        const double nx = d.fnx[f], ny = d.fny[f];
        const int l = d.fl[f], r = d.fr[f];
        double fk[4];
        bool ok;
        if (MIXED) {
            double vl[4], vr[4];
            float dl[20], dr[20];
            const float fnx = float(nx), fny = float(ny);
            const double lx = d.gl[(2 * k) * F + f], ly = d.gl[(2 * k + 1) * F + f];
            recon_val(d, w, x, l, lx, ly, vl);
            recon_der(d, x32, l, float(lx), float(ly), dl);
            to_face_val(vl, nx, ny);
            to_face_der(dl, fnx, fny);
            if (r >= 0) {
                const double rx = d.gr[(2 * k) * F + f], ry = d.gr[(2 * k + 1) * F + f];
                recon_val(d, w, x, r, rx, ry, vr);
                recon_der(d, x32, r, float(rx), float(ry), dr);
                to_face_val(vr, nx, ny);
                to_face_der(dr, fnx, fny);
            } else {
                const double bc[4] = {d.bc[f], d.bc[F + f], d.bc[2 * F + f], d.bc[3 * F + f]};
                ghost_val(d.ftag[f], bc, nx, ny, gamma, vl, vr);
                const float vlf[4] = {float(vl[0]), float(vl[1]), float(vl[2]), float(vl[3])};
                ghost_der(d.ftag[f], bc, fnx, fny, float(gamma), vlf, dl, dr);
            }
            ok = kin::gp_flux_mixed_split<HEAT, KIN>(vl, vr, dl, dr, dt, gamma, K, mu, tau2, fk, prandtl);
        } else {
            double gl[24], wl[24], wr[24];
            recon(d, w, x, l, d.gl[(2 * k) * F + f], d.gl[(2 * k + 1) * F + f], gl);
            to_face(gl, nx, ny, wl);
            if (r >= 0) {
                recon(d, w, x, r, d.gr[(2 * k) * F + f], d.gr[(2 * k + 1) * F + f], gl);
                to_face(gl, nx, ny, wr);
            } else {
                const double bc[4] = {d.bc[f], d.bc[F + f], d.bc[2 * F + f], d.bc[3 * F + f]};
                ghost(d.ftag[f], bc, nx, ny, gamma, wl, wr);
            }
            ok = kin::gp_flux<double, HEAT, KIN>(wl, wr, dt, gamma, mu, tau2, fk, prandtl);
        }
        if (!ok) atomicOr(&status[cs], kStatusNonPhys);
        const double s = 0.5 * d.flen[f];      // Gauss weight 1/2 times the face length
        out[0] = s * fk[0];
        out[1] = s * (nx * fk[1] - ny * fk[2]);
        out[2] = s * (ny * fk[1] + nx * fk[2]);
        out[3] = s * fk[3];
    }
#pragma unroll
    for (int q = 0; q < 4; ++q) out[q] += __shfl_xor_sync(0xffffffffu, out[q], 1);
    if (f < F && k == 0)
#pragma unroll
        for (int q = 0; q < 4; ++q) flux[q * F + f] = out[q];
}

// Warp-specialised mixed flux (flux_split, without the Prandtl correction).
// GB300 runs FP64 at 1/64 of the FP32 rate, so the flux is bound by the FP64
// pipe; in k_face_flux every warp alternates an FP64 phase and a longer FP32
// phase and the pipe idles whenever all warps of a scheduler are in the latter.
// Here each block is persistent and splits its NW warps: NL lead warps form the
// FP64 values, the interface state, the collision time and the zeroth-order
// terms of a tile of 32 NL Gauss points and publish them in shared memory; the
// other warps (body) take the published values of each point, reconstruct its
// FP32 derivative rows, add the slope-carrying terms and write the face fluxes
// (NL / (NW - NL) points per body thread).  Two buffers: the lead warps run up
// to two tiles ahead.  The hand-over uses hardware named barriers (bar.arrive
// by the producer, bar.sync by the consumer; ids 1-2 full, 3-4 empty); both
// roles walk the same tile sequence, so every barrier phase gets its 32 NW
// arrivals.  Same arithmetic as k_face_flux<true, false, KIN>; the fluxes agree
// to rounding (the compiler may contract multiply-adds differently in the two
// kernels).  Measured on GB300 (1,000,000 triangles, one launch): 5 lead + 5
// body warps, two blocks per SM (96 registers) 2.67 ms; 4 + 4 (128 registers)
// 2.72 ms; 4 + 4 at three blocks per SM 2.72 ms; 8 + 4 2.70 ms; 6 + 6 2.75 ms;
// 6 + 2 3.36 ms (the two FP32 warps fall behind); k_face_flux 2.83 ms.
constexpr int kWsLead = 5, kWsWarps = 10, kWsMinBlocks = 2;

template <int TILE>
struct WsBuf {
    double lead[4][TILE];                     // zeroth-order flux terms (FP64)
    float vl[4][TILE], vr[4][TILE];           // FP32 roundings of the face-frame values
    float w0[4][TILE];                        // ... of the interface state
    float tau[TILE];                          // ... of the collision time
    int ok[TILE];                             // states physical
};

__device__ __forceinline__ void bar_sync_named(int id, int nthreads)
{
    asm volatile("bar.sync %0, %1;" ::"r"(id), "r"(nthreads) : "memory");
}

__device__ __forceinline__ void bar_arrive_named(int id, int nthreads)
{
    asm volatile("bar.arrive %0, %1;" ::"r"(id), "r"(nthreads) : "memory");
}

// NL lead warps of NW, MINB blocks per SM (the register budget)
template <bool KIN, int NL, int NW, int MINB>
__global__ void __launch_bounds__(32 * NW, MINB) k_face_flux_ws(DeviceMesh d, const double *__restrict__ w,
                                                                const double *__restrict__ x,
                                                                const float *__restrict__ x32, double dt_const,
                                                                const double *__restrict__ dt_dev, double gamma,
                                                                double K, double mu, int tau2,
                                                                double *__restrict__ flux, int32_t *status)
{
    constexpr int NT = 32 * NW, TILE = 32 * NL, NBT = NT - TILE, PER = TILE / NBT;
    static_assert(NL > 0 && NL < NW && TILE % NBT == 0, "lead warps must divide the tile evenly");
    __shared__ WsBuf<TILE> buf[2];
    const int64_t F = d.F;
    const int64_t ntiles = (2 * F + TILE - 1) / TILE;
    const bool lead = threadIdx.x < TILE;                // warp-uniform
    int n = 0;
    for (int64_t tile = blockIdx.x; tile < ntiles; tile += gridDim.x, ++n) {
        const int b = n & 1;
        WsBuf<TILE> &B = buf[b];
        if (lead) {
            const int p = threadIdx.x;
            const int64_t g = tile * TILE + p;
            const int64_t f = g >> 1;
            const int k = (int)(g & 1);
            const int cs = f < F ? d.face_case[f] : 0;
            const double dt = f < F ? (dt_dev ? dt_dev[cs] : dt_const) : 0.0;
            const bool valid = f < F && dt > 0.0;
            if (n >= 2) bar_sync_named(3 + b, NT);       // the body warps are done with buffer b
            double lf[4] = {0.0, 0.0, 0.0, 0.0};
            float vl4[4] = {0.0f, 0.0f, 0.0f, 0.0f}, vr4[4] = {0.0f, 0.0f, 0.0f, 0.0f};
            float w0f[4] = {0.0f, 0.0f, 0.0f, 0.0f}, tauf = 0.0f;
            int ok = 1;
            if (valid) {
                const double nx = d.fnx[f], ny = d.fny[f];
                const int l = d.fl[f], r = d.fr[f];
                double vl[4], vr[4];
                recon_val(d, w, x, l, d.gl[(2 * k) * F + f], d.gl[(2 * k + 1) * F + f], vl);
                to_face_val(vl, nx, ny);
                if (r >= 0) {
                    recon_val(d, w, x, r, d.gr[(2 * k) * F + f], d.gr[(2 * k + 1) * F + f], vr);
                    to_face_val(vr, nx, ny);
                } else {
                    const double bc[4] = {d.bc[f], d.bc[F + f], d.bc[2 * F + f], d.bc[3 * F + f]};
                    ghost_val(d.ftag[f], bc, nx, ny, gamma, vl, vr);
                }
                kin::MixedLead o;
                ok = kin::gp_lead_mixed<false>(vl, vr, dt, gamma, K, mu, o) ? 1 : 0;
                if (ok) {
#pragma unroll
                    for (int q = 0; q < 4; ++q) {
                        lf[q] = o.f[q];
                        vl4[q] = float(vl[q]);
                        vr4[q] = float(vr[q]);
                        w0f[q] = float(o.w0[q]);
                    }
                    tauf = float(o.tau);
                } else {
                    atomicOr(&status[cs], kStatusNonPhys);
                }
            }
#pragma unroll
            for (int q = 0; q < 4; ++q) {
                B.lead[q][p] = lf[q];
                B.vl[q][p] = vl4[q];
                B.vr[q][p] = vr4[q];
                B.w0[q][p] = w0f[q];
            }
            B.tau[p] = tauf;
            B.ok[p] = ok;
            bar_arrive_named(1 + b, NT);
        } else {
            bar_sync_named(1 + b, NT);                   // the lead warps' values of this tile
            for (int j = 0; j < PER; ++j) {
                // consecutive lanes take consecutive points: the two points of a face share a warp
                const int p = j * NBT + (threadIdx.x - TILE);
                const int64_t g = tile * TILE + p;
                const int64_t f = g >> 1;
                const int k = (int)(g & 1);
                const int cs = f < F ? d.face_case[f] : 0;
                const double dt = f < F ? (dt_dev ? dt_dev[cs] : dt_const) : 0.0;
                const bool valid = f < F && dt > 0.0;
                double out[4] = {0.0, 0.0, 0.0, 0.0};
                if (valid) {
                    const double nx = d.fnx[f], ny = d.fny[f];
                    double fk[4] = {0.0, 0.0, 0.0, 0.0};
                    if (B.ok[p]) {
                        const int l = d.fl[f], r = d.fr[f];
                        const float fnx = float(nx), fny = float(ny);
                        float dl[20], dr[20];
                        recon_der(d, x32, l, float(d.gl[(2 * k) * F + f]), float(d.gl[(2 * k + 1) * F + f]), dl);
                        to_face_der(dl, fnx, fny);
                        if (r >= 0) {
                            recon_der(d, x32, r, float(d.gr[(2 * k) * F + f]), float(d.gr[(2 * k + 1) * F + f]),
                                      dr);
                            to_face_der(dr, fnx, fny);
                        } else {
                            const double bc[4] = {d.bc[f], d.bc[F + f], d.bc[2 * F + f], d.bc[3 * F + f]};
                            const float vlf[4] = {B.vl[0][p], B.vl[1][p], B.vl[2][p], B.vl[3][p]};
                            ghost_der(d.ftag[f], bc, fnx, fny, float(gamma), vlf, dl, dr);
                        }
                        float vl4[4], vr4[4], w0f[4], gq[4], dg[4];
#pragma unroll
                        for (int q = 0; q < 4; ++q) {
                            vl4[q] = B.vl[q][p];
                            vr4[q] = B.vr[q][p];
                            w0f[q] = B.w0[q][p];
                        }
                        kin::gp_body_mixed<false, KIN>(vl4, vr4, dl, dr, w0f, B.tau[p], float(dt), float(gamma),
                                                       float(K), tau2, gq, dg);
#pragma unroll
                        for (int q = 0; q < 4; ++q) fk[q] = B.lead[q][p] + double(gq[q]);
                    }
                    const double s = 0.5 * d.flen[f];    // Gauss weight 1/2 times the face length
                    out[0] = s * fk[0];
                    out[1] = s * (nx * fk[1] - ny * fk[2]);
                    out[2] = s * (ny * fk[1] + nx * fk[2]);
                    out[3] = s * fk[3];
                }
#pragma unroll
                for (int q = 0; q < 4; ++q) out[q] += __shfl_xor_sync(0xffffffffu, out[q], 1);
                if (f < F && k == 0)
#pragma unroll
                    for (int q = 0; q < 4; ++q) flux[q * F + f] = out[q];
            }
            // buffer b is free again; the lead warps wait for it only if this
            // block has a tile two steps on
            if (tile + 2 * (int64_t)gridDim.x < ntiles) bar_arrive_named(3 + b, NT);
        }
    }
}

template <bool KIN, int NL, int NW, int MINB>
gks_status launch_flux_ws(gks_mesh *m, const double *w, const double *x, double dt_const, const double *dt_dev,
                          double K, double *flux, cudaStream_t s)
{
    constexpr int TILE = 32 * NL;
    const gks_config &c = m->cfg;
    // persistent: as many blocks as fit on the GPU at once, at most one per tile
    const int key = ((NL * 16 + NW) * 8 + MINB) * 2 + (KIN ? 1 : 0);
    if (m->flux_ws_grid <= 0 || m->flux_ws_key != key) {
        int nsm = 0, per_sm = 0;
        GKS_CUDA(cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, m->device));
        GKS_CUDA(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k_face_flux_ws<KIN, NL, NW, MINB>, 32 * NW,
                                                               0));
        m->flux_ws_grid = (int64_t)nsm * (per_sm > 0 ? per_sm : 1);
        m->flux_ws_key = key;
    }
    const int64_t ntiles = (2 * m->d.F + TILE - 1) / TILE;
    const unsigned g = (unsigned)std::max<int64_t>(1, std::min<int64_t>(ntiles, m->flux_ws_grid));
    k_face_flux_ws<KIN, NL, NW, MINB><<<g, 32 * NW, 0, s>>>(m->d, w, x, m->wk.x32, dt_const, dt_dev, c.gamma, K, c.mu,
                                                     c.tau2_exact, flux, m->wk.status);
    return GKS_OK;
}

template <bool MIXED, bool HEAT, bool KIN>
__global__ void __launch_bounds__(kFluxBlock) k_point_flux(int64_t n, const double *__restrict__ wl,
                                                           const double *__restrict__ wr, double dt, double gamma,
                                                           double mu, int tau2, double prandtl,
                                                           double *__restrict__ out, int32_t *status)
{
    const int64_t q = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (q >= n) return;
    double a[24], b[24], f[4];
#pragma unroll
    for (int k = 0; k < 24; ++k) {
        a[k] = wl[24 * q + k];
        b[k] = wr[24 * q + k];
    }
    const bool ok = MIXED ? kin::gp_flux_mixed<HEAT, KIN>(a, b, dt, gamma, mu, tau2, f, prandtl)
                          : kin::gp_flux<double, HEAT, KIN>(a, b, dt, gamma, mu, tau2, f, prandtl);
    if (!ok && status) atomicOr(status, kStatusNonPhys);
#pragma unroll
    for (int k = 0; k < 4; ++k) out[4 * q + k] = f[k];
}

inline unsigned blocks(int64_t n, int b) { return (unsigned)((n + b - 1) / b); }

// f(std::bool_constant<a>, std::bool_constant<b>, std::bool_constant<c>): one
// kernel instantiation per combination of three compile-time switches
template <typename F>
void dispatch3(bool a, bool b, bool c, F &&f)
{
    using Y = std::true_type;
    using N = std::false_type;
    if (a) {
        if (b) c ? f(Y{}, Y{}, Y{}) : f(Y{}, Y{}, N{});
        else c ? f(Y{}, N{}, Y{}) : f(Y{}, N{}, N{});
    } else {
        if (b) c ? f(N{}, Y{}, Y{}) : f(N{}, Y{}, N{});
        else c ? f(N{}, N{}, Y{}) : f(N{}, N{}, N{});
    }
}

lead::LeadConst lead_const(const gks_config &c)
{
    const double K = 2.0 / (c.gamma - 1.0) - 2.0;
    lead::LeadConst lc;
    lc.gm1 = dfm::from_double(c.gamma - 1.0);
    lc.igm1 = dfm::from_double(1.0 / (c.gamma - 1.0));
    lc.K = dfm::from_double(K);
    lc.kp1 = dfm::from_double(K + 1.0);
    lc.mu = dfm::from_double(c.mu);
    lc.c001 = dfm::from_double(0.01);
    lc.hisp = dfm::from_double(0.28209479177387814347);    // 1 / (2 sqrt(pi))
    return lc;
}

}  // namespace

gks_status launch_flux(gks_mesh *m, const double *w, const double *x, double dt_const, const double *dt_dev,
                       double *flux, cudaStream_t s)
{
    const int64_t npts = 2 * m->d.F;
    const double K = 2.0 / (m->cfg.gamma - 1.0) - 2.0;
    const int slot = prof_start(m, kProfFlux, s);
    const gks_config &c = m->cfg;
    const bool heat = c.prandtl != 1.0;
    const unsigned g = blocks(npts, kFluxBlock);
    const bool mixed = c.precision == GKS_MIXED;
    if (mixed && c.flux_lead) {
        // FP32 pairs of the state and the coefficients, then the double-FP32 flux
        k_to_df<<<blocks(m->d.T, kBlock), kBlock, 0, s>>>(w, x, m->wk.w2, m->wk.x2, m->d.T);
        note_launch();
        const lead::LeadConst lc = lead_const(c);
        const df pr_fac = dfm::from_double(1.0 / c.prandtl - 1.0);
        const bool kin = c.slope0_mode == 1;
        auto go = [&](auto H, auto Kw) {
            k_face_flux_df<decltype(H)::value, decltype(Kw)::value><<<g, kFluxBlock, 0, s>>>(
                m->d, m->wk.w2, m->wk.x2, dt_const, dt_dev, lc, float(c.gamma), float(K), c.tau2_exact, pr_fac, flux,
                m->wk.status);
        };
        using Y = std::true_type;
        using N = std::false_type;
        if (heat) kin ? go(Y{}, Y{}) : go(Y{}, N{});
        else kin ? go(N{}, Y{}) : go(N{}, N{});
    } else {
    if (mixed) {
        // FP32 copy of the coefficients: the slope-carrying rows of every Gauss
        // point of a cell read it instead of converting the FP64 values again
        k_to_f32<<<blocks(20 * m->d.T, kBlock), kBlock, 0, s>>>(x, m->wk.x32, 20 * m->d.T);
        note_launch();
    }
    if (mixed && !heat && c.flux_split) {
        const gks_status st =
            c.slope0_mode == 1
                ? launch_flux_ws<true, kWsLead, kWsWarps, kWsMinBlocks>(m, w, x, dt_const, dt_dev, K, flux, s)
                : launch_flux_ws<false, kWsLead, kWsWarps, kWsMinBlocks>(m, w, x, dt_const, dt_dev, K, flux, s);
        if (st != GKS_OK) return st;
    } else {
        dispatch3(mixed, heat, c.slope0_mode == 1, [&](auto M, auto H, auto Kw) {
            k_face_flux<decltype(M)::value, decltype(H)::value, decltype(Kw)::value><<<g, kFluxBlock, 0, s>>>(
                m->d, w, x, mixed ? m->wk.x32 : nullptr, dt_const, dt_dev, c.gamma, K, c.mu, c.tau2_exact, c.prandtl,
                flux, m->wk.status);
        });
    }
    }
    note_launch();
    prof_stop(m, slot, s);
    GKS_CUDA(cudaGetLastError());
    return GKS_OK;
}

namespace {

// Point flux of the double-FP32 mixed path from FP64 rows [6][4] (face frame):
// the values as FP32 pairs, the derivative rows rounded to FP32.
template <bool HEAT, bool KIN>
__global__ void __launch_bounds__(kFluxBlock) k_point_flux_df(int64_t n, const double *__restrict__ wl,
                                                              const double *__restrict__ wr, double dt,
                                                              lead::LeadConst lc, float gamma_f, float K_f, int tau2,
                                                              df pr_fac, double *__restrict__ out, int32_t *status)
{
    const int64_t q = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (q >= n) return;
    df vl[4], vr[4];
    float dl[20], dr[20];
#pragma unroll
    for (int k = 0; k < 4; ++k) {
        vl[k] = dfm::split_double(wl[24 * q + k]);
        vr[k] = dfm::split_double(wr[24 * q + k]);
    }
#pragma unroll
    for (int k = 0; k < 20; ++k) {
        dl[k] = float(wl[24 * q + 4 + k]);
        dr[k] = float(wr[24 * q + 4 + k]);
    }
    const df dtd = dfm::split_double(dt);
    lead::Lead o;
    double f[4] = {0.0, 0.0, 0.0, 0.0};
    if (lead::gp_lead(vl, vr, dtd, lc, o)) {
        float vl4[4], vr4[4], w0f[4], gq[4], dg[4];
#pragma unroll
        for (int k = 0; k < 4; ++k) {
            vl4[k] = vl[k].hi;
            vr4[k] = vr[k].hi;
            w0f[k] = o.w0[k].hi;
        }
        kin::gp_body_mixed<HEAT, KIN>(vl4, vr4, dl, dr, w0f, o.tau.hi, dtd.hi, gamma_f, K_f, tau2, gq, dg);
        df fk[4];
#pragma unroll
        for (int k = 0; k < 4; ++k) fk[k] = dfm::add(o.f[k], gq[k]);
        if (HEAT) {
            df D[4];
#pragma unroll
            for (int k = 0; k < 4; ++k) D[k] = dfm::add(dfm::mul(o.c0c6, o.w0[k]), dg[k]);
            fk[3] = dfm::add(fk[3], dfm::mul(pr_fac, lead::heat_flux(fk, D, o.zu, o.zv)));
        }
#pragma unroll
        for (int k = 0; k < 4; ++k) f[k] = dfm::to_double(fk[k]);
    } else if (status) {
        atomicOr(status, kStatusNonPhys);
    }
#pragma unroll
    for (int k = 0; k < 4; ++k) out[4 * q + k] = f[k];
}


}  // namespace

gks_status launch_point_flux(int64_t n, const double *wl, const double *wr, double dt, const gks_config &cfg,
                             double *out, int32_t *status, cudaStream_t s)
{
    if (n <= 0) return GKS_OK;
    const unsigned g = blocks(n, kFluxBlock);
    const bool heat = cfg.prandtl != 1.0;
    if (cfg.precision == GKS_MIXED && cfg.flux_lead) {
        const double K = 2.0 / (cfg.gamma - 1.0) - 2.0;
        const lead::LeadConst lc = lead_const(cfg);
        const df pr_fac = dfm::from_double(1.0 / cfg.prandtl - 1.0);
        auto go = [&](auto H, auto Kw) {
            k_point_flux_df<decltype(H)::value, decltype(Kw)::value><<<g, kFluxBlock, 0, s>>>(
                n, wl, wr, dt, lc, float(cfg.gamma), float(K), cfg.tau2_exact, pr_fac, out, status);
        };
        using Y = std::true_type;
        using N = std::false_type;
        const bool kin = cfg.slope0_mode == 1;
        if (heat) kin ? go(Y{}, Y{}) : go(Y{}, N{});
        else kin ? go(N{}, Y{}) : go(N{}, N{});
    } else {
        dispatch3(cfg.precision == GKS_MIXED, heat, cfg.slope0_mode == 1, [&](auto M, auto H, auto Kw) {
            k_point_flux<decltype(M)::value, decltype(H)::value, decltype(Kw)::value><<<g, kFluxBlock, 0, s>>>(
                n, wl, wr, dt, cfg.gamma, cfg.mu, cfg.tau2_exact, cfg.prandtl, out, status);
        });
    }
    note_launch();
    GKS_CUDA(cudaGetLastError());
    return GKS_OK;
}

}  // namespace gks
