// Face fluxes (Eqs. (7), (11), (15)): reconstruction at the Gauss points,
// ghost states, and the kinetic flux; one thread per face Gauss point, the two
// points of a face in neighbouring lanes summed with one shuffle, so each face
// flux is written once, without atomics.
#include <cfloat>

#include <type_traits>

#include "gks_internal.h"
#include "gks_kinetic.cuh"

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

// Mixed precision reconstruction: FP64 values, FP32 derivative rows (global frame).
__device__ __forceinline__ void recon_mixed(const DeviceMesh &d, const double *__restrict__ w,
                                            const double *__restrict__ x, const float *__restrict__ x32, int c,
                                            double dx, double dy, double *val, float *der)
{
    const int64_t T = d.T;
    const double qx = dx * dx - d.mxx[c], qxy = dx * dy - d.mxy[c], qy = dy * dy - d.myy[c];
    const float ih = d.ih32[c];
    const float fx = float(dx), fy = float(dy);
#pragma unroll
    for (int v = 0; v < 4; ++v) {
        const double u1 = x[(v * 5 + 0) * T + c], u2 = x[(v * 5 + 1) * T + c], u3 = x[(v * 5 + 2) * T + c];
        const double u4 = x[(v * 5 + 3) * T + c], u5 = x[(v * 5 + 4) * T + c];
        val[v] = w[v * T + c] + u1 * dx + u2 * dy + 0.5 * u3 * qx + u4 * qxy + 0.5 * u5 * qy;
        const float f1 = x32[(v * 5 + 0) * T + c], f2 = x32[(v * 5 + 1) * T + c], f3 = x32[(v * 5 + 2) * T + c];
        const float f4 = x32[(v * 5 + 3) * T + c], f5 = x32[(v * 5 + 4) * T + c];
        der[v] = (f1 + f3 * fx + f4 * fy) * ih;
        der[4 + v] = (f2 + f4 * fx + f5 * fy) * ih;
        der[8 + v] = f3 * ih * ih;
        der[12 + v] = f4 * ih * ih;
        der[16 + v] = f5 * ih * ih;
    }
}

// Face frame of FP64 values (momentum) and FP32 derivative rows (directions and momentum).
__device__ __forceinline__ void to_face_mixed(double *val, float *der, double nx, double ny)
{
    const double mx = val[1], my = val[2];
    val[1] = nx * mx + ny * my;
    val[2] = -ny * mx + nx * my;
    const float fnx = float(nx), fny = float(ny), tx = -fny, ty = fnx;
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

// Ghost state of a boundary face for the split (FP64 values, FP32 derivatives) layout.
__device__ __forceinline__ void ghost_mixed(int tag, const double *bc, double nx, double ny, double gamma,
                                            const double *vl, const float *dl, double *vr, float *dr)
{
    if (tag == GKS_BC_DIRICHLET) {
        vr[0] = bc[0];
        vr[1] = nx * bc[1] + ny * bc[2];
        vr[2] = -ny * bc[1] + nx * bc[2];
        vr[3] = bc[3];
#pragma unroll
        for (int q = 0; q < 20; ++q) dr[q] = 0.0f;
        return;
    }
    if (tag == GKS_BC_OUTFLOW) {
#pragma unroll
        for (int q = 0; q < 4; ++q) vr[q] = vl[q];
#pragma unroll
        for (int q = 0; q < 20; ++q) dr[q] = dl[q];
        return;
    }
    const bool noslip = tag == GKS_BC_NOSLIP;
    const int npar[5] = {1, 0, 0, 1, 0};   // parity of the n-order of rows d/dn .. d2/dt2
#pragma unroll
    for (int r = 0; r < 5; ++r)
#pragma unroll
        for (int v = 0; v < 4; ++v) {
            float sg = (v == 1 || (noslip && v == 2)) ? -1.0f : 1.0f;
            if (npar[r]) sg = -sg;
            dr[4 * r + v] = sg * dl[4 * r + v];
        }
    if (noslip) {
        const double rho = vl[0], un = vl[1] / rho, ut = vl[2] / rho;
        const double p = (gamma - 1.0) * (vl[3] - 0.5 * rho * (un * un + ut * ut));
        const double uwn = nx * bc[0] + ny * bc[1], uwt = -ny * bc[0] + nx * bc[1];
        const double tg = 2.0 * bc[2] - p / rho;
        const double gn = 2.0 * uwn - un, gt = 2.0 * uwt - ut;
        vr[0] = rho;
        vr[1] = rho * gn;
        vr[2] = rho * gt;
        vr[3] = rho * tg / (gamma - 1.0) + 0.5 * rho * (gn * gn + gt * gt);
    } else {
        vr[0] = vl[0];
        vr[1] = -vl[1];
        vr[2] = vl[2];
        vr[3] = vl[3];
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
    // mirror image: q_R(n, t) = s_q q_L(-n, t); a derivative of order p in n gets (-1)^p
    const bool noslip = tag == GKS_BC_NOSLIP;
    const int npar[6] = {0, 1, 0, 0, 1, 0};   // parity of the n-order of each row
#pragma unroll
    for (int r = 0; r < 6; ++r)
#pragma unroll
        for (int v = 0; v < 4; ++v) {
            double s = (v == 1 || (noslip && v == 2)) ? -1.0 : 1.0;
            if (npar[r]) s = -s;
            wr[4 * r + v] = s * wl[4 * r + v];
        }
    if (noslip) {
        const double rho = wl[0], un = wl[1] / rho, ut = wl[2] / rho;
        const double p = (gamma - 1.0) * (wl[3] - 0.5 * rho * (un * un + ut * ut));
        const double uwn = nx * bc[0] + ny * bc[1], uwt = -ny * bc[0] + nx * bc[1];
        const double tg = 2.0 * bc[2] - p / rho;
        const double gn = 2.0 * uwn - un, gt = 2.0 * uwt - ut;
        wr[0] = rho;
        wr[1] = rho * gn;
        wr[2] = rho * gt;
        wr[3] = rho * tg / (gamma - 1.0) + 0.5 * rho * (gn * gn + gt * gt);
    }
}

// y = float(x), n values
__global__ void k_to_f32(const double *__restrict__ x, float *__restrict__ y, int64_t n)
{
    const int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (i < n) y[i] = float(x[i]);
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
            recon_mixed(d, w, x, x32, l, d.gl[(2 * k) * F + f], d.gl[(2 * k + 1) * F + f], vl, dl);
            to_face_mixed(vl, dl, nx, ny);
            if (r >= 0) {
                recon_mixed(d, w, x, x32, r, d.gr[(2 * k) * F + f], d.gr[(2 * k + 1) * F + f], vr, dr);
                to_face_mixed(vr, dr, nx, ny);
            } else {
                const double bc[4] = {d.bc[f], d.bc[F + f], d.bc[2 * F + f], d.bc[3 * F + f]};
                ghost_mixed(d.ftag[f], bc, nx, ny, gamma, vl, dl, vr, dr);
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
    if (mixed) {
        // FP32 copy of the coefficients: the slope-carrying rows of every Gauss
        // point of a cell read it instead of converting the FP64 values again
        k_to_f32<<<blocks(20 * m->d.T, kBlock), kBlock, 0, s>>>(x, m->wk.x32, 20 * m->d.T);
        note_launch();
    }
    dispatch3(mixed, heat, c.slope0_mode == 1, [&](auto M, auto H, auto Kw) {
        k_face_flux<decltype(M)::value, decltype(H)::value, decltype(Kw)::value><<<g, kFluxBlock, 0, s>>>(
            m->d, w, x, mixed ? m->wk.x32 : nullptr, dt_const, dt_dev, c.gamma, K, c.mu, c.tau2_exact, c.prandtl,
            flux, m->wk.status);
    });
    note_launch();
    prof_stop(m, slot, s);
    GKS_CUDA(cudaGetLastError());
    return GKS_OK;
}

gks_status launch_point_flux(int64_t n, const double *wl, const double *wr, double dt, const gks_config &cfg,
                             double *out, int32_t *status, cudaStream_t s)
{
    if (n <= 0) return GKS_OK;
    const unsigned g = blocks(n, kFluxBlock);
    const bool heat = cfg.prandtl != 1.0;
    dispatch3(cfg.precision == GKS_MIXED, heat, cfg.slope0_mode == 1, [&](auto M, auto H, auto Kw) {
        k_point_flux<decltype(M)::value, decltype(H)::value, decltype(Kw)::value><<<g, kFluxBlock, 0, s>>>(
            n, wl, wr, dt, cfg.gamma, cfg.mu, cfg.tau2_exact, cfg.prandtl, out, status);
    });
    note_launch();
    GKS_CUDA(cudaGetLastError());
    return GKS_OK;
}

}  // namespace gks
