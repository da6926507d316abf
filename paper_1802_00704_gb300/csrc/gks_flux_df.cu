// Mixed-precision face flux with its FP64-accuracy part in double-FP32
// arithmetic on the FP32 pipe (flux_lead = 1): the kernel, its conversion of
// the state and coefficients to FP32 pairs, and the point-flux variant.
#include <type_traits>

#include "gks_face.cuh"
#include "gks_kinetic.cuh"
#include "gks_lead_df.cuh"

namespace gks {
namespace {

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
// NT threads per block, MINB blocks per SM: the register budget, 65536 /
// (NT MINB) per thread (128 for the default 128 x 4, with some spills; the
// autotuner also times 128 x 3 and 128 x 2).
template <bool HEAT, bool KIN, int NT = kFluxBlock, int MINB = 4>
__global__ void __launch_bounds__(NT, MINB)
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

inline unsigned blocks(int64_t n, int b) { return (unsigned)((n + b - 1) / b); }

}  // namespace

gks_status launch_flux_df(gks_mesh *m, const double *w, const double *x, double dt_const, const double *dt_dev,
                          double *flux, cudaStream_t s)
{
    const double K = 2.0 / (m->cfg.gamma - 1.0) - 2.0;
    const gks_config &c = m->cfg;
    const bool heat = c.prandtl != 1.0;
    const unsigned g = blocks(2 * m->d.F, kFluxBlock);
    {
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
        if (heat) {
            kin ? go(Y{}, Y{}) : go(Y{}, N{});
        } else if (kin) {
            go(N{}, Y{});
        } else {
            const float gf = float(c.gamma), kf = float(K);
            switch (c.flux_shape) {
            case 1:
                k_face_flux_df<false, false, 128, 3><<<g, 128, 0, s>>>(m->d, m->wk.w2, m->wk.x2, dt_const, dt_dev, lc,
                                                                      gf, kf, c.tau2_exact, pr_fac, flux,
                                                                      m->wk.status);
                break;
            case 2:
                k_face_flux_df<false, false, 128, 2><<<g, 128, 0, s>>>(m->d, m->wk.w2, m->wk.x2, dt_const, dt_dev, lc,
                                                                      gf, kf, c.tau2_exact, pr_fac, flux,
                                                                      m->wk.status);
                break;
            default:
                go(N{}, N{});
                break;
            }
        }
    }
    GKS_CUDA(cudaGetLastError());
    return GKS_OK;
}

gks_status launch_point_flux_df(int64_t n, const double *wl, const double *wr, double dt, const gks_config &cfg,
                                double *out, int32_t *status, cudaStream_t s)
{
    const unsigned g = blocks(n, kFluxBlock);
    const bool heat = cfg.prandtl != 1.0;
    {
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
    }
    GKS_CUDA(cudaGetLastError());
    return GKS_OK;
}

}  // namespace gks
