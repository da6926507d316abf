// Face fluxes (Eqs. (7), (11), (15)): reconstruction at the Gauss points,
// ghost states, and the kinetic flux; one thread per face Gauss point, the two
// points of a face in neighbouring lanes summed with one shuffle, so each face
// flux is written once, without atomics.
#include <algorithm>
#include <cfloat>

#include <type_traits>

#include "gks_face.cuh"
#include "gks_kinetic.cuh"

namespace gks {
namespace {

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
    // flux_lead = 2: the mixed solver with the FP64 path's flux kernel
    const bool mixed = c.precision == GKS_MIXED && c.flux_lead != 2;
    if (mixed && c.flux_lead == 1) {
        const gks_status st = launch_flux_df(m, w, x, dt_const, dt_dev, flux, s);
        if (st != GKS_OK) return st;
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

gks_status launch_point_flux(int64_t n, const double *wl, const double *wr, double dt, const gks_config &cfg,
                             double *out, int32_t *status, cudaStream_t s)
{
    if (n <= 0) return GKS_OK;
    const unsigned g = blocks(n, kFluxBlock);
    const bool heat = cfg.prandtl != 1.0;
    const bool mixed = cfg.precision == GKS_MIXED && cfg.flux_lead != 2;
    if (mixed && cfg.flux_lead == 1) {
        const gks_status st = launch_point_flux_df(n, wl, wr, dt, cfg, out, status, s);
        if (st != GKS_OK) return st;
    } else {
        dispatch3(mixed, heat, cfg.slope0_mode == 1, [&](auto M, auto H, auto Kw) {
            k_point_flux<decltype(M)::value, decltype(H)::value, decltype(Kw)::value><<<g, kFluxBlock, 0, s>>>(
                n, wl, wr, dt, cfg.gamma, cfg.mu, cfg.tau2_exact, cfg.prandtl, out, status);
        });
    }
    note_launch();
    GKS_CUDA(cudaGetLastError());
    return GKS_OK;
}

}  // namespace gks
