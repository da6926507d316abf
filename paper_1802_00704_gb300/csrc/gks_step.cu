// Conservative update, CFL time step, step control, permutations and the
// steady residual: the per-cell passes of a step around the flux.
//
// The update (Eq. (6)) gathers the (at most three) face fluxes of each cell: no
// atomics, a fixed summation order, one write per cell.
#include <cfloat>

#include "gks_internal.h"

namespace gks {
namespace {

// w_i -= (1/|Omega_i|) sum_f sigma_if F_f; flags non-physical results.
__global__ void k_update(DeviceMesh d, double *__restrict__ w, const double *__restrict__ flux, double gamma,
                         int32_t *status)
{
    const int64_t T = d.T, F = d.F;
    const int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (i >= T) return;
    double acc[4] = {0.0, 0.0, 0.0, 0.0};
#pragma unroll
    for (int s = 0; s < 3; ++s) {
        const int cf = d.cf[s * T + i];
        if (cf < 0) continue;
        const int64_t f = cf >> 1;
        const double sg = (cf & 1) ? 1.0 : -1.0;
#pragma unroll
        for (int v = 0; v < 4; ++v) acc[v] += sg * flux[v * F + f];
    }
    const double ia = d.inv_area[i];
    double wn[4];
#pragma unroll
    for (int v = 0; v < 4; ++v) {
        wn[v] = w[v * T + i] + acc[v] * ia;
        w[v * T + i] = wn[v];
    }
    // rho > 0 and p > 0, the latter as 2 rho E - |rho U|^2 > 0 (the same sign for
    // rho > 0): no FP64 division, which GB300 runs on its slow FP64 pipe
    const double q = 2.0 * wn[3] * wn[0] - (wn[1] * wn[1] + wn[2] * wn[2]);
    if (!(wn[0] > 0.0) || !(q > 0.0)) atomicOr(&status[d.blk_case[blockIdx.x]], kStatusNonPhys);
}

// v truncated to FP32 on the integer pipe (no FP64 instruction): false if v is
// not zero and outside the normal FP32 range (or not finite).
__device__ __forceinline__ bool trunc_f32(double v, float &f)
{
    const unsigned long long u = (unsigned long long)__double_as_longlong(v);
    const unsigned hw = (unsigned)(u >> 32);
    const unsigned E = (hw >> 20) & 0x7FFu;
    if ((u << 1) == 0ull) {
        f = 0.0f;
        return true;
    }
    if (E < 897u || E > 1150u) {
        f = 0.0f;
        return false;
    }
    f = __uint_as_float((hw & 0x80000000u) | ((E - 896u) << 23) | ((hw & 0xFFFFFu) << 3) | ((unsigned)u >> 29));
    return true;
}

// dt_i = r_i / (|U_i| + c_i + 2 mu / (rho_i r_i)) in FP64, as the oracle forms it
__device__ __forceinline__ double cfl_cell64(const double *__restrict__ w, int64_t T, int64_t i, double r,
                                             double gamma, double mu)
{
    const double rho = w[i], u = w[T + i] / rho, v = w[2 * T + i] / rho;
    const double p = (gamma - 1.0) * (w[3 * T + i] - 0.5 * rho * (u * u + v * v));
    const double c = sqrt(gamma * p / rho);
    const double dti = r / (sqrt(u * u + v * v) + c + 2.0 * mu / (rho * r));
    return dti > 0.0 ? dti : 0.0;                   // non-physical cell: forces dt = 0
}

// Block minima of the CFL step.  GB300's FP64 pipe would make the per-cell
// divisions and square roots the cost of this pass, so every cell first forms
// its step in FP32 from truncated inputs (relative error below 5e-5 when the
// pressure is not a cancellation, p >= 0.01 E); only the cells within 1e-3 of
// the block's smallest FP32 step, and the cells the screen cannot bound
// (cancellation, non-physical, outside the FP32 range), evaluate the FP64
// formula.  The FP64 minimiser is always among them, so the block minimum is
// the FP64 minimum bit for bit.
__global__ void k_cfl_partial(DeviceMesh d, const double *__restrict__ w, double gamma, double mu,
                              double *__restrict__ part)
{
    __shared__ float shf[kBlock / 32];
    __shared__ double shd[kBlock / 32];
    const int64_t T = d.T;
    const int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    float s = FLT_MAX;
    bool need64 = false;                             // the screen cannot bound the step: FP64
    double r = 0.0;
    if (i < T) {
        r = d.inrad[i];
        float rho, m1, m2, E, rf;
        bool ok = trunc_f32(w[i], rho) & trunc_f32(w[T + i], m1) & trunc_f32(w[2 * T + i], m2) &
                  trunc_f32(w[3 * T + i], E) & trunc_f32(r, rf);
        if (ok && rho > 0.0f) {
            const float gf = float(gamma), u = m1 / rho, v = m2 / rho;
            const float p = (gf - 1.0f) * (E - 0.5f * rho * (u * u + v * v));
            if (p >= 0.01f * E && p > 0.0f)
                s = rf / (sqrtf(u * u + v * v) + sqrtf(gf * p / rho) + 2.0f * float(mu) / (rho * rf));
            else
                need64 = true;
        } else {
            need64 = true;
        }
    }
    // block minimum of the screen
    float m = s;
    for (int o = 16; o > 0; o >>= 1) m = fminf(m, __shfl_xor_sync(0xffffffffu, m, o));
    if (lane == 0) shf[warp] = m;
    __syncthreads();
    m = shf[0];
    for (int k = 1; k < kBlock / 32; ++k) m = fminf(m, shf[k]);
    double dti = DBL_MAX;
    if (i < T && (need64 || s <= m * 1.001f)) dti = cfl_cell64(w, T, i, r, gamma, mu);
    for (int o = 16; o > 0; o >>= 1) dti = fmin(dti, __shfl_xor_sync(0xffffffffu, dti, o));
    if (lane == 0) shd[warp] = dti;
    __syncthreads();
    if (threadIdx.x == 0) {
        double b = shd[0];
        for (int k = 1; k < kBlock / 32; ++k) b = fmin(b, shd[k]);
        part[blockIdx.x] = b;
    }
}

// out[c] = scale * min of the block minima of case c (one block per case)
__global__ void k_min_final(const double *__restrict__ part, const int32_t *__restrict__ case_blk, double scale,
                            double *out)
{
    __shared__ double sh[kBlock];
    const int c = blockIdx.x;
    double m = DBL_MAX;
    for (int b = case_blk[c] + threadIdx.x; b < case_blk[c + 1]; b += blockDim.x) m = fmin(m, part[b]);
    sh[threadIdx.x] = m;
    __syncthreads();
    for (int o = blockDim.x / 2; o > 0; o >>= 1) {
        if (threadIdx.x < o) sh[threadIdx.x] = fmin(sh[threadIdx.x], sh[threadIdx.x + o]);
        __syncthreads();
    }
    if (threadIdx.x == 0) out[c] = scale * sh[0];
}

// Per-case step control: dt = min(cfl step, t_final - t), 0 once done; t += dt.
__global__ void k_clip_dt(double *dt, double *t, const double *__restrict__ tf, int32_t *done, int n)
{
    const int c = blockIdx.x * blockDim.x + threadIdx.x;
    if (c >= n) return;
    if (done[c] || (tf[c] > 0.0 && t[c] >= tf[c] * (1.0 - 1e-14))) {
        done[c] = 1;
        dt[c] = 0.0;
        return;
    }
    if (tf[c] > 0.0) dt[c] = fmin(dt[c], tf[c] - t[c]);
    t[c] += dt[c];
}

// dt of each case clipped to its end time; 0 for a case that is done or has
// reached its end (which marks it done); the time is advanced after the step
__global__ void k_clip_only(double *dt, const double *__restrict__ t, const double *__restrict__ tf, int32_t *done,
                            int n)
{
    const int c = blockIdx.x * blockDim.x + threadIdx.x;
    if (c >= n) return;
    if (done[c] || (tf[c] > 0.0 && t[c] >= tf[c] * (1.0 - 1e-14))) {
        done[c] = 1;
        dt[c] = 0.0;
        return;
    }
    if (tf[c] > 0.0) dt[c] = fmin(dt[c], tf[c] - t[c]);
}

// after a step: a case with status bits set stops (done); every other case
// that took a step advances its time, step count and last step
__global__ void k_after_step(const double *__restrict__ dt, double *t, int32_t *done,
                             const int32_t *__restrict__ status, int64_t *nstep, double *last_dt, int n)
{
    const int c = blockIdx.x * blockDim.x + threadIdx.x;
    if (c >= n || done[c] || !(dt[c] > 0.0)) return;
    if (status[c]) {
        done[c] = 1;
        return;
    }
    t[c] += dt[c];
    nstep[c] += 1;
    last_dt[c] = dt[c];
}

// acc[s] += iterations of system s in the last solve
__global__ void k_acc_iters(const int32_t *__restrict__ it, int64_t *acc, int ns)
{
    const int q = blockIdx.x * blockDim.x + threadIdx.x;
    if (q < ns) acc[q] += it[q];
}

// Internal rows [nvar][n] <-> caller rows [nvar][nc]; padding (perm < 0) untouched.
__global__ void k_permute(const double *__restrict__ src, double *__restrict__ dst, const int32_t *__restrict__ perm,
                          int64_t n, int64_t nc, int nvar, int gather)
{
    const int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (i >= n) return;
    const int64_t p = perm[i];
    if (p < 0) return;
    for (int v = 0; v < nvar; ++v) {
        if (gather) dst[v * n + i] = src[v * nc + p];
        else dst[v * nc + p] = src[v * n + i];
    }
}

// partial sums over cells of area * (w - w_old)^2 per variable
__global__ void k_steady_partial(DeviceMesh d, const double *__restrict__ w, const double *__restrict__ w_old,
                                 double *__restrict__ part)
{
    __shared__ double sh[kBlock];
    const int64_t T = d.T;
    const int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    for (int v = 0; v < 4; ++v) {
        double s = 0.0;
        if (i < T) {
            const double dw = w[v * T + i] - w_old[v * T + i];
            s = d.area[i] * dw * dw;
        }
        sh[threadIdx.x] = s;
        __syncthreads();
        for (int o = blockDim.x / 2; o > 0; o >>= 1) {
            if (threadIdx.x < o) sh[threadIdx.x] += sh[threadIdx.x + o];
            __syncthreads();
        }
        if (threadIdx.x == 0) part[blockIdx.x * 4 + v] = sh[0];
        __syncthreads();
    }
}

__global__ void k_sum4_final(const double *__restrict__ part, int n, double *out)
{
    __shared__ double sh[kBlock];
    for (int v = 0; v < 4; ++v) {
        double s = 0.0;
        for (int b = threadIdx.x; b < n; b += blockDim.x) s += part[b * 4 + v];
        sh[threadIdx.x] = s;
        __syncthreads();
        for (int o = blockDim.x / 2; o > 0; o >>= 1) {
            if (threadIdx.x < o) sh[threadIdx.x] += sh[threadIdx.x + o];
            __syncthreads();
        }
        if (threadIdx.x == 0) out[v] = sh[0];
        __syncthreads();
    }
}

inline unsigned blocks(int64_t n, int b) { return (unsigned)((n + b - 1) / b); }

}  // namespace

gks_status launch_update(gks_mesh *m, double *w, const double *flux, cudaStream_t s)
{
    const int slot = prof_start(m, kProfUpdate, s);
    k_update<<<blocks(m->d.T, kBlock), kBlock, 0, s>>>(m->d, w, flux, m->cfg.gamma, m->wk.status); note_launch();
    prof_stop(m, slot, s);
    GKS_CUDA(cudaGetLastError());
    return GKS_OK;
}

gks_status launch_cfl_dt(gks_mesh *m, const double *w, double *dt_dev, cudaStream_t s)
{
    const unsigned nb = blocks(m->d.T, kBlock);
    const int slot = prof_start(m, kProfCtl, s);
    k_cfl_partial<<<nb, kBlock, 0, s>>>(m->d, w, m->cfg.gamma, m->cfg.mu, m->wk.dpart); note_launch();
    k_min_final<<<m->d.ncase, kBlock, 0, s>>>(m->wk.dpart, m->d.case_blk, m->cfg.cfl, dt_dev); note_launch();
    prof_stop(m, slot, s);
    GKS_CUDA(cudaGetLastError());
    return GKS_OK;
}

gks_status launch_permute(const double *src, double *dst, const int32_t *perm, int64_t n, int64_t ncaller, int nvar,
                          bool gather, cudaStream_t s)
{
    k_permute<<<blocks(n, kBlock), kBlock, 0, s>>>(src, dst, perm, n, ncaller, nvar, gather ? 1 : 0); note_launch();
    GKS_CUDA(cudaGetLastError());
    return GKS_OK;
}

gks_status launch_clip_dt(gks_mesh *m, cudaStream_t s)
{
    const int n = m->d.ncase;
    k_clip_dt<<<(n + 127) / 128, 128, 0, s>>>(m->wk.dt, m->wk.tcase, m->wk.tfinal, m->wk.done, n); note_launch();
    GKS_CUDA(cudaGetLastError());
    return GKS_OK;
}

gks_status launch_clip_only(gks_mesh *m, cudaStream_t s)
{
    const int n = m->d.ncase;
    k_clip_only<<<(n + 127) / 128, 128, 0, s>>>(m->wk.dt, m->wk.tcase, m->wk.tfinal, m->wk.done, n); note_launch();
    GKS_CUDA(cudaGetLastError());
    return GKS_OK;
}

gks_status launch_after_step(gks_mesh *m, cudaStream_t s)
{
    const int n = m->d.ncase;
    Work &k = m->wk;
    k_after_step<<<(n + 127) / 128, 128, 0, s>>>(k.dt, k.tcase, k.done, k.status, k.nstep, k.last_dt, n);
    note_launch();
    GKS_CUDA(cudaGetLastError());
    return GKS_OK;
}

gks_status launch_acc_iters(gks_mesh *m, cudaStream_t s)
{
    const int ns = m->wk.ns;
    k_acc_iters<<<(ns + 127) / 128, 128, 0, s>>>(m->wk.ctl + kCtlIters * ns, m->wk.iters_acc, ns); note_launch();
    GKS_CUDA(cudaGetLastError());
    return GKS_OK;
}

// m->wk.scal[0..3] = sum over cells of area (w - w_old)^2 per variable
gks_status launch_steady_partial(gks_mesh *m, cudaStream_t s)
{
    const unsigned nb = blocks(m->d.T, kBlock);
    k_steady_partial<<<nb, kBlock, 0, s>>>(m->d, m->wk.w, m->wk.w_old, m->wk.dpart); note_launch();
    k_sum4_final<<<1, kBlock, 0, s>>>(m->wk.dpart, (int)nb, m->wk.scal); note_launch();
    GKS_CUDA(cudaGetLastError());
    return GKS_OK;
}

}  // namespace gks
