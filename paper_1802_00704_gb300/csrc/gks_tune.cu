// Autotuner of the solver knobs that change the cost of a step but not its
// result beyond the GMRES tolerance (gks_autotune).
//
// The cost of a step is dominated by the CLS solve, whose iteration count and
// cost per iteration depend on the workload: the number of ILU(0) sweeps trades
// preconditioner quality for passes over the factors, the extrapolated warm
// start pays off when the solution changes smoothly in time, and in mixed
// precision the inner tolerance trades FP32 Arnoldi iterations for FP64
// refinement residuals; the backward relation may take fewer sweeps than the
// forward one.  The tuner times a few steps of the handle's own cases for every
// combination and keeps the fastest; then it times shorter GMRES restarts with
// those knobs (a shorter restart orthogonalises against fewer vectors per
// iteration but may need more iterations), and the launch shapes of the
// double-FP32 flux kernel (its register budget against the warps per SM).
#include <cfloat>
#include <vector>

#include "gks_internal.h"

namespace gks {
namespace {

// One step of every case of the handle on the internal state m->wk.w (no end
// time, no host round trip); status bits accumulate in m->wk.status.
gks_status trial_step(gks_mesh *m, cudaStream_t s)
{
    Work &k = m->wk;
    gks_status st;
    if ((st = launch_cfl_dt(m, k.w, k.dt, s)) != GKS_OK) return st;
    if ((st = launch_clip_dt(m, s)) != GKS_OK) return st;
    if ((st = cls_solve(m, s, nullptr, nullptr, nullptr)) != GKS_OK) return st;
    if (m->cfg.limiter && (st = launch_limiter(m, k.w, k.x, s)) != GKS_OK) return st;
    if ((st = launch_flux(m, k.w, m->cfg.limiter ? k.xl : k.x, 0.0, k.dt, k.flux, s)) != GKS_OK) return st;
    return launch_update(m, k.w, k.flux, s);
}

// Time trial_steps steps of the current configuration from the caller's state w
// after 3 untimed ones.  *ms = time per step, or DBL_MAX if a step failed.
gks_status time_candidate(gks_mesh *m, const double *w, int trial_steps, cudaStream_t s, cudaEvent_t e0,
                          cudaEvent_t e1, double *ms)
{
    Work &k = m->wk;
    const int32_t n = m->n_case;
    gks_status st;
    GKS_CUDA(cudaMemsetAsync(k.x, 0, sizeof(double) * 20 * m->d.T, s));
    GKS_CUDA(cudaMemsetAsync(k.bnorm, 0, sizeof(double) * k.ns, s));
    GKS_CUDA(cudaMemsetAsync(k.nsolve, 0, sizeof(int64_t), s));
    GKS_CUDA(cudaMemsetAsync(k.tfinal, 0, sizeof(double) * n, s));
    GKS_CUDA(cudaMemsetAsync(k.tcase, 0, sizeof(double) * n, s));
    GKS_CUDA(cudaMemsetAsync(k.done, 0, sizeof(int32_t) * n, s));
    GKS_CUDA(cudaMemsetAsync(k.status, 0, sizeof(int32_t) * n, s));
    if ((st = launch_permute(w, k.w, m->d.perm, m->d.T, m->n_tri, 4, true, s)) != GKS_OK) return st;
    for (int q = 0; q < 3; ++q)
        if ((st = trial_step(m, s)) != GKS_OK) return st;
    GKS_CUDA(cudaEventRecord(e0, s));
    for (int q = 0; q < trial_steps; ++q)
        if ((st = trial_step(m, s)) != GKS_OK) return st;
    GKS_CUDA(cudaEventRecord(e1, s));
    std::vector<int32_t> stat(n);
    GKS_CUDA(cudaMemcpyAsync(stat.data(), k.status, sizeof(int32_t) * n, cudaMemcpyDeviceToHost, s));
    GKS_CUDA(cudaStreamSynchronize(s));
    float el = 0.0f;
    GKS_CUDA(cudaEventElapsedTime(&el, e0, e1));
    *ms = el / trial_steps;
    for (int32_t c = 0; c < n; ++c)
        if (stat[c]) *ms = DBL_MAX;
    return GKS_OK;
}

struct Candidate {
    int32_t sweeps, warm;
    double eta;
    int32_t bwd;
    int32_t m;                       // GMRES restart length
};

void apply(gks_mesh *m, const Candidate &c)
{
    m->cfg.ilu_sweeps = c.sweeps;
    m->cfg.warm_extrap = c.warm;
    m->cfg.inner_rtol = c.eta;
    m->cfg.ilu_sweeps_bwd = c.bwd;
    m->cfg.gmres_m = c.m;
    m->wk.m = c.m;
}

}  // namespace
}  // namespace gks

using namespace gks;

extern "C" gks_status gks_autotune(gks_mesh *m, const double *w, int32_t trial_steps, gks_tune_result *out,
                                   void *stream)
{
    if (!m || !w || !out || trial_steps < 1) {
        set_error("gks_autotune: NULL argument or trial_steps < 1");
        return GKS_EINVAL;
    }
    int prev = -1;
    GKS_CUDA(cudaGetDevice(&prev));
    if (prev != m->device) GKS_CUDA(cudaSetDevice(m->device));
    cudaStream_t s = (cudaStream_t)stream;
    const gks_config before = m->cfg;
    const bool mixed = m->cfg.precision == GKS_MIXED;
    const bool sweep = m->cfg.precond == GKS_PC_ILU_SWEEP;
    std::vector<Candidate> cand;
    // (forward, backward) sweeps: the same number each way (bwd -1), one
    // backward sweep after two or three forward ones, and one forward sweep
    // before a backward pair (one launch, k_ilu_bwd2)
    const int32_t pairs[6][2] = {{1, -1}, {2, -1}, {3, -1}, {2, 1}, {3, 1}, {1, 2}};
    for (const auto &pr : pairs) {
        const int32_t sw = pr[0], bwd = pr[1];
        if (!sweep && (sw != 1 || bwd != -1)) continue;
        for (int32_t wx : {0, 1, 2})
            for (double eta : {1e-4, 1e-5, 1e-6}) {
                if (!mixed && eta != 1e-6) continue;
                cand.push_back({sweep ? sw : before.ilu_sweeps, wx, mixed ? eta : before.inner_rtol,
                                sweep ? bwd : before.ilu_sweeps_bwd, m->wk.m});
            }
    }
    cudaEvent_t e0 = nullptr, e1 = nullptr;
    gks_status st = GKS_OK;
    if (cudaEventCreate(&e0) != cudaSuccess || cudaEventCreate(&e1) != cudaSuccess) {
        set_error("gks_autotune: cudaEventCreate failed");
        st = GKS_ECUDA;
    }
    double best = DBL_MAX, base = DBL_MAX;
    const int32_t m0 = m->wk.m;
    Candidate pick{before.ilu_sweeps, before.warm_extrap, before.inner_rtol, before.ilu_sweeps_bwd, m0};
    int32_t nfail = 0, ntimed = 0;
    auto try_one = [&](const Candidate &c) {
        apply(m, c);
        double ms = DBL_MAX;
        st = time_candidate(m, w, trial_steps, s, e0, e1, &ms);
        ++ntimed;
        if (st != GKS_OK) return;
        if (ms == DBL_MAX) ++nfail;
        if (ms < best) {
            best = ms;
            pick = c;
        }
    };
    // the configuration the handle had, then every candidate
    if (st == GKS_OK) st = time_candidate(m, w, trial_steps, s, e0, e1, &base);
    if (st == GKS_OK) best = base;
    for (size_t q = 0; st == GKS_OK && q < cand.size(); ++q) try_one(cand[q]);
    // second stage: the restart length with the best solver knobs (the Krylov
    // buffers hold m_alloc vectors, so only shorter restarts are possible)
    const Candidate knobs = pick;
    for (int32_t mr : {16, 8}) {
        if (st != GKS_OK || mr >= m->wk.m_alloc || mr == m0) continue;
        Candidate c = knobs;
        c.m = mr;
        try_one(c);
    }
    // third stage: the launch shape (register budget) of the double-FP32 flux
    // kernel, with the best knobs and restart length
    const int32_t v0 = m->cfg.flux_shape;
    int32_t vpick = v0;
    const bool df_flux = mixed && m->cfg.flux_lead == 1 && m->cfg.prandtl == 1.0 && m->cfg.slope0_mode == 0;
    if (df_flux && st == GKS_OK) {
        apply(m, pick);
        for (int32_t v = 0; v < kFluxDfVariants && st == GKS_OK; ++v) {
            if (v == v0) continue;
            m->cfg.flux_shape = v;
            double ms = DBL_MAX;
            st = time_candidate(m, w, trial_steps, s, e0, e1, &ms);
            ++ntimed;
            if (st == GKS_OK && ms < best) {
                best = ms;
                vpick = v;
            }
        }
        m->cfg.flux_shape = v0;
    }
    if (e0) cudaEventDestroy(e0);
    if (e1) cudaEventDestroy(e1);
    m->cfg = before;
    m->wk.m = m0;
    if (st == GKS_OK) {
        apply(m, pick);
        m->cfg.flux_shape = vpick;
        out->flux_variant = vpick;
        out->gmres_m = pick.m;
        out->ilu_sweeps = pick.sweeps;
        out->ilu_sweeps_bwd = pick.bwd;
        out->warm_extrap = pick.warm;
        out->inner_rtol = pick.eta;
        out->ms_per_step = best;
        out->ms_per_step_before = base;
        out->n_candidates = ntimed;
        out->n_failed = nfail;
    }
    // leave the handle as a fresh one: cleared warm start and case state
    cudaMemsetAsync(m->wk.x, 0, sizeof(double) * 20 * m->d.T, s);
    cudaMemsetAsync(m->wk.bnorm, 0, sizeof(double) * m->wk.ns, s);
    cudaMemsetAsync(m->wk.done, 0, sizeof(int32_t) * m->n_case, s);
    cudaMemsetAsync(m->wk.status, 0, sizeof(int32_t) * m->n_case, s);
    cudaMemsetAsync(m->wk.nsolve, 0, sizeof(int64_t), s);
    cudaError_t e = cudaStreamSynchronize(s);
    flush_solve_counters(m);
    if (st == GKS_OK && e != cudaSuccess) {
        set_error("gks_autotune: %s", cudaGetErrorString(e));
        st = GKS_ECUDA;
    }
    if (prev != m->device) cudaSetDevice(prev);
    return st;
}
