// C ABI entry points (include/gks.h).
#include <algorithm>
#include <cmath>
#include <vector>
#include <cstring>
#include <new>

#include "gks_internal.h"

namespace gks {
const char *last_error();
std::atomic<int64_t> g_launches{0};

int prof_start(gks_mesh *m, int cls, cudaStream_t s)
{
    gks_profiler &p = m->prof;
    if (!(p.mask & (1 << cls))) return -1;
    while (p.events.size() < p.used + 2) {
        cudaEvent_t e;
        if (cudaEventCreate(&e) != cudaSuccess) return -1;
        p.events.push_back(e);
    }
    const int slot = (int)p.used;
    p.used += 2;
    p.cls.push_back(cls);
    cudaEventRecord(p.events[slot], s);
    return slot;
}

void prof_stop(gks_mesh *m, int slot, cudaStream_t s)
{
    if (slot >= 0) cudaEventRecord(m->prof.events[slot + 1], s);
}
}  // namespace gks

using namespace gks;

namespace {

struct DeviceGuard {
    int prev = -1;
    bool changed = false;
    explicit DeviceGuard(int dev)
    {
        if (cudaGetDevice(&prev) == cudaSuccess && prev != dev) changed = cudaSetDevice(dev) == cudaSuccess;
    }
    ~DeviceGuard()
    {
        if (changed) cudaSetDevice(prev);
    }
};

gks_status check_config(const gks_config &c)
{
    bool ok = c.gamma > 1.0 && c.cfl > 0.0 && c.mu >= 0.0 && c.cls_w > 0.0 && c.gmres_m >= 1 &&
              c.gmres_m <= kMaxRestart && c.gmres_maxit >= 1 && c.gmres_rtol > 0.0 &&
              (c.tau2_exact == 0 || c.tau2_exact == 1) && c.ilu_sweeps >= 0 && c.ilu_sweeps <= 16;
    ok = ok && c.limiter >= 0 && c.limiter <= 2;
    ok = ok && (c.basis_fp32 == 0 || (c.basis_fp32 == 1 && c.precision == GKS_MIXED));
    ok = ok && c.warm_extrap >= 0 && c.warm_extrap <= 2;
    ok = ok && c.inner_rtol > 0.0 && c.inner_rtol < 1.0 && c.prandtl > 0.0;
    ok = ok && (c.second_order == 0 || c.second_order == 1);
    ok = ok && c.no_graphs >= 0 && c.no_graphs <= 2;
    ok = ok && (c.limit_char == 0 || c.limit_char == 1);
    ok = ok && (c.slope0_mode == 0 || c.slope0_mode == 1);
    ok = ok && (c.ilu_fp16 == 0 || (c.ilu_fp16 == 1 && c.precision == GKS_MIXED));
    ok = ok && (c.cls_global == 0 || c.cls_global == 1);
    ok = ok && c.cls_M >= 0 && c.cls_M <= 2 && (c.cls_M > 0 || c.second_order == 1);
    ok = ok && c.ilu_sweeps_bwd >= -1 && c.ilu_sweeps_bwd <= 8;
    ok = ok && (c.ilu_fuse_first == 0 || c.ilu_fuse_first == 1);
    ok = ok && (c.flux_split == 0 || c.flux_split == 1);
    ok = ok && c.flux_lead >= 0 && c.flux_lead <= 2;
    ok = ok && c.flux_shape >= 0 && c.flux_shape < kFluxDfVariants && c.reserved == 0;
    ok = ok && (c.ilu_sweep_pairs == 0 || c.ilu_sweep_pairs == 1);
    ok = ok && (c.spmv_dots == 0 || c.spmv_dots == 1);
    if (!ok) {
        set_error("invalid gks_config");
        return GKS_EINVAL;
    }
    if (c.precision != GKS_FP64 && c.precision != GKS_MIXED) {
        set_error("gks_config.precision: GKS_FP64 or GKS_MIXED");
        return GKS_EINVAL;
    }
    if (c.precond < GKS_PC_ILU_EXACT || c.precond > GKS_PC_ILU_LEVELS) {
        set_error("gks_config.precond: one of GKS_PC_ILU_EXACT, GKS_PC_ILU_SWEEP, GKS_PC_BJACOBI, GKS_PC_ILU_LEVELS");
        return GKS_EINVAL;
    }
    return GKS_OK;
}

// The status code of a case's status bits; a wait that gave up comes first
// (the results of that step are not usable), and sets the error message.
gks_status code_of(int32_t bits)
{
    if (bits & kStatusTimeout) {
        set_error("a bounded wait of the sync-free ILU solve gave up (GKS_PC_ILU_EXACT)");
        return GKS_ETIMEOUT;
    }
    if (bits & kStatusNonPhys) {
        set_error("non-physical state (rho <= 0 or p <= 0)");
        return GKS_ENONPHYS;
    }
    if (bits & kStatusNoConv) {
        set_error("GMRES did not reach gmres_rtol within gmres_maxit");
        return GKS_ENOCONV;
    }
    return GKS_OK;
}

gks_status read_status(gks_mesh *m, cudaStream_t s, int32_t *out)
{
    GKS_CUDA(cudaMemcpyAsync(m->wk.h_flags + 2, m->wk.status, sizeof(int32_t), cudaMemcpyDeviceToHost, s));
    GKS_CUDA(cudaStreamSynchronize(s));
    *out = m->wk.h_flags[2];
    return GKS_OK;
}

gks_status require_single(const gks_mesh *m, const char *who)
{
    if (m->n_case != 1) {
        set_error("%s: the handle holds %d cases; use gks_batch_run", who, m->n_case);
        return GKS_EINVAL;
    }
    return GKS_OK;
}

// one step of a single-case handle on the internal state m->wk.w; dt_fixed > 0 fixes the step
gks_status step_internal(gks_mesh *m, double dt_fixed, cudaStream_t s, gks_step_info *info, double *dt_taken)
{
    gks_status st;
    Work &k = m->wk;
    if (dt_fixed > 0.0) {
        k.h_scal[7] = dt_fixed;
        GKS_CUDA(cudaMemcpyAsync(k.dt, &k.h_scal[7], sizeof(double), cudaMemcpyHostToDevice, s));
    } else if ((st = launch_cfl_dt(m, k.w, k.dt, s)) != GKS_OK) {
        return st;
    }
    int32_t iters[4], conv = 1;
    double relres[4];
    if ((st = cls_solve(m, s, iters, relres, &conv)) != GKS_OK) return st;
    if (m->cfg.limiter && (st = launch_limiter(m, k.w, k.x, s)) != GKS_OK) return st;
    if ((st = launch_flux(m, k.w, m->cfg.limiter ? k.xl : k.x, 0.0, k.dt, k.flux, s)) != GKS_OK) return st;
    if ((st = launch_update(m, k.w, k.flux, s)) != GKS_OK) return st;
    GKS_CUDA(cudaMemcpyAsync(&k.h_scal[6], k.dt, sizeof(double), cudaMemcpyDeviceToHost, s));
    int32_t stat = 0;
    if ((st = read_status(m, s, &stat)) != GKS_OK) return st;
    if (dt_taken) *dt_taken = k.h_scal[6];
    gks_status res = code_of(stat | (conv ? 0 : kStatusNoConv));
    if (info) {
        info->dt = k.h_scal[6];
        for (int v = 0; v < 4; ++v) {
            info->iters[v] = iters[v];
            info->relres[v] = relres[v];
        }
        info->status = res;
    }
    return res;
}

gks_status create(const CaseIn *cases, int32_t n, const gks_config *cfg, gks_mesh **out)
{
    set_error("");
    if (!out) {
        set_error("gks_mesh_create: out is NULL");
        return GKS_EINVAL;
    }
    *out = nullptr;
    gks_mesh *m = new (std::nothrow) gks_mesh();
    if (!m) {
        set_error("gks_mesh_create: host allocation failed");
        return GKS_ENOMEM;
    }
    if (cfg) m->cfg = *cfg;
    else gks_config_default(&m->cfg);
    gks_status st = check_config(m->cfg);
    if (st == GKS_OK && cudaGetDevice(&m->device) != cudaSuccess) {
        set_error("gks_mesh_create: no CUDA device");
        st = GKS_ECUDA;
    }
    if (st == GKS_OK) st = build_batch(m, cases, n);
    if (st != GKS_OK) {
        free_mesh(m);
        delete m;
        return st;
    }
    *out = m;
    return GKS_OK;
}

// One CFL step of a single-case handle (state already in m->wk.w) as one
// launch of the step-loop graph (loop limit 1, no end time), its results
// enqueued for the host: *used = false when the graph cannot be used (graphs
// off, the profiler on), and nothing was launched.
gks_status step_graph_launch(gks_mesh *m, cudaStream_t s, bool *used)
{
    Work &k = m->wk;
    *used = false;
    GKS_CUDA(cudaMemsetAsync(k.tfinal, 0, sizeof(double), s));
    GKS_CUDA(cudaMemsetAsync(k.tcase, 0, sizeof(double), s));
    gks_status st = run_graph_launch(m, 1, s, used);
    if (st != GKS_OK || !*used) return st;
    // the solve's iterations and residuals, the step taken and the status bits
    const int ns = k.ns;
    GKS_CUDA(cudaMemcpyAsync(k.h_step, k.beta, sizeof(double) * ns, cudaMemcpyDeviceToHost, s));
    GKS_CUDA(cudaMemcpyAsync(k.h_step + 4, k.bnorm, sizeof(double) * ns, cudaMemcpyDeviceToHost, s));
    GKS_CUDA(cudaMemcpyAsync(k.h_step + 8, k.last_dt, sizeof(double), cudaMemcpyDeviceToHost, s));
    GKS_CUDA(cudaMemcpyAsync(k.h_stepi, k.ctl + kCtlIters * ns, sizeof(int32_t) * ns, cudaMemcpyDeviceToHost, s));
    GKS_CUDA(cudaMemcpyAsync(k.h_stepi + 4, k.status, sizeof(int32_t), cudaMemcpyDeviceToHost, s));
    return GKS_OK;
}

// The results of step_graph_launch once the stream has been synchronised.
gks_status step_graph_results(gks_mesh *m, gks_step_info *info, double *dt_taken)
{
    const Work &k = m->wk;
    const double rtol = m->cfg.gmres_rtol;
    int32_t conv = 1;
    double rr[4];
    for (int v = 0; v < 4; ++v) {
        rr[v] = k.h_step[4 + v] > 0.0 ? k.h_step[v] / k.h_step[4 + v] : 0.0;
        if (rr[v] > rtol) conv = 0;
    }
    const gks_status res = code_of(k.h_stepi[4] | (conv ? 0 : kStatusNoConv));
    if (dt_taken) *dt_taken = k.h_step[8];
    if (info) {
        info->dt = k.h_step[8];
        for (int v = 0; v < 4; ++v) {
            info->iters[v] = k.h_stepi[v];
            info->relres[v] = rr[v];
        }
        info->status = res;
    }
    return res;
}

}  // namespace

extern "C" {

void gks_config_default(gks_config *c)
{
    if (!c) return;
    std::memset(c, 0, sizeof(*c));
    c->gamma = 1.4;
    c->cfl = 0.3;
    c->mu = 0.0;
    c->cls_w = 0.3;
    c->gmres_m = 30;
    c->gmres_maxit = 1000;
    c->gmres_rtol = 1e-12;
    c->precision = GKS_FP64;
    c->precond = GKS_PC_ILU_SWEEP;
    c->ilu_sweeps = 2;
    c->tau2_exact = 0;
    c->inner_rtol = 1e-6;
    c->prandtl = 1.0;
    c->slope0_mode = 0;
    c->ilu_fp16 = 0;
    c->cls_global = 0;
    c->cls_M = 1;
    c->ilu_sweeps_bwd = -1;
    c->ilu_fuse_first = 1;
    c->flux_split = 1;
    c->ilu_sweep_pairs = 1;
    c->spmv_dots = 1;
    c->flux_lead = 1;
    c->flux_shape = 0;
    c->reserved = 0;
}

const char *gks_last_error(void) { return gks::last_error(); }

gks_status gks_mesh_create(const double *nodes, int64_t n_nodes, const int32_t *tris, int64_t n_tri,
                           const int32_t *faces, const double *face_shift, int64_t n_face, const double *bc_state,
                           const gks_config *cfg, gks_mesh **out)
{
    const CaseIn c{nodes, n_nodes, tris, n_tri, faces, face_shift, n_face, bc_state};
    return create(&c, 1, cfg, out);
}

gks_status gks_batch_create(const gks_case_desc *cases, int32_t n_cases, const gks_config *cfg, gks_mesh **out)
{
    if (!cases || n_cases <= 0) {
        set_error("gks_batch_create: no case");
        if (out) *out = nullptr;
        return GKS_EINVAL;
    }
    std::vector<CaseIn> in(n_cases);
    for (int32_t c = 0; c < n_cases; ++c)
        in[c] = CaseIn{cases[c].nodes, cases[c].n_nodes, cases[c].tris, cases[c].n_tri, cases[c].faces,
                       cases[c].face_shift, cases[c].n_face, cases[c].bc_state};
    return create(in.data(), n_cases, cfg, out);
}

gks_status gks_mesh_destroy(gks_mesh *m)
{
    if (!m) return GKS_OK;
    DeviceGuard g(m->device);
    for (cudaEvent_t e : m->prof.events) cudaEventDestroy(e);
    free_mesh(m);
    delete m;
    return GKS_OK;
}

gks_status gks_mesh_get_stats(const gks_mesh *m, gks_mesh_stats *s)
{
    if (!m || !s) {
        set_error("gks_mesh_get_stats: NULL argument");
        return GKS_EINVAL;
    }
    s->n_tri = m->n_tri;
    s->n_face = m->n_face;
    s->n_boundary_face = m->n_bface;
    s->n_k1 = m->n_k1;
    s->nnzb = m->nnzb;
    s->levels_lower = (int32_t)m->lvl_lo_ptr.size() - 1;
    s->levels_upper = (int32_t)m->lvl_up_ptr.size() - 1;
    s->rcm_bandwidth = m->bandwidth;
    s->device_bytes = m->device_bytes;
    s->n_case = m->n_case;
    return GKS_OK;
}

gks_status gks_cfl_dt(gks_mesh *m, const double *w, double *dt_out, void *stream)
{
    if (!m || !w || !dt_out) {
        set_error("gks_cfl_dt: NULL argument");
        return GKS_EINVAL;
    }
    if (require_single(m, "gks_cfl_dt") != GKS_OK) return GKS_EINVAL;
    DeviceGuard g(m->device);
    cudaStream_t s = (cudaStream_t)stream;
    gks_status st;
    if ((st = launch_permute(w, m->wk.w, m->d.perm, m->d.T, m->n_tri, 4, true, s)) != GKS_OK) return st;
    if ((st = launch_cfl_dt(m, m->wk.w, m->wk.dt, s)) != GKS_OK) return st;
    GKS_CUDA(cudaMemcpyAsync(&m->wk.h_scal[6], m->wk.dt, sizeof(double), cudaMemcpyDeviceToHost, s));
    GKS_CUDA(cudaStreamSynchronize(s));
    *dt_out = m->wk.h_scal[6];
    return GKS_OK;
}

gks_status gks_cls_reconstruct(gks_mesh *m, const double *w, double *coef, gks_solve_info *info, void *stream)
{
    if (!m || !w || !coef) {
        set_error("gks_cls_reconstruct: NULL argument");
        return GKS_EINVAL;
    }
    DeviceGuard g(m->device);
    cudaStream_t s = (cudaStream_t)stream;
    gks_status st;
    if ((st = launch_permute(w, m->wk.w, m->d.perm, m->d.T, m->n_tri, 4, true, s)) != GKS_OK) return st;
    GKS_CUDA(cudaMemsetAsync(m->wk.done, 0, sizeof(int32_t) * m->n_case, s));
    std::vector<int32_t> it(m->wk.ns);
    std::vector<double> rr(m->wk.ns);
    gks_solve_info si{};
    if ((st = cls_solve(m, s, it.data(), rr.data(), &si.converged)) != GKS_OK) return st;
    if ((st = launch_permute(m->wk.x, coef, m->d.perm, m->d.T, m->n_tri, 20, false, s)) != GKS_OK) return st;
    for (int q = 0; q < m->wk.ns; ++q) {         // per variable: the largest over the cases
        si.iters[q & 3] = std::max(si.iters[q & 3], it[q]);
        si.relres[q & 3] = std::max(si.relres[q & 3], rr[q]);
    }
    if (info) *info = si;
    if (m->cfg.precond == GKS_PC_ILU_EXACT) {
        int32_t waited_out = 0;
        GKS_CUDA(cudaMemcpyAsync(&waited_out, m->wk.sf_ctl + 3, sizeof(int32_t), cudaMemcpyDeviceToHost, s));
        GKS_CUDA(cudaStreamSynchronize(s));
        if (waited_out) return code_of(kStatusTimeout);
    }
    if (!si.converged) return code_of(kStatusNoConv);
    return GKS_OK;
}

gks_status gks_reset_warm_start(gks_mesh *m)
{
    if (!m) {
        set_error("gks_reset_warm_start: NULL mesh");
        return GKS_EINVAL;
    }
    DeviceGuard g(m->device);
    GKS_CUDA(cudaMemset(m->wk.x, 0, sizeof(double) * 20 * m->d.T));
    GKS_CUDA(cudaMemset(m->wk.bnorm, 0, sizeof(double) * m->wk.ns));
    GKS_CUDA(cudaMemset(m->wk.nsolve, 0, sizeof(int64_t)));
    return GKS_OK;
}

gks_status gks_limit(gks_mesh *m, const double *w, const double *coef, double *coef_out, int32_t *flags,
                     void *stream)
{
    if (!m || !w || !coef || !coef_out) {
        set_error("gks_limit: NULL argument");
        return GKS_EINVAL;
    }
    if (!m->cfg.limiter) {
        set_error("gks_limit: the mesh was created with gks_config.limiter = 0");
        return GKS_EINVAL;
    }
    DeviceGuard g(m->device);
    cudaStream_t s = (cudaStream_t)stream;
    gks_status st;
    Work &k = m->wk;
    if ((st = launch_permute(w, k.w, m->d.perm, m->d.T, m->n_tri, 4, true, s)) != GKS_OK) return st;
    if ((st = launch_permute(coef, k.r, m->d.perm, m->d.T, m->n_tri, 20, true, s)) != GKS_OK) return st;
    if ((st = launch_limiter(m, k.w, k.r, s)) != GKS_OK) return st;
    if ((st = launch_permute(k.xl, coef_out, m->d.perm, m->d.T, m->n_tri, 20, false, s)) != GKS_OK) return st;
    if (flags && (st = launch_scatter_flags(m, flags, s)) != GKS_OK) return st;
    return GKS_OK;
}

gks_status gks_flux(gks_mesh *m, const double *w, const double *coef, double dt, double *face_flux, void *stream)
{
    if (!m || !w || !coef || !face_flux || !(dt > 0.0)) {
        set_error("gks_flux: NULL argument or dt <= 0");
        return GKS_EINVAL;
    }
    DeviceGuard g(m->device);
    cudaStream_t s = (cudaStream_t)stream;
    gks_status st;
    Work &k = m->wk;
    GKS_CUDA(cudaMemsetAsync(k.status, 0, sizeof(int32_t) * m->n_case, s));
    if ((st = launch_permute(w, k.w, m->d.perm, m->d.T, m->n_tri, 4, true, s)) != GKS_OK) return st;
    if ((st = launch_permute(coef, k.r, m->d.perm, m->d.T, m->n_tri, 20, true, s)) != GKS_OK) return st;
    if ((st = launch_flux(m, k.w, k.r, dt, nullptr, k.flux, s)) != GKS_OK) return st;
    if ((st = launch_permute(k.flux, face_flux, m->d.fperm, m->d.F, m->n_face, 4, false, s)) != GKS_OK) return st;
    std::vector<int32_t> stat(m->n_case);
    GKS_CUDA(cudaMemcpyAsync(stat.data(), k.status, sizeof(int32_t) * m->n_case, cudaMemcpyDeviceToHost, s));
    GKS_CUDA(cudaStreamSynchronize(s));
    for (int32_t v : stat)
        if (v & kStatusNonPhys) {
            set_error("non-physical state at a Gauss point");
            return GKS_ENONPHYS;
        }
    return GKS_OK;
}

gks_status gks_step(gks_mesh *m, double *w, double *dt_inout, gks_step_info *info, void *stream)
{
    if (!m || !w) {
        set_error("gks_step: NULL argument");
        return GKS_EINVAL;
    }
    if (require_single(m, "gks_step") != GKS_OK) return GKS_EINVAL;
    DeviceGuard g(m->device);
    cudaStream_t s = (cudaStream_t)stream;
    gks_status st;
    // a new step of the case: no status bits, not done (a run may have ended it)
    GKS_CUDA(cudaMemsetAsync(m->wk.status, 0, sizeof(int32_t) * m->n_case, s));
    GKS_CUDA(cudaMemsetAsync(m->wk.done, 0, sizeof(int32_t) * m->n_case, s));
    if ((st = launch_permute(w, m->wk.w, m->d.perm, m->d.T, m->n_tri, 4, true, s)) != GKS_OK) return st;
    double dt = 0.0;
    gks_status res;
    // the CFL step as one launch of the step-loop graph, read back with one
    // synchronisation; a fixed step (or graphs off) takes the host path
    bool graph = false;
    if ((!dt_inout || *dt_inout <= 0.0) && (st = step_graph_launch(m, s, &graph)) != GKS_OK) return st;
    if (graph) {
        if ((st = launch_permute(m->wk.w, w, m->d.perm, m->d.T, m->n_tri, 4, false, s)) != GKS_OK) return st;
        GKS_CUDA(cudaStreamSynchronize(s));
        res = step_graph_results(m, info, &dt);
    } else {
        res = step_internal(m, dt_inout ? *dt_inout : 0.0, s, info, &dt);
        if (res != GKS_OK && res != GKS_ENOCONV && res != GKS_ENONPHYS && res != GKS_ETIMEOUT) return res;
        if ((st = launch_permute(m->wk.w, w, m->d.perm, m->d.T, m->n_tri, 4, false, s)) != GKS_OK) return st;
        GKS_CUDA(cudaStreamSynchronize(s));
    }
    if (dt_inout) *dt_inout = dt;
    return res;
}

namespace gks {
namespace {

constexpr int64_t kCheckEvery = 16;      // loops between the host's looks at the done flags

// Reset the per-case clocks and counters of a run: end times tf (host, n values;
// 0 = no end time), time 0, nothing done, no status, no steps, no iterations.
gks_status run_begin(gks_mesh *m, const double *tf, cudaStream_t s)
{
    Work &k = m->wk;
    const int32_t n = m->n_case;
    GKS_CUDA(cudaMemcpyAsync(k.tfinal, tf, sizeof(double) * n, cudaMemcpyHostToDevice, s));
    GKS_CUDA(cudaMemsetAsync(k.tcase, 0, sizeof(double) * n, s));
    GKS_CUDA(cudaMemsetAsync(k.done, 0, sizeof(int32_t) * n, s));
    GKS_CUDA(cudaMemsetAsync(k.status, 0, sizeof(int32_t) * n, s));
    GKS_CUDA(cudaMemsetAsync(k.nstep, 0, sizeof(int64_t) * n, s));
    GKS_CUDA(cudaMemsetAsync(k.last_dt, 0, sizeof(double) * n, s));
    GKS_CUDA(cudaMemsetAsync(k.iters_acc, 0, sizeof(int64_t) * k.ns, s));
    // tf is host memory that the caller may free on return
    GKS_CUDA(cudaStreamSynchronize(s));
    return GKS_OK;
}

// The step loop on the device state without a host round trip per step: every
// loop takes one step of each case that is not done (CFL step clipped to the
// case's end time, CLS solve, limiter, flux, update), then a case whose status
// bits are set stops and the others advance their clocks.  With graphs on, the
// loop is one launch of a graph whose while node the device ends once every
// case is done or max_steps loops ran; otherwise the host enqueues the steps
// and looks at the done flags every kCheckEvery loops.
gks_status run_steps_async(gks_mesh *m, int64_t max_steps, cudaStream_t s)
{
    Work &k = m->wk;
    const int32_t n = m->n_case;
    gks_status st;
    bool graph = false;
    if (max_steps > 0 && (st = run_graph_launch(m, max_steps, s, &graph)) != GKS_OK) return st;
    if (graph) return GKS_OK;
    std::vector<int32_t> done(n);
    int64_t q = 0;
    while (q < max_steps) {
        const int64_t chunk = std::min<int64_t>(kCheckEvery, max_steps - q);
        for (int64_t r = 0; r < chunk; ++r) {
            if ((st = launch_cfl_dt(m, k.w, k.dt, s)) != GKS_OK) return st;
            if ((st = launch_clip_only(m, s)) != GKS_OK) return st;
            if ((st = cls_solve(m, s, nullptr, nullptr, nullptr)) != GKS_OK) return st;
            if ((st = launch_acc_iters(m, s)) != GKS_OK) return st;
            if (m->cfg.limiter && (st = launch_limiter(m, k.w, k.x, s)) != GKS_OK) return st;
            if ((st = launch_flux(m, k.w, m->cfg.limiter ? k.xl : k.x, 0.0, k.dt, k.flux, s)) != GKS_OK) return st;
            if ((st = launch_update(m, k.w, k.flux, s)) != GKS_OK) return st;
            if ((st = launch_after_step(m, s)) != GKS_OK) return st;
        }
        q += chunk;
        if (q >= max_steps) break;
        GKS_CUDA(cudaMemcpyAsync(done.data(), k.done, sizeof(int32_t) * n, cudaMemcpyDeviceToHost, s));
        GKS_CUDA(cudaStreamSynchronize(s));
        bool all = true;
        for (int32_t c = 0; c < n; ++c) all = all && done[c];
        if (all) break;
    }
    return GKS_OK;
}

// per-case results of a run (host arrays of n values, may be NULL) and the
// iterations summed over systems
gks_status run_end(gks_mesh *m, cudaStream_t s, int64_t *nstep, double *t, double *last_dt, int32_t *status,
                   int64_t *iters)
{
    Work &k = m->wk;
    const int32_t n = m->n_case;
    std::vector<int64_t> ns(n), it(k.ns);
    std::vector<double> tt(n), ld(n);
    std::vector<int32_t> stv(n);
    GKS_CUDA(cudaMemcpyAsync(ns.data(), k.nstep, sizeof(int64_t) * n, cudaMemcpyDeviceToHost, s));
    GKS_CUDA(cudaMemcpyAsync(tt.data(), k.tcase, sizeof(double) * n, cudaMemcpyDeviceToHost, s));
    GKS_CUDA(cudaMemcpyAsync(ld.data(), k.last_dt, sizeof(double) * n, cudaMemcpyDeviceToHost, s));
    GKS_CUDA(cudaMemcpyAsync(stv.data(), k.status, sizeof(int32_t) * n, cudaMemcpyDeviceToHost, s));
    GKS_CUDA(cudaMemcpyAsync(it.data(), k.iters_acc, sizeof(int64_t) * k.ns, cudaMemcpyDeviceToHost, s));
    GKS_CUDA(cudaStreamSynchronize(s));
    // the device-controlled solve graphs counted their launches and work on the
    // device; bring those counters to the host once per run
    flush_solve_counters(m);
    for (int32_t c = 0; c < n; ++c) {
        if (nstep) nstep[c] = ns[c];
        if (t) t[c] = tt[c];
        if (last_dt) last_dt[c] = ld[c];
        if (status) status[c] = stv[c];
    }
    if (iters) {
        int64_t sum = 0;
        for (int64_t v : it) sum += v;
        *iters = sum;
    }
    return GKS_OK;
}

}  // namespace
}  // namespace gks

gks_status gks_run(gks_mesh *m, double *w, double t_final, int64_t max_steps, double steady_tol, gks_run_info *info,
                   void *stream)
{
    if (!m || !w || max_steps < 0) {
        set_error("gks_run: NULL argument or max_steps < 0");
        return GKS_EINVAL;
    }
    if (require_single(m, "gks_run") != GKS_OK) return GKS_EINVAL;
    DeviceGuard g(m->device);
    cudaStream_t s = (cudaStream_t)stream;
    gks_status st, res = GKS_OK;
    Work &k = m->wk;
    if (steady_tol <= 0.0) {
        // no steady residual to watch: the whole loop on the device, one host
        // round trip every few steps
        const double tf = t_final > 0.0 ? t_final : 0.0;
        if ((st = run_begin(m, &tf, s)) != GKS_OK) return st;
        if ((st = launch_permute(w, k.w, m->d.perm, m->d.T, m->n_tri, 4, true, s)) != GKS_OK) return st;
        if ((st = run_steps_async(m, max_steps, s)) != GKS_OK) return st;
        if ((st = launch_permute(k.w, w, m->d.perm, m->d.T, m->n_tri, 4, false, s)) != GKS_OK) return st;
        int64_t nst = 0, its = 0;
        double tr = 0.0, ld = 0.0;
        int32_t stat = 0;
        if ((st = run_end(m, s, &nst, &tr, &ld, &stat, &its)) != GKS_OK) return st;
        res = code_of(stat);
        if (info) {
            info->steps = nst;
            info->t = tr;
            info->last_dt = ld;
            info->gmres_iters = its;
            info->steady_res = 0.0;
            info->status = res;
        }
        return res;
    }
    GKS_CUDA(cudaMemsetAsync(k.status, 0, sizeof(int32_t) * m->n_case, s));
    if ((st = launch_permute(w, k.w, m->d.perm, m->d.T, m->n_tri, 4, true, s)) != GKS_OK) return st;
    double t = 0.0, last_dt = 0.0, res0 = -1.0, sres = 0.0;
    int64_t steps = 0, iters = 0;
    while (steps < max_steps) {
        double dt_fixed = 0.0;
        if (t_final > 0.0) {
            if (t >= t_final * (1.0 - 1e-14)) break;
            if ((st = launch_cfl_dt(m, k.w, k.dt, s)) != GKS_OK) return st;
            GKS_CUDA(cudaMemcpyAsync(&k.h_scal[6], k.dt, sizeof(double), cudaMemcpyDeviceToHost, s));
            GKS_CUDA(cudaStreamSynchronize(s));
            dt_fixed = std::fmin(k.h_scal[6], t_final - t);
        }
        if (steady_tol > 0.0)
            GKS_CUDA(cudaMemcpyAsync(k.w_old, k.w, sizeof(double) * 4 * m->d.T, cudaMemcpyDeviceToDevice, s));
        gks_step_info si;
        double dt = 0.0;
        res = step_internal(m, dt_fixed, s, &si, &dt);
        if (res != GKS_OK) break;
        ++steps;
        t += dt;
        last_dt = dt;
        for (int v = 0; v < 4; ++v) iters += si.iters[v];
        if (steady_tol > 0.0) {
            if ((st = launch_steady_partial(m, s)) != GKS_OK) return st;
            GKS_CUDA(cudaMemcpyAsync(k.h_scal, k.scal, sizeof(double) * 4, cudaMemcpyDeviceToHost, s));
            GKS_CUDA(cudaStreamSynchronize(s));
            double r = 0.0;
            for (int v = 0; v < 4; ++v) r = std::fmax(r, std::sqrt(k.h_scal[v]) / dt);
            if (res0 < 0.0) res0 = r > 0.0 ? r : 1.0;
            sres = r / res0;
            if (sres < steady_tol) break;
        }
    }
    if ((st = launch_permute(k.w, w, m->d.perm, m->d.T, m->n_tri, 4, false, s)) != GKS_OK) return st;
    GKS_CUDA(cudaStreamSynchronize(s));
    if (info) {
        info->steps = steps;
        info->t = t;
        info->last_dt = last_dt;
        info->gmres_iters = iters;
        info->steady_res = sres;
        info->status = res;
    }
    return res;
}

gks_status gks_batch_run(gks_mesh *m, double *w, const double *t_final, int64_t max_steps, double *t_reached,
                         int32_t *case_status, gks_batch_info *info, void *stream)
{
    if (!m || !w || max_steps < 0) {
        set_error("gks_batch_run: NULL argument or max_steps < 0");
        return GKS_EINVAL;
    }
    DeviceGuard g(m->device);
    cudaStream_t s = (cudaStream_t)stream;
    Work &k = m->wk;
    const int32_t n = m->n_case;
    gks_status st;
    std::vector<double> tf(n, 0.0);
    if (t_final)
        for (int32_t c = 0; c < n; ++c) tf[c] = t_final[c];
    if ((st = run_begin(m, tf.data(), s)) != GKS_OK) return st;
    if ((st = launch_permute(w, k.w, m->d.perm, m->d.T, m->n_tri, 4, true, s)) != GKS_OK) return st;
    // a case that fails stops advancing; the others go on
    if ((st = run_steps_async(m, max_steps, s)) != GKS_OK) return st;
    if ((st = launch_permute(k.w, w, m->d.perm, m->d.T, m->n_tri, 4, false, s)) != GKS_OK) return st;
    std::vector<int64_t> nst(n);
    std::vector<double> tr(n);
    std::vector<int32_t> stat(n);
    int64_t iters = 0;
    if ((st = run_end(m, s, nst.data(), tr.data(), nullptr, stat.data(), &iters)) != GKS_OK) return st;
    int64_t steps = 0;
    int32_t nfail = 0, ndone = 0;
    for (int32_t c = 0; c < n; ++c) {
        const int32_t cs = code_of(stat[c]);
        if (t_reached) t_reached[c] = tr[c];
        if (case_status) case_status[c] = cs;
        nfail += cs != GKS_OK;
        ndone += cs == GKS_OK && tf[c] > 0.0 && tr[c] >= tf[c] * (1.0 - 1e-14);
        // a failing case's step counts in the loop too
        steps = std::max<int64_t>(steps, nst[c] + (cs != GKS_OK ? 1 : 0));
    }
    if (info) {
        info->steps = steps;
        info->gmres_iters = iters;
        info->n_failed = nfail;
        info->n_finished = ndone;
    }
    return GKS_OK;
}

gks_status gks_profile_begin(gks_mesh *m, int32_t class_mask)
{
    if (!m || class_mask < 0 || class_mask >= (1 << kProfClasses)) {
        set_error("gks_profile_begin: bad argument");
        return GKS_EINVAL;
    }
    flush_solve_counters(m);                        // work of earlier calls stays out
    m->prof.mask = class_mask;
    m->prof.used = 0;
    m->prof.cls.clear();
    m->prof.arnoldi = m->prof.arnoldi_jsum = m->prof.precond = m->prof.residuals = 0;
    return GKS_OK;
}

gks_status gks_profile_end(gks_mesh *m, gks_profile *out)
{
    if (!m || !out) {
        set_error("gks_profile_end: NULL argument");
        return GKS_EINVAL;
    }
    DeviceGuard g(m->device);
    std::memset(out, 0, sizeof(*out));
    flush_solve_counters(m);
    gks_profiler &p = m->prof;
    for (size_t q = 0; q < p.cls.size(); ++q) {
        GKS_CUDA(cudaEventSynchronize(p.events[2 * q + 1]));
        float ms = 0.0f;
        GKS_CUDA(cudaEventElapsedTime(&ms, p.events[2 * q], p.events[2 * q + 1]));
        out->ms[p.cls[q]] += ms;
        out->n[p.cls[q]] += 1;
    }
    out->arnoldi = p.arnoldi;
    out->arnoldi_jsum = p.arnoldi_jsum;
    out->precond = p.precond;
    out->residuals = p.residuals;
    p.mask = 0;
    p.used = 0;
    p.cls.clear();
    return GKS_OK;
}

int64_t gks_launch_count(void) { return g_launches.load(); }

gks_status gks_point_flux(int64_t n, const double *wl, const double *wr, double dt, const gks_config *cfg, double *out,
                          void *stream)
{
    if (n < 0 || (n > 0 && (!wl || !wr || !out)) || !(dt > 0.0)) {
        set_error("gks_point_flux: bad argument");
        return GKS_EINVAL;
    }
    gks_config c;
    if (cfg) c = *cfg;
    else gks_config_default(&c);
    gks_status st = check_config(c);
    if (st != GKS_OK) return st;
    return launch_point_flux(n, wl, wr, dt, c, out, nullptr, (cudaStream_t)stream);
}

}  // extern "C"
