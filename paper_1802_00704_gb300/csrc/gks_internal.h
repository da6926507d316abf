// Internal declarations of the GB300 gas-kinetic library (not installed).
//
// A handle holds one or more independent cases (meshes).  Their cells are
// stored one case after the other, each case in its own RCM order and padded
// to a whole number of kBlock-cell blocks, so that every block of a cell kernel
// belongs to exactly one case and every reduction is a segmented one.  A
// single mesh is the one-case instance (no padding).
#pragma once

#include <cuda_fp16.h>
#include <cuda_runtime.h>

#include <atomic>
#include <cstdint>
#include <string>
#include <vector>

#include "../../include/gks.h"

namespace gks {

constexpr int kBlock = 256;          // cells per block of the cell kernels (and padding unit)
constexpr int kMaxRestart = 64;      // upper bound on gmres_m

void set_error(const char *fmt, ...);

#define GKS_CUDA(call)                                                                    \
    do {                                                                                  \
        cudaError_t e_ = (call);                                                          \
        if (e_ != cudaSuccess) {                                                          \
            ::gks::set_error("%s failed: %s (%s:%d)", #call, cudaGetErrorString(e_),       \
                             __FILE__, __LINE__);                                         \
            return GKS_ECUDA;                                                             \
        }                                                                                 \
    } while (0)

// Process-wide count of kernel launches issued by the library.
extern std::atomic<int64_t> g_launches;
inline void note_launch() { g_launches.fetch_add(1, std::memory_order_relaxed); }

// Kernel classes timed by the optional CUDA-event profiler.
enum : int {
    kProfFlux = 0, kProfSpmv = 1, kProfIlu = 2, kProfOrth = 3, kProfUpdate = 4, kProfResid = 5, kProfCorr = 6,
    kProfCtl = 7, kProfClasses = GKS_PROF_CLASSES
};

// Device status bits (per case words the kernels OR into).
enum : int { kStatusNonPhys = 1, kStatusNoConv = 2, kStatusTimeout = 4 };

// GMRES control words, ctl[field * ns + system] with system = case * 4 + variable.
enum : int { kCtlActive = 0, kCtlRunning = 1, kCtlJv = 2, kCtlIters = 3, kCtlFields = 4 };

// Device data, all in internal (per-case RCM, padded) cell order.
struct DeviceMesh {
    int64_t T = 0, F = 0;            // internal cells (with padding) and faces
    int32_t ncase = 1;
    int32_t *blk_case = nullptr;     // [T / kBlock rounded up] case of each cell block
    int32_t *case_blk = nullptr;     // [ncase + 1] first cell block of each case
    int32_t *face_case = nullptr;    // [F] case of each face
    // cells
    double *area = nullptr, *inv_area = nullptr, *h = nullptr, *mxx = nullptr, *mxy = nullptr, *myy = nullptr;
    double *inrad = nullptr;         // padding cells: +inf (never limit the step)
    int32_t *nb = nullptr;           // [3][T] neighbour (internal index) or -1
    double *alpha = nullptr;         // [3][T] w^2 h_i / h_j
    double *ex = nullptr, *ey = nullptr;  // [3][T] centroid offsets of j in i's frame (0 when k_i = 1)
    // global normal equations (cls_global, Eq. (33)): the reverse slot's coefficients,
    // alpha_ji and i's centroid in j's frame (0 when k_j = 1); NULL otherwise
    double *alr = nullptr, *exr = nullptr, *eyr = nullptr;  // [3][T]
    // second-derivative equations (cls_M = 2): beta of the diagonal coupling of the
    // unknowns 3..5 with the neighbour's (plus the reverse one in the global system)
    double *bdg = nullptr;           // [3][T]; with alr.. allocated for either option (zeros if unused)
    double *a0 = nullptr;            // [3][5][T] weighted row 0 of A_ij (right-hand side)
    float *a0p = nullptr;            // [30][T] FP32 pairs of a0 (the 15 high parts, then the low parts)
    double *D = nullptr;             // [15][T] symmetric diagonal block, upper triangle row-major
    double *P = nullptr;             // [25][T] inverse of the ILU(0) diagonal block, row-major
    // FP32 copies of the operator and factors (mixed precision)
    float *D32 = nullptr, *P32 = nullptr, *alpha32 = nullptr, *ex32 = nullptr, *ey32 = nullptr;
    float *alr32 = nullptr, *exr32 = nullptr, *eyr32 = nullptr, *bdg32 = nullptr;
    // FP16 copies of the ILU(0) factors for the FP32 preconditioner (ilu_fp16;
    // NULL when not asked for or a value is outside FP16's range)
    __half *P16 = nullptr, *alpha16 = nullptr, *ex16 = nullptr, *ey16 = nullptr;
    __half *alr16 = nullptr, *exr16 = nullptr, *eyr16 = nullptr, *bdg16 = nullptr;
    float *ih32 = nullptr;           // [T] 1 / h_i (mixed flux)
    // FP32 pairs (hi, lo) of the geometry for the double-FP32 flux (mixed precision)
    float *m2 = nullptr;             // [6][T] mxx, mxy, myy, then their low parts
    float *gl2 = nullptr, *gr2 = nullptr;  // [8][F] the 4 rows of gl / gr, then their low parts
    float *fn2 = nullptr;            // [4][F] nx, ny, then their low parts
    float *flen2 = nullptr;          // [2][F] half the face length (Gauss weight 1/2), its low part
    // the operator as FP32 pairs hi + lo for the double-FP32 refinement residual
    // (mixed mode with an FP32 basis; NULL when a value is outside the pair range)
    float *D2 = nullptr;             // [30][T] the 15 diagonal-block values, then their low parts
    float *S2 = nullptr;             // [18][T] sa, sa dx, sa dy per neighbour slot (sa = -alpha, 0
                                     //         without neighbour), then their low parts
    float *SR2 = nullptr;            // [18][T] the same for the reverse slots (global normal equations)
    float *SB2 = nullptr;            // [6][T] -beta per slot, then the low parts (second-derivative equations)
    double *ox = nullptr, *oy = nullptr;  // [3][T] neighbour centroid in i's scaled frame (limiter)
    int32_t *kord = nullptr;         // [T] reconstruction order k_i of Eq. (28) (limiter)
    int32_t *cf = nullptr;           // [3][T] (face << 1) | side, -1 unused
    int32_t *perm = nullptr;         // [T] internal -> caller cell (-1 for padding)
    int32_t *lvl_lo = nullptr;       // rows sorted by forward level
    int32_t *lvl_up = nullptr;       // rows sorted by backward level
    // faces (internal order)
    int32_t *fl = nullptr, *fr = nullptr, *ftag = nullptr;
    int32_t *fperm = nullptr;        // [F] internal -> caller face
    double *fnx = nullptr, *fny = nullptr, *flen = nullptr;
    double *gl = nullptr;            // [4][F] Gauss points in l's scaled frame: dx0 dy0 dx1 dy1
    double *gr = nullptr;            // [4][F] Gauss points in r's scaled frame
    double *bc = nullptr;            // [4][F]
};

struct Work {
    int m = 0;                       // restart length in use (the autotuner may lower it)
    int m_alloc = 0;                 // restart length the Krylov buffers were sized for
    int nblk = 0;                    // cell blocks (kBlock cells each)
    int sm_count = 0;                // multiprocessors of the handle's device
    int ns = 4;                      // GMRES systems: 4 per case
    double *w = nullptr;             // [4][T] state (internal order)
    double *w_old = nullptr;         // [4][T]
    double *x = nullptr;             // [20][T] CLS coefficients (warm start)
    double *x_prev = nullptr;        // [20][T] the solution before (extrapolated warm start)
    double *x_prev2 = nullptr;       // [20][T] the one before that
    int64_t *nsolve = nullptr;       // [1] solves since creation or the last warm-start reset,
                                     //     counted on the device: its parity says which history
                                     //     buffer holds the latest solution, its value the order
                                     //     of the extrapolation (no host state, so a step can repeat
                                     //     inside a graph)
    double *xl = nullptr;            // [20][T] limited coefficients (limiter on)
    float *x32 = nullptr;            // [20][T] FP32 copy of the coefficients the mixed flux reads
                                     //         (the first half of x2)
    float *x2 = nullptr;             // [40][T] FP32 pairs of the coefficients: x32, then the low parts
    float *w2 = nullptr;             // [8][T] FP32 pairs of the state: hi, then lo
    int32_t *lflag = nullptr;        // [T] 0 untouched, 1 limited, 2 reset to the average
    double *b = nullptr, *r = nullptr, *t2 = nullptr, *t3 = nullptr;  // [20][T]
    float *t2_32 = nullptr, *t3_32 = nullptr;  // [20][T] FP32 preconditioner work
    float *r32 = nullptr;            // [20][T] FP32 copy of the preconditioner's source (sweeps)
    double *V = nullptr;             // [(m+1)][20][T] Krylov basis, unnormalised: v_k = V_k / vn_k
    float *V32 = nullptr;            // the same stored in FP32 (mixed mode with basis_fp32; V unused)
    double *Z = nullptr;             // [m][20][T] M^{-1} V_k (FP64 path)
    float *Z32 = nullptr;            // [m][20][T] M^{-1} V_k (mixed path)
    double *flux = nullptr;          // [4][F]
    double *part = nullptr;          // [nblk][4][m+2] partial sums per cell block
    double *dpart = nullptr;         // [nblk][4] partial minima / sums
    // small GMRES state (device), one row per system
    double *H = nullptr;             // [ns][m+1][m]  (Givens-rotated Hessenberg)
    double *cs = nullptr, *sn = nullptr;  // [ns][m]
    double *g = nullptr;             // [ns][m+1]
    double *y = nullptr;             // [ns][m]
    float *y32 = nullptr;            // [ns][m] FP32 copy of y (mixed mode)
    double *hcol = nullptr;          // [ns][m+2] raw sums <V_k, u> of the current column, then |V_{j+1}|
    double *hco = nullptr;           // [ns][m+2] Gram-Schmidt coefficients <V_k, u> / vn_k^2
    double *vn = nullptr;            // [ns][m+1] norms vn_k of the stored basis vectors
    double *bnorm = nullptr, *beta = nullptr;  // [ns]
    int32_t *ctl = nullptr;          // [kCtlFields][ns]
    int32_t *sexp = nullptr;         // [2][ns] FP32 basis: first basis vector stored as 2^-e r; e of the
                                     //         current cycle, then that of the next residual
    int32_t *flags = nullptr;        // [4]: any active, any running, all cases done
    double *dt = nullptr;            // [ncase] step of each case (0: case inactive)
    double *tcase = nullptr;         // [ncase] time reached
    double *tfinal = nullptr;        // [ncase] end time (<= 0: none)
    int32_t *done = nullptr;         // [ncase] case finished or stopped
    double *scal = nullptr;          // [8] misc device scalars
    int32_t *status = nullptr;       // [ncase] status bits
    // the asynchronous step loop (gks_run, gks_batch_run): per-case steps taken,
    // last step, and per-system GMRES iterations summed on the device
    int64_t *nstep = nullptr;        // [ncase]
    double *last_dt = nullptr;       // [ncase]
    int64_t *iters_acc = nullptr;    // [ns]
    // the device-controlled step loop (one graph launch per run): loops of the
    // current launch, the launch's loop limit, loops over all launches
    int64_t *run_ctl = nullptr;      // [4]
    // sync-free exact ILU solves (GKS_PC_ILU_EXACT): per-row ready tags, and
    // the epoch, the forward and backward block tickets and the sticky wait error
    int32_t *sf_flag = nullptr;      // [T]
    int32_t *sf_ctl = nullptr;       // [4]
    // pinned host mirrors
    int32_t *h_flags = nullptr;      // [4]
    double *h_scal = nullptr;        // [8]
    // gks_step's results when it runs as one launch of the step-loop graph:
    // beta, |b| per variable and the step; iterations per variable and status
    double *h_step = nullptr;        // [9]
    int32_t *h_stepi = nullptr;      // [5]
};

// CUDA graphs of the fixed launch sequences of the CLS solve (the start, one
// per Arnoldi index, the restart), captured on first use on a private stream
// and replayed on the caller's stream; rebuilt when a knob baked into their
// kernel arguments changes.
//
// The whole solve is also built as one graph with device-side control: a
// while node over the GMRES cycles whose body holds the Arnoldi indices as
// nested if nodes, their conditions set by one-block kernels from the
// per-system masks, so a solve needs no host round trip.  Device counters
// (ctr) record how often each part ran, for the launch and work counts.
constexpr int kCtrCycles = kMaxRestart;             // ctr[j]: runs of Arnoldi index j; then cycles
constexpr int kCtrGuard = kMaxRestart + 1;          // cycles of the current solve (loop guard)
constexpr int kCtrRun = kMaxRestart + 2;            // loops of the device-controlled step loop
constexpr int kCtrLen = kMaxRestart + 3;
struct SolveGraphs {
    cudaStream_t cap = nullptr;
    std::vector<cudaGraphExec_t> iter;
    std::vector<int64_t> iter_launches;
    cudaGraphExec_t start = nullptr, restart = nullptr;
    int64_t start_launches = 0, restart_launches = 0;
    int32_t sweeps = -1, sweeps_bwd = -2, fuse = -1, precond = -1, maxit = -1, pairs = -1, spmv_dots = -1;
    double eta = -1.0, rtol = -1.0;
    bool disabled = false;                          // a capture failed: launch directly
    // device-controlled whole solve
    cudaGraphExec_t whole = nullptr;
    bool whole_failed = false;                      // building it failed: per-part graphs
    int64_t whole_start_launches = 0, whole_cycle_launches = 0;
    std::vector<int64_t> whole_iter_launches;       // per Arnoldi index
    int64_t *ctr = nullptr;                         // [kCtrLen] device counters
    int64_t *h_ctr = nullptr;                       // pinned mirror
    std::vector<int64_t> ctr_seen;                  // counts already added to the host totals
    // the step loop of gks_run / gks_batch_run as one graph with device control
    // (a while node over the steps, the whole solve nested in its body)
    cudaGraphExec_t run = nullptr;
    bool run_failed = false;                        // building it failed: the host loop from now on
    gks_config run_cfg{};                           // configuration it was built for
    int64_t run_loop_launches = 0;                  // kernels per loop outside the solve's cycles
    int64_t *h_run = nullptr;                       // pinned: the loop limit of the next launch
};
void destroy_graph_execs(SolveGraphs *g);
// Add the counts of the device-controlled solves run so far to the launch and
// work totals (synchronises the device).
void flush_solve_counters(gks_mesh *m);

}  // namespace gks

struct gks_profiler {
    int mask = 0;                                   // bit c: time class c
    std::vector<cudaEvent_t> events;                // pool
    size_t used = 0;
    std::vector<int> cls;                           // class of each start/stop pair
    int64_t arnoldi = 0, arnoldi_jsum = 0, precond = 0, residuals = 0;  // work counters
};

struct gks_mesh {
    gks_config cfg{};
    gks_profiler prof;
    int device = 0;
    int32_t n_case = 1;
    int64_t n_tri = 0, n_face = 0, n_bface = 0, n_k1 = 0, nnzb = 0, bandwidth = 0;  // caller totals
    std::vector<int64_t> case_tri, case_face;      // caller sizes per case
    std::vector<int32_t> lvl_lo_ptr, lvl_up_ptr;   // level offsets (host)
    gks::DeviceMesh d;
    gks::Work wk;
    int64_t device_bytes = 0;
    std::vector<void *> allocations;
    gks::SolveGraphs *graphs = nullptr;
    int64_t flux_ws_grid = 0;                      // blocks of the persistent flux kernel
    int32_t flux_ws_key = -1;                      // ... for this variant
};

namespace gks {

// One case as given to the ABI (host arrays).
struct CaseIn {
    const double *nodes;
    int64_t n_nodes;
    const int32_t *tris;
    int64_t n_tri;
    const int32_t *faces;
    const double *face_shift;
    int64_t n_face;
    const double *bc_state;
};

// set-up (gks_setup.cu)
gks_status build_batch(gks_mesh *m, const CaseIn *cases, int32_t n_cases);
void free_mesh(gks_mesh *m);

// CLS reconstruction (gks_cls.cu): rhs from m->wk.w, solution in m->wk.x.
// Per system (case * 4 + variable, may be NULL): iterations, relative residuals;
// *converged = 1 if every active system met the tolerance.
gks_status cls_solve(gks_mesh *m, cudaStream_t s, int32_t *iters, double *relres, int32_t *converged);
// The step loop of a run (CFL step clipped to the end times, CLS solve, limiter,
// flux, update, per-case clocks) for at most max_steps loops as one launch of a
// graph with device-side control; *used = false when graphs are off, the
// profiler is on or the graph could not be built (the caller's host loop then
// runs the steps).
gks_status run_graph_launch(gks_mesh *m, int64_t max_steps, cudaStream_t s, bool *used);

// flux and update (gks_flux.cu)
gks_status launch_flux(gks_mesh *m, const double *w, const double *x, double dt_const, const double *dt_dev,
                       double *flux, cudaStream_t s);
gks_status launch_update(gks_mesh *m, double *w, const double *flux, cudaStream_t s);
// the mixed flux with its FP64-accuracy part in FP32 pairs (gks_flux_df.cu);
// launch shapes (threads per block, blocks per SM, i.e. the register budget)
// the autotuner may choose from for the flux without the Prandtl correction
// and with mean interface slopes
constexpr int kFluxDfVariants = 3;
gks_status launch_flux_df(gks_mesh *m, const double *w, const double *x, double dt_const, const double *dt_dev,
                          double *flux, cudaStream_t s);
gks_status launch_point_flux_df(int64_t n, const double *wl, const double *wr, double dt, const gks_config &cfg,
                                double *out, int32_t *status, cudaStream_t s);
gks_status launch_cfl_dt(gks_mesh *m, const double *w, double *dt_dev, cudaStream_t s);
gks_status launch_point_flux(int64_t n, const double *wl, const double *wr, double dt, const gks_config &cfg,
                             double *out, int32_t *status, cudaStream_t s);
// gather (internal[v][i] = caller[v][perm[i]], padding untouched) or scatter
gks_status launch_permute(const double *src, double *dst, const int32_t *perm, int64_t n, int64_t ncaller, int nvar,
                          bool gather, cudaStream_t s);
gks_status launch_steady_partial(gks_mesh *m, cudaStream_t s);
// per-case step control for runs: dt = min(cfl dt, t_final - t) or 0 when done; t += dt
gks_status launch_clip_dt(gks_mesh *m, cudaStream_t s);
// the asynchronous step loop: dt of each case clipped to its end time (0 once
// the case is done, time not advanced yet); after the step, a case whose status
// is set stops, the others advance their time and step count
gks_status launch_clip_only(gks_mesh *m, cudaStream_t s);
gks_status launch_after_step(gks_mesh *m, cudaStream_t s);
gks_status launch_acc_iters(gks_mesh *m, cudaStream_t s);
// shock detector + DWBAP limiter: m->wk.xl from m->wk.x (gks_limiter.cu)
gks_status launch_limiter(gks_mesh *m, const double *w, const double *x, cudaStream_t s);
// caller-ordered copy of the limiter flags of the last launch_limiter
gks_status launch_scatter_flags(gks_mesh *m, int32_t *flags_out, cudaStream_t s);

// optional CUDA-event timing of one kernel class (no-op unless enabled)
int prof_start(gks_mesh *m, int cls, cudaStream_t s);
void prof_stop(gks_mesh *m, int slot, cudaStream_t s);

}  // namespace gks
