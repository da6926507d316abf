/*
 * gks.h -- C ABI of the GB300 (sm_103a) implementation of one explicit step of
 * the third-order gas-kinetic scheme with compact least-squares (CLS)
 * reconstruction on unstructured triangular grids
 * (J. Li, C. Zhong, C. Zhuo, "A third order gas-kinetic scheme for
 * unstructured grid", arXiv:1802.00704).
 *
 * One step (Eq. (6), a single stage):
 *   1. time step from a CFL condition (not stated in the paper; see gks_cfl_dt);
 *   2. CLS reconstruction (Sec. III.A, Eqs. (16)-(29)): per cell a quadratic
 *      zero-mean polynomial (k = 2, linear k = 1 at boundary cells, Eq. (28))
 *      whose coefficients solve the sparse block system of the per-cell
 *      least-squares normal equations (Eqs. (32)-(33)); solved by GMRES with an
 *      ILU(0) preconditioner on a Reverse-Cuthill-McKee order (Sec. III.B);
 *   3. third-order BGK flux (Sec. II.B, Eqs. (8)-(15)) at two Gauss points per
 *      face (Eq. (7)), integrated analytically over [0, dt];
 *   4. conservative update of the cell averages (Eq. (6)).
 *
 * Conventions
 *  - Every array argument documented as "device" is a pointer to device
 *    memory owned by the caller; "host" arrays are read during the call only.
 *    The library keeps no pointer to caller memory after a call returns.
 *  - Cell and face numbering in every argument is the caller's (the order of
 *    the arrays given to gks_mesh_create).  The library stores its data in RCM
 *    order and permutes on the way in and out.
 *  - Cell-average arrays w are float64 SoA [4][n_tri]: rho, rho*u, rho*v, E.
 *  - Reconstruction coefficients are float64 [4][5][n_tri]: variable, basis
 *    index l = 1..5 of Eq. (19) stored at 0..4, cell.  At cells with k = 1
 *    basis indices 3..5 are zero.
 *  - Face fluxes are float64 [4][n_face]: int_0^dt of the Gauss-summed flux
 *    (Eq. (7)) times the face length, signed along the normal from cell_l to
 *    cell_r, in the global frame.
 *  - `stream` is a cudaStream_t (NULL: the legacy default stream).  Calls are
 *    stream-ordered; where a call returns host-visible results (info structs,
 *    dt_out) it synchronises `stream` before returning.
 *  - A mesh handle must not be used from two host threads or two streams at
 *    once.  No C++ exception crosses this ABI.
 *  - Errors: every call returns a gks_status; gks_last_error() gives a
 *    thread-local message for the last failing call.  Argument errors are
 *    detected before any device work is queued.  Numerical failures
 *    (non-physical state, GMRES not converged) are detected on the device and
 *    reported by the calls that read back an info struct.
 */
#ifndef GKS_H
#define GKS_H

#include <stdint.h>

#if defined(__GNUC__)
#define GKS_EXPORT __attribute__((visibility("default")))
#else
#define GKS_EXPORT
#endif

#ifdef __cplusplus
extern "C" {
#endif

typedef enum gks_status {
    GKS_OK = 0,
    GKS_EINVAL = 1,        /* bad argument (sizes, indices, pointers, config)        */
    GKS_ENOMEM = 2,        /* device or host allocation failed                        */
    GKS_ECUDA = 3,         /* a CUDA runtime call failed                              */
    GKS_ENOCONV = 4,       /* GMRES reached gmres_maxit before gmres_rtol             */
    GKS_ENONPHYS = 5,      /* rho <= 0 or p <= 0 at a Gauss point or a cell           */
    GKS_ETIMEOUT = 6,      /* a bounded device wait gave up                           */
    GKS_EUNSUPPORTED = 7   /* option not implemented                                  */
} gks_status;

/* Boundary tags of a face (column 4 of the faces array). */
enum {
    GKS_BC_INTERIOR = 0,   /* two cells                                               */
    GKS_BC_PERIODIC = 1,   /* two cells; face_shift moves cell_r next to cell_l        */
    GKS_BC_DIRICHLET = 2,  /* ghost = bc_state (conservative), zero derivatives       */
    GKS_BC_OUTFLOW = 3,    /* ghost = interior state and derivatives                  */
    GKS_BC_SLIP = 4,       /* ghost = mirror image (normal momentum reversed)         */
    GKS_BC_NOSLIP = 5      /* ghost: velocity reflected about the wall velocity,
                              temperature about the wall temperature; bc_state =
                              (u_wall, v_wall, T_wall, 0), T = p / rho               */
};

/* Preconditioner of the CLS GMRES. */
enum {
    GKS_PC_ILU_EXACT = 0,  /* block ILU(0) on the RCM order with exact triangular
                              solves (Sec. III.B as written), each one launch: a row
                              waits for its lower (upper) neighbours' ready flags and
                              rows are taken in RCM order by block tickets, so a
                              block only waits on blocks that already run (a
                              sync-free level schedule); every wait is bounded
                              (1 s), and a wait that gives up ends the step with
                              GKS_ETIMEOUT                                            */
    GKS_PC_ILU_SWEEP = 1,  /* the same ILU(0) factors, each triangular solve applied
                              by ilu_sweeps block-Jacobi sweeps (fully parallel)     */
    GKS_PC_BJACOBI = 2,    /* block-diagonal (cell) inverse only                      */
    GKS_PC_ILU_LEVELS = 3  /* the exact solves of GKS_PC_ILU_EXACT launched level by
                              level (one launch per level of the RCM graph); the
                              same results bit for bit                               */
};

enum { GKS_FP64 = 0, GKS_MIXED = 1 };

typedef struct gks_config {
    double gamma;          /* ratio of specific heats; K = 2/(gamma-1) - 2 (Eq. (3)) */
    double cfl;            /* CFL number                                              */
    double mu;             /* dynamic viscosity; 0: inviscid collision time Eq. (39),
                              > 0: viscous collision time Eq. (40)                    */
    double cls_w;          /* derivative weight w of Eq. (29) (paper: 0.3)             */
    int32_t gmres_m;       /* GMRES restart length (<= 64)                             */
    int32_t gmres_maxit;   /* iteration cap per variable and reconstruction            */
    double gmres_rtol;     /* ||b - A x||_2 <= gmres_rtol ||b||_2                       */
    int32_t precision;     /* GKS_FP64: everything in FP64.  GKS_MIXED: the GMRES
                              operator and ILU(0) applications in FP32 inside FP64
                              iterative refinement (FP64 residual, Arnoldi and
                              Givens); the flux's interface state, collision time,
                              time integrals and zeroth-order terms in double-FP32
                              or FP64 (flux_lead) and its slope-carrying terms in
                              FP32; FP64 update                                     */
    int32_t precond;       /* GKS_PC_*                                                 */
    int32_t ilu_sweeps;    /* sweeps per triangular solve for GKS_PC_ILU_SWEEP         */
    int32_t tau2_exact;    /* 0: c4, c5, c6 exactly as printed in Eq. (13);
                              1: with the 2 tau^2 (1 - e^{-t/tau}) term that the exact
                              time integral of Eq. (8) carries                          */
    int32_t limiter;       /* 1: shock detector (Eq. (37)) and DWBAP limiter (Eqs.
                              (34)-(36)) on the reconstruction before the flux; 2: the
                              detector with first order (cell average) in the cells
                              it flags (robust mode for density ratios near 10; not
                              in the paper)                                           */
    int32_t basis_fp32;    /* mixed precision only: 1 stores the Krylov basis in FP32
                              (dot products, updates, norms and Givens stay FP64)     */
    int32_t warm_extrap;   /* initial guess of each solve: 0 the last solution x_{n-1};
                              1 its linear extrapolation 2 x_{n-1} - x_{n-2}; 2 the
                              quadratic one 3 x_{n-1} - 3 x_{n-2} + x_{n-3} (as many
                              past solutions as exist); the same tolerance is met,
                              in fewer iterations when the flow changes smoothly      */
    int32_t second_order;  /* 1: second-order variant, k_i = 1 (linear CLS
                              reconstruction) for every cell (the paper's second- vs
                              third-order comparison, Sec. IV)                        */
    int32_t no_graphs;     /* how the CLS solve and the step loop are launched (same
                              kernels, same order, same results): 0 one CUDA graph per
                              solve whose while and if nodes take the GMRES cycle and
                              Arnoldi decisions on the device (no host round trip),
                              and gks_run / gks_batch_run (without a steady tolerance)
                              as one graph launch whose while node over the steps,
                              with the solve nested in its body, ends on the device
                              once every case is done or max_steps loops ran; 1 the
                              kernels one by one, the host reading the stop flags
                              after every Arnoldi step and the done flags every 16
                              steps; 2 as 1 but replaying a graph per solve part     */
    int32_t limit_char;    /* 1: the DWBAP limiter works on characteristic variables
                              (eigenvectors of the Euler flux Jacobian at the cell
                              average, Sec. IV.B) instead of conservative ones        */
    double inner_rtol;     /* mixed precision: an inner FP32 GMRES cycle stops once its
                              residual estimate has dropped by this factor (0 < r < 1,
                              default 1e-6); the next FP64 residual then restarts it   */
    double prandtl;        /* Prandtl number (> 0, default 1 = the BGK model's own):
                              != 1 rescales the heat flux relative to the interface
                              velocity by 1/Pr in the energy flux (not in the paper)  */
    int32_t slope0_mode;   /* derivatives of the interface equilibrium W0 (the paper
                              defers their construction to its references, Sec. II.B):
                              0 the mean of the left and right reconstructed
                              derivatives (default); 1 kinetic weighting, the
                              half-space moments rho_l <psi g_l'/g_l>_{u>0} +
                              rho_r <psi g_r'/g_r>_{u<0} of the derivatives of the two
                              distributions                                            */
    int32_t ilu_fp16;      /* 1 (GKS_MIXED only): the FP32 preconditioner reads its ILU(0)
                              factors (block inverses, off-diagonal coefficients) from
                              FP16 copies, FP32 arithmetic; a fixed preconditioner, so
                              the solution meets the same tolerance; kept in FP32 when
                              a factor is outside FP16's normal range                  */
    int32_t cls_global;    /* 1: the CLS system is the global normal equations of all
                              cells' equations together, C^T C u = C^T b (Eq. (33),
                              symmetric positive definite); 0 (default): each cell's
                              own least-squares equations (non-symmetric), the reading
                              that suits GMRES with ILU(0) (Sec. III.B)                */
    int32_t cls_M;         /* highest derivative order of the CLS equations of Eq. (29)
                              (M <= k): 1 (default) value and first derivatives;
                              2 also the second derivatives (w h_i)^2 of quadratic
                              cells; 0 the values only, which needs the second-order
                              variant (k_i = 1) and two face neighbours per cell       */
    int32_t ilu_sweeps_bwd; /* GKS_PC_ILU_SWEEP: sweeps of the backward (upper) relation;
                              -1 (default) the same as ilu_sweeps, 0..8 otherwise; a
                              fixed preconditioner either way                          */
    int32_t ilu_fuse_first; /* GKS_PC_ILU_SWEEP with ilu_sweeps > 0: 1 (default) the
                              block-diagonal pass z^0 = P r is folded into the first
                              forward sweep (each cell forms its lower neighbours'
                              z^0 itself); 0 a separate pass.  Same arithmetic, same
                              results                                                  */
    int32_t flux_split;    /* mixed precision without the Prandtl correction: 1 (default)
                              half of the warps of the persistent face flux kernel
                              form the FP64 part (values, interface state, collision
                              time, zeroth-order terms), the other half the FP32
                              slope-carrying part, which keeps GB300's FP64 pipe
                              busy; 0 every thread does both.  Same arithmetic;
                              results agree to rounding (multiply-adds may contract
                              differently in the two kernels)                          */
    int32_t ilu_sweep_pairs; /* GKS_PC_ILU_SWEEP with the per-cell equations: 1 (default)
                              a pair of consecutive backward sweeps runs in one
                              launch, each cell forming its upper neighbours'
                              first-sweep values itself; 0 one sweep per launch.
                              Same arithmetic, same results                         */
    int32_t spmv_dots;     /* mixed precision with basis_fp32 and the per-cell equations:
                              1 (default) the operator kernel of an Arnoldi step also
                              forms the Gram-Schmidt products with the basis (the new
                              vector is not read back); 0 a separate dot-product
                              kernel.  Results agree to rounding                      */
    int32_t flux_lead;     /* mixed precision: 1 (default) the flux's parts that need
                              more than FP32 (Gauss-point values, interface state,
                              collision time, zeroth-order terms) in double-FP32
                              arithmetic (pairs of FP32 numbers, about 48 bits) on
                              the FP32 pipe, one thread per Gauss point doing both
                              parts (flux_split is then ignored); 0 those parts in
                              FP64 (flux_split chooses the kernel); 2 the whole flux
                              in FP64 (the FP64 path's kernel, reading the FP64
                              coefficients of the refinement), for viscous flows
                              whose FP32 slope-carrying terms (the viscous stress)
                              would limit the agreement with the FP64 path         */
    int32_t flux_shape;    /* launch shape of the double-FP32 flux kernel: 0 (default)
                              128 threads x 4 blocks per SM (128 registers), 1 x 3
                              (168 registers), 2 x 2 (255 registers).  The same
                              source, compiled once per shape, so results of two
                              shapes may differ in the last bits; the autotuner's
                              last stage picks one                                     */
    int32_t reserved;      /* must be 0                                                */
} gks_config;

typedef struct gks_mesh gks_mesh;

typedef struct gks_solve_info {
    int32_t iters[4];      /* GMRES iterations per conserved variable                  */
    double relres[4];      /* final ||b - A x|| / ||b|| (0 when b = 0)                  */
    int32_t converged;     /* 1 if all four met gmres_rtol                              */
} gks_solve_info;

typedef struct gks_step_info {
    double dt;             /* step taken                                               */
    int32_t iters[4];
    double relres[4];
    int32_t status;        /* GKS_OK, GKS_ENONPHYS or GKS_ENOCONV                      */
} gks_step_info;

typedef struct gks_run_info {
    int64_t steps;         /* steps taken                                              */
    double t;              /* time reached                                             */
    double last_dt;
    int64_t gmres_iters;   /* sum over steps and variables                             */
    double steady_res;     /* max over variables of the area-weighted L2 norm of
                              (w^{n+1} - w^n)/dt, relative to its first-step value       */
    int32_t status;
} gks_run_info;

typedef struct gks_mesh_stats {
    int64_t n_tri, n_face, n_boundary_face;
    int64_t n_k1;          /* cells reconstructed at k = 1                              */
    int64_t nnzb;          /* 5x5 blocks of the CLS operator                            */
    int32_t levels_lower;  /* level-schedule depth of the forward ILU solve             */
    int32_t levels_upper;  /* ... and of the backward solve                             */
    int64_t rcm_bandwidth; /* max |i - j| over neighbouring cells in RCM order          */
    int64_t device_bytes;  /* device memory held by the handle                          */
    int32_t n_case;        /* independent cases held by the handle (1 for a mesh)        */
} gks_mesh_stats;

/* One independent case of a batch: the same arrays as gks_mesh_create. */
typedef struct gks_case_desc {
    const double *nodes;
    int64_t n_nodes;
    const int32_t *tris;
    int64_t n_tri;
    const int32_t *faces;
    const double *face_shift;
    int64_t n_face;
    const double *bc_state;
} gks_case_desc;

typedef struct gks_batch_info {
    int64_t steps;         /* steps taken (the step loop of the whole batch)           */
    int64_t gmres_iters;   /* GMRES iterations summed over cases and variables         */
    int32_t n_failed;      /* cases stopped by GKS_ENONPHYS or GKS_ENOCONV             */
    int32_t n_finished;    /* cases that reached their t_final                          */
} gks_batch_info;

/* Fill *cfg with defaults: gamma 1.4, cfl 0.3, mu 0, cls_w 0.3, gmres_m 30,
 * gmres_maxit 1000, gmres_rtol 1e-12, FP64, GKS_PC_ILU_SWEEP with 2 sweeps,
 * tau2_exact 0. */
GKS_EXPORT void gks_config_default(gks_config *cfg);

/* Build the mesh handle on the current CUDA device (host set-up: geometry,
 * k_i of Eq. (28), RCM order, CLS blocks of Eq. (29), block ILU(0) factors and
 * level sets; then one upload).  All inputs are host arrays, copied:
 *   nodes      [n_nodes][2] float64 coordinates;
 *   tris       [n_tri][3] int32 node indices (any orientation);
 *   faces      [n_face][5] int32: n0, n1 (node indices in cell_l's frame),
 *              cell_l, cell_r (-1 on a non-periodic boundary), bc tag
 *              (GKS_BC_*); every cell has at most three faces;
 *   face_shift [n_face][2] float64: translation added to cell_r's coordinates
 *              to place it next to cell_l across a periodic face, else 0;
 *   bc_state   [n_face][4] float64: per-face boundary data (see GKS_BC_*);
 *   cfg        may be NULL for the defaults.
 * Errors: GKS_EINVAL (sizes <= 0, an index out of range, degenerate triangle,
 * a cell with more than three faces, tag/cell_r mismatch, bad config),
 * GKS_ENOMEM, GKS_ECUDA.  On error *out is NULL. */
GKS_EXPORT gks_status gks_mesh_create(const double *nodes, int64_t n_nodes, const int32_t *tris, int64_t n_tri,
                           const int32_t *faces, const double *face_shift, int64_t n_face,
                           const double *bc_state, const gks_config *cfg, gks_mesh **out);

/* Build one handle holding n_cases independent meshes (each described as in
 * gks_mesh_create) that advance together: every kernel launch covers all
 * cases, and each case keeps its own time step, GMRES convergence masks and
 * status.  State arrays of a batch are float64 [4][sum of n_tri] (and
 * coefficients [4][5][sum of n_tri], face fluxes [4][sum of n_face]) with the
 * cases' cells (faces) concatenated in case order.  Errors as gks_mesh_create;
 * the message names the failing case. */
GKS_EXPORT gks_status gks_batch_create(const gks_case_desc *cases, int32_t n_cases, const gks_config *cfg,
                                       gks_mesh **out);

/* Advance every case of a batch handle (or a single mesh) with its own CFL
 * step until its t_final (host [n_cases]; NULL or <= 0: no limit; the last step
 * is cut to land on it) or max_steps steps of the batch.  A case whose state
 * goes non-physical or whose GMRES hits gmres_maxit stops; the others go on.
 * w: device [4][sum n_tri].  t_reached, case_status (GKS_OK, GKS_ENONPHYS,
 * GKS_ENOCONV): host [n_cases], may be NULL.  Returns GKS_OK unless an argument
 * or CUDA error occurs.  No host round trip per step: with graphs on
 * (no_graphs = 0) the steps are one graph launch that the device ends, else the
 * host looks at the done flags every 16 steps; the stream is synchronised at the
 * start and at the end of the call. */
GKS_EXPORT gks_status gks_batch_run(gks_mesh *batch, double *w, const double *t_final, int64_t max_steps,
                                    double *t_reached, int32_t *case_status, gks_batch_info *info, void *stream);

/* Free every device and host resource of the handle (NULL is accepted). */
GKS_EXPORT gks_status gks_mesh_destroy(gks_mesh *mesh);

/* Sizes and solver structure of a handle (host output). */
GKS_EXPORT gks_status gks_mesh_get_stats(const gks_mesh *mesh, gks_mesh_stats *stats);

/* Time step dt = cfl * min_i r_i / (|U_i| + c_i + 2 mu / (rho_i r_i)), r_i the
 * inradius of cell i (the paper does not state its CFL rule).
 * w: device [4][n_tri].  *dt_out: host.  Synchronises the stream. */
GKS_EXPORT gks_status gks_cfl_dt(gks_mesh *mesh, const double *w, double *dt_out, void *stream);
/* (gks_cfl_dt, gks_step and gks_run take single-mesh handles; GKS_EINVAL for a batch.) */

/* Same time step as gks_cfl_dt, for callers that cannot allocate device
 * memory when they need it: time loops of solvers that reserve all their
 * device memory at start-up and forbid allocation afterwards, and hosts whose
 * device memory belongs to another allocator (a framework's caching pool that
 * must not be bypassed, or that has handed out all it holds).  The paper has
 * no counterpart; this entry point only changes where the scratch lives.
 *   w      device [4][n_tri], caller's cell order (read only);
 *   dt_dev device pointer to one double that receives the step; nothing is
 *          copied to the host and the stream is not synchronised.
 * The call allocates nothing: the block minima of its reduction live in a
 * 128 KiB static device array of the library, held by every GPU that loads
 * it until exit, which limits meshes to 4,194,304 cells (GKS_EINVAL above, and
 * for batch handles).
 * The first call on each device looks up that array's device address and
 * keeps it for the life of the process; make that call before any stream
 * capture.  A device reset (cudaDeviceReset) may move the array, after which
 * this entry point must not be called again in the same process.  All calls
 * share the array, so calls that overlap on the GPU (two streams, or two
 * handles on one device) race; each call writes every entry it reads, so
 * nothing has to start at zero. */
GKS_EXPORT gks_status gks_cfl_dt_noalloc(const gks_mesh *mesh, const double *w, double *dt_dev, void *stream);

/* CLS reconstruction (Sec. III): solves the per-cell least-squares system
 * for the four variables of w (device [4][n_tri]) and writes the coefficients
 * to coef (device [4][5][n_tri]).  GMRES starts from the handle's previous
 * solution (zero after creation or gks_reset_warm_start).  info (host, may be
 * NULL) receives iterations and residuals; GKS_ENOCONV when a variable did not
 * converge within gmres_maxit. */
GKS_EXPORT gks_status gks_cls_reconstruct(gks_mesh *mesh, const double *w, double *coef, gks_solve_info *info,
                               void *stream);

/* Forget the warm start of the reconstruction. */
GKS_EXPORT gks_status gks_reset_warm_start(gks_mesh *mesh);

/* Third-order BGK face fluxes (Sec. II.B) for given cell averages w (device
 * [4][n_tri]) and coefficients coef (device [4][5][n_tri]) over the step dt > 0;
 * writes face_flux (device [4][n_face]).  Returns GKS_ENONPHYS if a Gauss-point
 * state had rho <= 0 or p <= 0 (synchronises the stream to find out). */
GKS_EXPORT gks_status gks_flux(gks_mesh *mesh, const double *w, const double *coef, double dt, double *face_flux,
                    void *stream);

/* Shock detector (Eq. (37)) and DWBAP limiter (Eqs. (34)-(36)) on a
 * reconstruction: w (device [4][n_tri]) and coef (device [4][5][n_tri], as
 * returned by gks_cls_reconstruct) in, limited coefficients coef_out (device
 * [4][5][n_tri], may not alias coef) out; flags (device [n_tri], may be NULL)
 * receives 0 for an untouched cell, 1 for a limited one and 2 for a limited
 * cell reset to its average (robust mode, or its limited polynomial still had
 * rho <= 0 or p <= 0 at a face Gauss point).  A cell is limited when the
 * detector flags it or its polynomial has rho <= 0 or p <= 0 at a face Gauss
 * point.  Derivatives are replaced by
 * u_0 tan(sum_j omega_j arctan(u_j / u_0)) over the cell's own and its face
 * neighbours' polynomials at the centroid, omega_j from the distances to the
 * face midpoints and the spread of the neighbour pressures (Eqs. (35)-(36)).
 * Requires a mesh created with gks_config.limiter = 1 or 2 (GKS_EINVAL otherwise);
 * with it, gks_step, gks_run and gks_batch_run limit every reconstruction
 * before the flux.  Stream-ordered, no synchronisation. */
GKS_EXPORT gks_status gks_limit(gks_mesh *mesh, const double *w, const double *coef, double *coef_out,
                                int32_t *flags, void *stream);

/* One explicit step (Eq. (6)) in place on w (device [4][n_tri]).
 * *dt_inout (host): > 0 fixes the step; <= 0 takes the CFL step and returns it
 * (with graphs on, as one launch of the step-loop graph of gks_run, read back
 * with one synchronisation).  The step always advances the case, also after a
 * gks_run that ended it at its end time.  info (host, may be NULL).  The call
 * synchronises the stream. */
GKS_EXPORT gks_status gks_step(gks_mesh *mesh, double *w, double *dt_inout, gks_step_info *info, void *stream);

/* Steps w (device [4][n_tri]) in place until t_final (the last step is cut to
 * land on it; t_final <= 0: no time limit), max_steps steps, or, if
 * steady_tol > 0, until the steady residual (gks_run_info) drops below it.
 * info (host, may be NULL).  Without a steady tolerance the steps run as in
 * gks_batch_run (one graph launch with graphs on); with one, the host reads the
 * residual after every step. */
GKS_EXPORT gks_status gks_run(gks_mesh *mesh, double *w, double t_final, int64_t max_steps, double steady_tol,
                   gks_run_info *info, void *stream);

/* Gauss-point flux kernel on its own (Sec. II.B), for n independent points in
 * their face frames: wl, wr device [n][6][4] (rows: value, d/dn, d/dt,
 * d2/dn2, d2/dndt, d2/dt2 of rho, rho*U, rho*V, E; U normal from left to
 * right); out device [n][4] = int_0^dt of the flux through a unit-length face.
 * cfg supplies gamma, mu and tau2_exact (NULL: defaults).  Stream-ordered, no
 * synchronisation. */
GKS_EXPORT gks_status gks_point_flux(int64_t n, const double *wl, const double *wr, double dt, const gks_config *cfg,
                          double *out, void *stream);

/* Autotuner.  Times trial steps of the handle's own workload (all its cases)
 * for each candidate of the knobs that change the cost of a step but not its
 * result beyond the solver tolerance: (ilu_sweeps, ilu_sweeps_bwd) in
 * {(1, -1), (2, -1), (3, -1), (2, 1), (3, 1), (1, 2)} (sweep preconditioner
 * only), warm_extrap in {0, 1, 2} and, in mixed precision,
 * inner_rtol in {1e-4, 1e-5, 1e-6}; then, with the best of those, the GMRES
 * restart length in {gmres_m, 16, 8} (at most the gmres_m the handle was
 * created with, which sized its Krylov buffers); then, for the mixed flux in
 * double-FP32 without the Prandtl correction and with mean interface slopes,
 * the launch shape (register budget) of the flux kernel.  Each candidate starts from w (device,
 * [4][n_tri], caller order, not modified) with a cleared warm start, takes
 * 3 untimed steps, then trial_steps (>= 1) steps timed with CUDA events; a
 * candidate whose steps fail is skipped.  The fastest candidate is written to
 * the handle's configuration and to *out (host), and the warm start is cleared.
 * Synchronises the stream. */
typedef struct gks_tune_result {
    int32_t ilu_sweeps;
    int32_t warm_extrap;
    double inner_rtol;
    double ms_per_step;           /* chosen candidate                               */
    double ms_per_step_before;    /* the configuration the handle had before        */
    int32_t n_candidates;         /* candidates timed                               */
    int32_t n_failed;             /* candidates skipped because a step failed       */
    int32_t ilu_sweeps_bwd;       /* chosen backward sweeps (-1: as ilu_sweeps)     */
    int32_t gmres_m;              /* chosen restart length (also in the config)     */
    int32_t flux_variant;         /* chosen launch shape of the double-FP32 flux
                                     kernel: 0 128 threads x 4 blocks per SM (128
                                     registers), 1 x 3 (168), 2 x 2 (255)          */
} gks_tune_result;

GKS_EXPORT gks_status gks_autotune(gks_mesh *mesh, const double *w, int32_t trial_steps, gks_tune_result *out,
                                   void *stream);

/* Optional CUDA-event timing of kernel classes, for benchmarks.  Bit c of
 * class_mask enables class c: 0 face flux, 1 CLS operator application in
 * GMRES, 2 ILU(0) preconditioner application, 3 Gram-Schmidt orthogonalisation
 * (dot products, updates, reductions), 4 conservative update, 5 FP64 residual
 * b - K x of the solve's start and restarts (with its norms), 6 correction of
 * a GMRES cycle (back-substitution, x += Z y), 7 the step's small kernels
 * (CFL time step, warm start, right-hand side, masks, Givens rotations, stop
 * conditions).  Events are recorded on the stream of each call between begin
 * and end; while any class is timed the solve launches its kernels one by one
 * (events between kernels), so the timed steps are slower than untimed ones. */
#define GKS_PROF_CLASSES 8
typedef struct gks_profile {
    int64_t n[GKS_PROF_CLASSES];  /* timed launches (or launch groups) per class       */
    double ms[GKS_PROF_CLASSES];  /* summed device time per class                      */
    int64_t arnoldi;       /* Arnoldi iterations (all systems of the handle together)  */
    int64_t arnoldi_jsum;  /* sum over those iterations of j + 1 (vectors orthogonalised
                              against), for the byte count of the class 3 kernels      */
    int64_t precond;       /* preconditioner applications                              */
    int64_t residuals;     /* FP64 residual evaluations (operator applications, mode 1) */
} gks_profile;

GKS_EXPORT gks_status gks_profile_begin(gks_mesh *mesh, int32_t class_mask);
/* Synchronises on the recorded events, fills *out, disables timing. */
GKS_EXPORT gks_status gks_profile_end(gks_mesh *mesh, gks_profile *out);
/* Number of kernel launches issued by the library in this process. */
GKS_EXPORT int64_t gks_launch_count(void);

/* Measurement probes (not part of the scheme).  A benchmark times them with
 * CUDA events on `stream` to measure the roofs of the kernels above on the GPU
 * it runs on.
 *   gks_probe_fma:  blocks_per_sm x (SM count) blocks of 256 threads, each
 *                   thread 8 independent chains of 64 iters multiply-adds in
 *                   FP64 (fp64 = 1) or FP32; *flops (host, may be NULL)
 *                   receives the flops of the launch (a multiply-add counts 2).
 *                   sink: device scratch of at least blocks_per_sm x (SM count)
 *                   doubles, never written in practice (it keeps the chains live).
 *   gks_probe_read: reads every 16-byte word of buf (device, 16-byte aligned,
 *                   bytes a positive multiple of 16) with streaming loads;
 *                   sink: device scratch of 4 x (SM count) doubles.
 *   gks_probe_copy: copies bytes from src to dst (device, same rules).
 * GKS_EINVAL for NULL pointers or misaligned buffers; asynchronous otherwise. */
GKS_EXPORT gks_status gks_probe_fma(int32_t fp64, int32_t blocks_per_sm, int32_t iters, double *sink, void *stream,
                                    double *flops);
GKS_EXPORT gks_status gks_probe_read(const void *buf, int64_t bytes, double *sink, void *stream);
GKS_EXPORT gks_status gks_probe_copy(const void *src, void *dst, int64_t bytes, void *stream);

/* Test probe of the double-FP32 arithmetic of the mixed flux (pairs of FP32
 * numbers, about 48 significant bits; not part of the scheme): for each i,
 * x[i] (and y[i]) are split into FP32 pairs, op is applied in pair arithmetic
 * and out[2 i] receives the result widened to FP64 (out[2 i + 1] = 0); for
 * GKS_DF_SPLIT out[2 i], out[2 i + 1] receive the pair itself.  x, y, out:
 * device arrays of n, n and 2 n doubles (y only for the two-argument ops).
 * Domains: GKS_DF_EXP x <= 88 (below -87 the result is flushed to 0),
 * GKS_DF_ERFCX 0 <= x <= 10, GKS_DF_SQRT x > 0.  GKS_EINVAL for a bad op or a
 * NULL array; asynchronous. */
enum {
    GKS_DF_SPLIT = 0, GKS_DF_EXP = 1, GKS_DF_EXPM1 = 2, GKS_DF_ERFCX = 3, GKS_DF_SQRT = 4, GKS_DF_DIV = 5,
    GKS_DF_MUL = 6, GKS_DF_ADD = 7, GKS_DF_RECIP = 8
};
GKS_EXPORT gks_status gks_probe_df(int32_t op, int64_t n, const double *x, const double *y, double *out,
                                   void *stream);

/* The bounded wait of the sync-free triangular solves on its own: one thread
 * waits for a device flag to reach 1, giving up after limit_ns nanoseconds of
 * the GPU's global timer (1 <= limit_ns <= 10^10).  set_flag = 1 sets the flag
 * before the wait (the wait returns at once), 0 leaves it at 0, which nothing
 * changes, so the wait runs out.  *timed_out (host) = 1 if it gave up, else 0;
 * *waited_ns (host, may be NULL) = the time the wait took.  GKS_EINVAL for a
 * limit outside the range or NULL timed_out.  Synchronises the stream. */
GKS_EXPORT gks_status gks_probe_wait(int64_t limit_ns, int32_t set_flag, int32_t *timed_out, int64_t *waited_ns,
                                     void *stream);

/* Thread-local message of the last error, or "" if none. */
GKS_EXPORT const char *gks_last_error(void);

#ifdef __cplusplus
}
#endif
#endif /* GKS_H */
