/*
 * Oracle: one explicit step of the third-order gas-kinetic scheme and the
 * public entry points of the oracle library (loaded from Python by ctypes).
 * TEST INFRASTRUCTURE ONLY (see or_internal.h).
 *
 * Step (Eq. (6), single stage): time step from the CFL condition, CLS
 * reconstruction (Sec. III) of the four conservative variables, the
 * time-integrated flux at two Gauss points per face (Eqs. (7), (11), (15)),
 * and the conservative update of the cell averages.
 *
 * Layouts (all float64): w is [4][T] (rho, rho u, rho v, E); coefficients
 * are [4][5][T] (variable, basis index, cell; basis indices 3..5 are zero at
 * cells with k = 1); face fluxes are [4][F], time-integrated, Gauss-summed,
 * multiplied by the face length and signed along the normal from cell_l to
 * cell_r.
 */
#include <math.h>
#include <stdlib.h>
#include <string.h>

#include "or_internal.h"

static void *xcalloc(size_t n, size_t s) { return calloc(n ? n : 1, s); }

void or_params_default(or_params *p)
{
    p->gamma = 1.4; p->cfl = 0.3; p->mu = 0.0; p->cls_w = 0.3;
    p->gmres_m = 30; p->gmres_maxit = 5000; p->gmres_rtol = 1e-14;
    p->tau2_exact = 0; p->slope0_mode = 0; p->limiter = 0; p->second_order = 0; p->prandtl = 1.0;
    p->limit_char = 0;
    p->cls_global = 0;
    p->cls_M = 1;
}

void or_mesh_free(or_mesh *m)
{
    if (!m) return;
    void *ptrs[] = {m->nodes, m->tri, m->face, m->shift, m->bc, m->area, m->cx, m->cy, m->crad, m->h,
                    m->inrad, m->mxx, m->mxy, m->myy, m->korder, m->cface, m->fnx, m->fny, m->flen,
                    m->gx, m->gy, m->dof_off, m->nb_cnt, m->nb_cell, m->nb_dx, m->nb_dy, m->a0,
                    m->perm, m->dperm, m->dinv, m->diag_pos, m->warm};
    for (size_t k = 0; k < sizeof(ptrs) / sizeof(ptrs[0]); ++k) free(ptrs[k]);
    or_csr_free(&m->K); or_csr_free(&m->Kp); or_csr_free(&m->LU);
    free(m);
}

or_mesh *or_mesh_new(const double *nodes, int64_t n_nodes, const int32_t *tris, int64_t n_tri,
                     const int32_t *faces, const double *face_shift, int64_t n_face,
                     const double *bc_state, const or_params *prm, int *err)
{
    *err = 0;
    if (n_tri <= 0 || n_nodes <= 0 || n_face <= 0 || (prm->slope0_mode != 0 && prm->slope0_mode != 1) ||
        prm->cls_M < 0 || prm->cls_M > 2 || (prm->cls_M == 0 && !prm->second_order)) {
        *err = -10;
        return NULL;
    }
    or_mesh *m = calloc(1, sizeof(or_mesh));
    if (!m) { *err = -1; return NULL; }
    m->prm = *prm;
    m->n_nodes = n_nodes; m->n_tri = n_tri; m->n_face = n_face;
    const size_t T = (size_t)n_tri, F = (size_t)n_face;
    m->nodes = xcalloc(2 * (size_t)n_nodes, sizeof(double));
    m->tri = xcalloc(3 * T, sizeof(int)); m->face = xcalloc(5 * F, sizeof(int));
    m->shift = xcalloc(2 * F, sizeof(double)); m->bc = xcalloc(4 * F, sizeof(double));
    double **cd[] = {&m->area, &m->cx, &m->cy, &m->crad, &m->h, &m->inrad, &m->mxx, &m->mxy, &m->myy};
    for (size_t k = 0; k < 9; ++k) *cd[k] = xcalloc(T, sizeof(double));
    m->korder = xcalloc(T, sizeof(int)); m->cface = xcalloc(3 * T, sizeof(int));
    m->fnx = xcalloc(F, sizeof(double)); m->fny = xcalloc(F, sizeof(double)); m->flen = xcalloc(F, sizeof(double));
    m->gx = xcalloc(2 * F, sizeof(double)); m->gy = xcalloc(2 * F, sizeof(double));
    m->dof_off = xcalloc(T, sizeof(int)); m->nb_cnt = xcalloc(T, sizeof(int)); m->nb_cell = xcalloc(3 * T, sizeof(int));
    m->nb_dx = xcalloc(3 * T, sizeof(double)); m->nb_dy = xcalloc(3 * T, sizeof(double));
    m->a0 = xcalloc(15 * T, sizeof(double));
    m->perm = xcalloc(T, sizeof(int)); m->dperm = xcalloc(5 * T, sizeof(int)); m->dinv = xcalloc(5 * T, sizeof(int));
    m->warm = xcalloc(20 * T, sizeof(double));
    if (!m->nodes || !m->tri || !m->face || !m->shift || !m->bc || !m->area || !m->cx || !m->cy || !m->crad ||
        !m->h || !m->inrad || !m->mxx || !m->mxy || !m->myy || !m->korder || !m->cface || !m->fnx || !m->fny ||
        !m->flen || !m->gx || !m->gy || !m->dof_off || !m->nb_cnt || !m->nb_cell || !m->nb_dx || !m->nb_dy ||
        !m->a0 || !m->perm || !m->dperm || !m->dinv || !m->warm) { or_mesh_free(m); *err = -1; return NULL; }
    memcpy(m->nodes, nodes, sizeof(double) * 2 * (size_t)n_nodes);
    for (size_t k = 0; k < 3 * T; ++k) {
        m->tri[k] = tris[k];
        if (tris[k] < 0 || tris[k] >= n_nodes) { or_mesh_free(m); *err = -11; return NULL; }
    }
    for (size_t k = 0; k < 5 * F; ++k) m->face[k] = faces[k];
    for (size_t f = 0; f < F; ++f) {
        const int *fc = &m->face[5 * f];
        if (fc[0] < 0 || fc[0] >= n_nodes || fc[1] < 0 || fc[1] >= n_nodes || fc[2] < 0 || fc[2] >= n_tri ||
            fc[3] < -1 || fc[3] >= n_tri || fc[4] < 0 || fc[4] > 5 ||
            ((fc[3] < 0) != (fc[4] >= OR_DIRICHLET))) { or_mesh_free(m); *err = -12; return NULL; }
    }
    memcpy(m->shift, face_shift, sizeof(double) * 2 * F);
    memcpy(m->bc, bc_state, sizeof(double) * 4 * F);
    int e;
    if ((e = or_build_geometry(m)) != 0) { or_mesh_free(m); *err = -20 + e; return NULL; }
    if ((e = or_build_cls(m)) != 0) { or_mesh_free(m); *err = -30 + e; return NULL; }
    if ((e = or_build_rcm(m)) != 0) { or_mesh_free(m); *err = -40 + e; return NULL; }
    if ((e = or_ilu0(&m->Kp, &m->LU, &m->diag_pos)) != 0) { or_mesh_free(m); *err = -50 + e; return NULL; }
    return m;
}

int64_t or_mesh_ndof(const or_mesh *m) { return m->ndof; }

/* cell geometry: 10 per cell: area, cx, cy, circumradius, h, inradius, <dx2>, <dxdy>, <dy2>, k */
void or_cell_geometry(const or_mesh *m, double *out)
{
    for (int64_t i = 0; i < m->n_tri; ++i) {
        double *o = out + 10 * i;
        o[0] = m->area[i]; o[1] = m->cx[i]; o[2] = m->cy[i]; o[3] = m->crad[i]; o[4] = m->h[i];
        o[5] = m->inrad[i]; o[6] = m->mxx[i]; o[7] = m->mxy[i]; o[8] = m->myy[i]; o[9] = m->korder[i];
    }
}

/* face geometry: 7 per face: nx, ny, length, gx0, gy0, gx1, gy1 */
void or_face_geometry(const or_mesh *m, double *out)
{
    for (int64_t f = 0; f < m->n_face; ++f) {
        double *o = out + 7 * f;
        o[0] = m->fnx[f]; o[1] = m->fny[f]; o[2] = m->flen[f];
        o[3] = m->gx[2 * f]; o[4] = m->gy[2 * f]; o[5] = m->gx[2 * f + 1]; o[6] = m->gy[2 * f + 1];
    }
}

void or_rcm_perm(const or_mesh *m, int32_t *perm) { for (int64_t i = 0; i < m->n_tri; ++i) perm[i] = m->perm[i]; }

/* CSR of the CLS matrix (natural dof order); pass NULL to query nnz. */
int64_t or_cls_matrix(const or_mesh *m, int32_t *rowptr, int32_t *col, double *val, int32_t *dof_off)
{
    if (rowptr) {
        for (int r = 0; r <= m->K.n; ++r) rowptr[r] = m->K.rowptr[r];
        for (int e = 0; e < m->K.nnz; ++e) { col[e] = m->K.col[e]; val[e] = m->K.val[e]; }
        for (int64_t i = 0; i < m->n_tri; ++i) dof_off[i] = m->dof_off[i];
    }
    return m->K.nnz;
}

/* CLS right-hand sides for the four variables, [4][ndof] natural order */
void or_cls_rhs(const or_mesh *m, const double *w, double *rhs)
{
    for (int v = 0; v < 4; ++v) or_cls_rhs_var(m, w + v * m->n_tri, rhs + (size_t)v * m->ndof);
}

static void unpack_coef(const or_mesh *m, const double *x, double *coef, int var)
{
    const int64_t T = m->n_tri;
    for (int64_t i = 0; i < T; ++i) {
        int ni = m->korder[i] == 2 ? 5 : 2;
        for (int l = 0; l < 5; ++l) coef[((size_t)var * 5 + l) * T + i] = (l < ni) ? x[m->dof_off[i] + l] : 0.0;
    }
}

/* CLS reconstruction by GMRES + ILU(0) on the RCM order.  use_warm: start from
 * the previous solution kept in the mesh object (else from zero).  iters and
 * relres receive 4 values.  Returns the number of variables not converged. */
int or_cls_solve(or_mesh *m, const double *w, double *coef, int use_warm, int32_t *iters, double *relres)
{
    const int n = m->ndof;
    double *rhs = malloc(sizeof(double) * (size_t)n), *bp = malloc(sizeof(double) * (size_t)n);
    double *xp = malloc(sizeof(double) * (size_t)n);
    int bad = 0;
    for (int v = 0; v < 4; ++v) {
        or_cls_rhs_var(m, w + v * m->n_tri, rhs);
        double *x = m->warm + (size_t)v * n;
        for (int r = 0; r < n; ++r) { bp[r] = rhs[m->dperm[r]]; xp[r] = use_warm ? x[m->dperm[r]] : 0.0; }
        int it = 0; double rr = 0.0;
        bad += or_gmres(&m->Kp, &m->LU, m->diag_pos, bp, xp, m->prm.gmres_m, m->prm.gmres_maxit,
                        m->prm.gmres_rtol, &it, &rr);
        for (int r = 0; r < n; ++r) x[m->dperm[r]] = xp[r];
        if (iters) iters[v] = it;
        if (relres) relres[v] = rr;
        unpack_coef(m, x, coef, v);
    }
    free(rhs); free(bp); free(xp);
    return bad;
}

/* Same system solved by dense LU with partial pivoting (tiny meshes only). */
int or_cls_dense(const or_mesh *m, const double *w, double *coef)
{
    const int n = m->ndof;
    if (n > 4000) return -1;
    double *A = malloc(sizeof(double) * (size_t)n * n), *b = malloc(sizeof(double) * (size_t)n);
    int st = 0;
    for (int v = 0; v < 4 && st == 0; ++v) {
        memset(A, 0, sizeof(double) * (size_t)n * n);
        for (int r = 0; r < n; ++r)
            for (int e = m->K.rowptr[r]; e < m->K.rowptr[r + 1]; ++e) A[(size_t)r * n + m->K.col[e]] = m->K.val[e];
        or_cls_rhs_var(m, w + v * m->n_tri, b);
        st = or_dense_lu_solve(n, A, b);
        unpack_coef(m, b, coef, v);
    }
    free(A); free(b);
    return st;
}

/* Value and derivatives (global frame) of the reconstruction of cell c, with
 * the point given in the cell's own frame.  out[6][4]: W, Wx, Wy, Wxx, Wxy, Wyy. */
static void eval_cell(const or_mesh *m, const double *w, const double *coef, int c, double x, double y, double *out)
{
    const int64_t T = m->n_tri;
    double h = m->h[c];
    double dx = (x - m->cx[c]) / h, dy = (y - m->cy[c]) / h;
    for (int v = 0; v < 4; ++v) {
        double u[5];
        for (int l = 0; l < 5; ++l) u[l] = coef[((size_t)v * 5 + l) * T + c];
        out[v] = w[(size_t)v * T + c] + u[0] * dx + u[1] * dy + 0.5 * u[2] * (dx * dx - m->mxx[c])
               + u[3] * (dx * dy - m->mxy[c]) + 0.5 * u[4] * (dy * dy - m->myy[c]);
        out[4 + v] = (u[0] + u[2] * dx + u[3] * dy) / h;
        out[8 + v] = (u[1] + u[3] * dx + u[4] * dy) / h;
        out[12 + v] = u[2] / (h * h);
        out[16 + v] = u[3] / (h * h);
        out[20 + v] = u[4] / (h * h);
    }
}

void or_eval_cell(const or_mesh *m, const double *w, const double *coef, int c, double x, double y, double *out)
{
    eval_cell(m, w, coef, c, x, y, out);
}

/* Global frame -> face frame (x along n, y along t = (-ny, nx)). */
static void to_face_frame(const double *g, double nx, double ny, double *f)
{
    double tx = -ny, ty = nx;
    double d[6][4];
    /* rotate the derivative directions */
    for (int v = 0; v < 4; ++v) {
        d[0][v] = g[v];
        d[1][v] = nx * g[4 + v] + ny * g[8 + v];
        d[2][v] = tx * g[4 + v] + ty * g[8 + v];
        d[3][v] = nx * nx * g[12 + v] + 2.0 * nx * ny * g[16 + v] + ny * ny * g[20 + v];
        d[4][v] = nx * tx * g[12 + v] + (nx * ty + ny * tx) * g[16 + v] + ny * ty * g[20 + v];
        d[5][v] = tx * tx * g[12 + v] + 2.0 * tx * ty * g[16 + v] + ty * ty * g[20 + v];
    }
    /* rotate the momentum components of every row */
    for (int r = 0; r < 6; ++r) {
        f[4 * r + 0] = d[r][0];
        f[4 * r + 1] = nx * d[r][1] + ny * d[r][2];
        f[4 * r + 2] = tx * d[r][1] + ty * d[r][2];
        f[4 * r + 3] = d[r][3];
    }
}

/* Second-order jets of a field at the Gauss point in the face frame:
 * j[0] value, j[1] d/dn, j[2] d/dt, j[3] d2/dn2, j[4] d2/dndt, j[5] d2/dt2
 * (the row order of the face-frame states).  Products and quotients follow
 * the Leibniz and quotient rules term by term. */
static const int jet_nord[6] = {0, 1, 0, 2, 1, 0};   /* order in n of each entry */

static void jet_of(const double *rows, int v, double *j)
{
    for (int r = 0; r < 6; ++r) j[r] = rows[4 * r + v];
}

static void jet_mul(const double *a, const double *b, double *c)
{
    double o[6];
    o[0] = a[0] * b[0];
    o[1] = a[1] * b[0] + a[0] * b[1];
    o[2] = a[2] * b[0] + a[0] * b[2];
    o[3] = a[3] * b[0] + 2.0 * a[1] * b[1] + a[0] * b[3];
    o[4] = a[4] * b[0] + a[1] * b[2] + a[2] * b[1] + a[0] * b[4];
    o[5] = a[5] * b[0] + 2.0 * a[2] * b[2] + a[0] * b[5];
    memcpy(c, o, sizeof(o));
}

/* c = a / b */
static void jet_div(const double *a, const double *b, double *c)
{
    /* 1/b: derivatives of 1/x are -1/x^2 and 2/x^3 */
    double ib[6], b0 = b[0];
    ib[0] = 1.0 / b0;
    ib[1] = -b[1] / (b0 * b0);
    ib[2] = -b[2] / (b0 * b0);
    ib[3] = -b[3] / (b0 * b0) + 2.0 * b[1] * b[1] / (b0 * b0 * b0);
    ib[4] = -b[4] / (b0 * b0) + 2.0 * b[1] * b[2] / (b0 * b0 * b0);
    ib[5] = -b[5] / (b0 * b0) + 2.0 * b[2] * b[2] / (b0 * b0 * b0);
    jet_mul(a, ib, c);
}

/* Mirror image across the face (x_n -> -x_n).  odd = 0: q_g(x_n, x_t) =
 * q(-x_n, x_t); odd = 1: q_g(x_n, x_t) = 2 c - q(-x_n, x_t), the reflection
 * about the wall value c.  An entry of order k in n picks up (-1)^k, and the
 * odd reflection negates every entry except for the value's 2 c. */
static void jet_reflect(const double *q, int odd, double c, double *g)
{
    for (int r = 0; r < 6; ++r) {
        double s = (jet_nord[r] & 1) ? -1.0 : 1.0;
        if (odd) s = -s;
        g[r] = s * q[r];
    }
    if (odd) g[0] += 2.0 * c;
}

/* Ghost right state of a boundary face from the left state wl (face frame
 * rows), the face normal (nx, ny) and the face's boundary data bc.
 *  Dirichlet: the prescribed state with zero derivatives.
 *  outflow:   a copy of the left state.
 *  slip wall: the mirror image of the conservative fields, normal momentum
 *             odd, everything else even.
 *  no-slip isothermal wall (bc = wall velocity x, y and wall temperature
 *             T_w = p/rho): the mirror image of the primitive fields with the
 *             pressure even, the velocity odd about the wall velocity and the
 *             temperature odd about T_w, so that a linear shear or a linear
 *             temperature profile at uniform pressure continues across the
 *             wall unchanged; the conservative rows of the ghost follow from
 *             rho = p / T, rho u, rho v and E = p / (gamma - 1) + rho |u|^2 / 2. */
void or_ghost_rows(int tag, const double *bc, double nx, double ny, double gamma, const double *wl, double *wr)
{
    if (tag == OR_OUTFLOW) { memcpy(wr, wl, sizeof(double) * 24); return; }
    if (tag == OR_DIRICHLET) {
        memset(wr, 0, sizeof(double) * 24);
        wr[0] = bc[0]; wr[1] = nx * bc[1] + ny * bc[2]; wr[2] = -ny * bc[1] + nx * bc[2]; wr[3] = bc[3];
        return;
    }
    if (tag == OR_SLIP) {
        double q[6], g[6];
        for (int v = 0; v < 4; ++v) {
            jet_of(wl, v, q);
            jet_reflect(q, v == 1, 0.0, g);
            for (int r = 0; r < 6; ++r) wr[4 * r + v] = g[r];
        }
        return;
    }
    /* OR_NOSLIP: primitive jets of the interior state */
    double rho[6], mn[6], mt[6], E[6], un[6], ut[6], ke[6], tmp[6], p[6], T[6];
    jet_of(wl, 0, rho); jet_of(wl, 1, mn); jet_of(wl, 2, mt); jet_of(wl, 3, E);
    jet_div(mn, rho, un);
    jet_div(mt, rho, ut);
    jet_mul(mn, un, ke);                       /* rho u_n^2 */
    jet_mul(mt, ut, tmp);                      /* rho u_t^2 */
    for (int r = 0; r < 6; ++r) p[r] = (gamma - 1.0) * (E[r] - 0.5 * (ke[r] + tmp[r]));
    jet_div(p, rho, T);
    /* reflected primitive jets */
    double uwn = nx * bc[0] + ny * bc[1], uwt = -ny * bc[0] + nx * bc[1];
    double pg[6], ung[6], utg[6], Tg[6], rhog[6], o[6];
    jet_reflect(p, 0, 0.0, pg);
    jet_reflect(un, 1, uwn, ung);
    jet_reflect(ut, 1, uwt, utg);
    jet_reflect(T, 1, bc[2], Tg);
    jet_div(pg, Tg, rhog);
    /* conservative rows of the ghost */
    for (int r = 0; r < 6; ++r) wr[4 * r + 0] = rhog[r];
    jet_mul(rhog, ung, o);
    for (int r = 0; r < 6; ++r) wr[4 * r + 1] = o[r];
    jet_mul(rhog, utg, o);
    for (int r = 0; r < 6; ++r) wr[4 * r + 2] = o[r];
    double kn[6], kt[6];
    jet_mul(ung, ung, kn);
    jet_mul(utg, utg, kt);
    for (int r = 0; r < 6; ++r) tmp[r] = kn[r] + kt[r];
    jet_mul(rhog, tmp, o);
    for (int r = 0; r < 6; ++r) wr[4 * r + 3] = pg[r] / (gamma - 1.0) + 0.5 * o[r];
}

/* Ghost right state of boundary face f, in the face frame. */
static void ghost_state(const or_mesh *m, int64_t f, const double *wl, double *wr)
{
    or_ghost_rows(m->face[5 * f + 4], &m->bc[4 * f], m->fnx[f], m->fny[f], m->prm.gamma, wl, wr);
}

/* Time-integrated flux of face f (global frame, 4 values).  Returns the
 * number of its Gauss points with a non-physical state. */
static int face_flux_one(const or_mesh *m, const double *w, const double *coef, double dt, int64_t f, double *out)
{
    const int *fc = &m->face[5 * f];
    const double nx = m->fnx[f], ny = m->fny[f];
    double acc[4] = {0, 0, 0, 0};
    int bad = 0;
    for (int g = 0; g < 2; ++g) {
        double x = m->gx[2 * f + g], y = m->gy[2 * f + g];
        double gl[24], gr[24], wl[24], wr[24], F4[4];
        eval_cell(m, w, coef, fc[2], x, y, gl);
        to_face_frame(gl, nx, ny, wl);
        if (fc[3] >= 0) {
            eval_cell(m, w, coef, fc[3], x - m->shift[2 * f], y - m->shift[2 * f + 1], gr);
            to_face_frame(gr, nx, ny, wr);
        } else {
            ghost_state(m, f, wl, wr);
        }
        if (or_gp_flux(wl, wr, dt, &m->prm, F4, NULL) != 0) ++bad;
        for (int v = 0; v < 4; ++v) acc[v] += 0.5 * F4[v];       /* Gauss weight 1/2 */
    }
    /* back to the global frame, times the face length (Eq. (7)) */
    double S = m->flen[f];
    out[0] = S * acc[0];
    out[1] = S * (nx * acc[1] - ny * acc[2]);
    out[2] = S * (ny * acc[1] + nx * acc[2]);
    out[3] = S * acc[3];
    return bad;
}

/* Time-integrated face fluxes [4][F] (global frame) for the states w, the CLS
 * coefficients and the step dt.  Returns the number of Gauss points with a
 * non-physical state. */
int or_face_flux(const or_mesh *m, const double *w, const double *coef, double dt, double *flux)
{
    const int64_t F = m->n_face;
    int bad = 0;
    /* faces are independent: optional OpenMP over faces */
    #pragma omp parallel for schedule(dynamic, 64) reduction(+ : bad)
    for (int64_t f = 0; f < F; ++f) {
        double o[4];
        bad += face_flux_one(m, w, coef, dt, f, o);
        for (int v = 0; v < 4; ++v) flux[v * F + f] = o[v];
    }
    return bad;
}

/* Fluxes of the listed faces only: out[4][n] (sampled checks on large meshes). */
int or_face_flux_subset(const or_mesh *m, const double *w, const double *coef, double dt, const int64_t *ids,
                        int64_t n, double *out)
{
    int bad = 0;
    #pragma omp parallel for schedule(dynamic, 16) reduction(+ : bad)
    for (int64_t q = 0; q < n; ++q) {
        double o[4];
        bad += face_flux_one(m, w, coef, dt, ids[q], o);
        for (int v = 0; v < 4; ++v) out[v * n + q] = o[v];
    }
    return bad;
}

/* w_i -= (1/|Omega_i|) sum_f sigma_if flux_f, Eq. (6). */
void or_update(const or_mesh *m, double *w, const double *flux)
{
    const int64_t T = m->n_tri, F = m->n_face;
    for (int64_t f = 0; f < F; ++f) {
        int l = m->face[5 * f + 2], r = m->face[5 * f + 3];
        for (int v = 0; v < 4; ++v) {
            w[(size_t)v * T + l] -= flux[(size_t)v * F + f] / m->area[l];
            if (r >= 0) w[(size_t)v * T + r] += flux[(size_t)v * F + f] / m->area[r];
        }
    }
}

/* CFL time step: dt = cfl * min_i r_i / (|U_i| + c_i + 2 mu / (rho_i r_i)),
 * r_i the inradius (the paper does not state its time-step rule). */
double or_cfl_dt(const or_mesh *m, const double *w)
{
    const int64_t T = m->n_tri;
    const double gamma = m->prm.gamma;
    double dt = INFINITY;
    for (int64_t i = 0; i < T; ++i) {
        double rho = w[i], u = w[T + i] / rho, v = w[2 * T + i] / rho;
        double p = (gamma - 1.0) * (w[3 * T + i] - 0.5 * rho * (u * u + v * v));
        double c = sqrt(gamma * p / rho);
        double r = m->inrad[i];
        double di = r / (sqrt(u * u + v * v) + c + 2.0 * m->prm.mu / (rho * r));
        if (di < dt) dt = di;
    }
    return m->prm.cfl * dt;
}

/* One step.  dt_in > 0 fixes the step; otherwise the CFL step is used.
 * info[0..3]: GMRES iterations; res[0..3]: relative residuals; *dt_out the
 * step taken.  Returns 0, or 1 if a state went non-physical, 2 if GMRES did
 * not converge. */
int or_step(or_mesh *m, double *w, double dt_in, double *dt_out, int32_t *iters, double *relres)
{
    const int64_t T = m->n_tri, F = m->n_face;
    double dt = dt_in > 0.0 ? dt_in : or_cfl_dt(m, w);
    double *coef = malloc(sizeof(double) * 20 * (size_t)T), *flux = malloc(sizeof(double) * 4 * (size_t)F);
    int st = 0;
    if (or_cls_solve(m, w, coef, 1, iters, relres) != 0) st = 2;
    if (m->prm.limiter) {
        double *lim = malloc(sizeof(double) * 20 * (size_t)T);
        int32_t *flag = malloc(sizeof(int32_t) * (size_t)T);
        or_limit(m, w, coef, lim, flag);
        memcpy(coef, lim, sizeof(double) * 20 * (size_t)T);
        free(lim); free(flag);
    }
    if (or_face_flux(m, w, coef, dt, flux) != 0) st = 1;
    or_update(m, w, flux);
    if (dt_out) *dt_out = dt;
    free(coef); free(flux);
    return st;
}

/* Gauss-point flux entry point for tests (face frame, unit length). */
int or_point_flux(const double *wl, const double *wr, double dt, const or_params *prm, double *f, double *aux)
{
    return or_gp_flux(wl, wr, dt, prm, f, aux);
}
