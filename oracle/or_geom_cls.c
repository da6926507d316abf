/*
 * Oracle: mesh geometry, compact least-squares (CLS) system, RCM ordering.
 * TEST INFRASTRUCTURE ONLY (see or_internal.h).
 *
 * Sec. III.A of the paper: zero-mean quadratic basis (Eqs. (16), (19)),
 * length scale h_i (Eq. (17)), derivative-mean conservation on the face
 * neighbours (Eqs. (21)-(25)), boundary order reduction (Eqs. (26)-(28)) and
 * the derivative weights w_{i,p} = (w h_i)^p (Eq. (29)).  Each cell's
 * over-determined equations are solved in the least-squares sense (Eqs.
 * (32)-(33)) with the neighbours' coefficients as unknowns too, which gives
 * one sparse block system over all cells.
 *
 * Cell means of polynomials of degree <= 2 are taken with the three-edge-
 * midpoint rule, which integrates quadratics on a triangle exactly.
 */
#include <math.h>
#include <stdlib.h>
#include <string.h>

#include "or_internal.h"

/* Number of reconstruction unknowns of cell i: DOF(k_i), Eq. (18). */
static int ndof_of(int k) { return (k + 1) * (k + 2) / 2 - 1; }

int or_build_geometry(or_mesh *m)
{
    const int64_t T = m->n_tri, F = m->n_face;
    for (int64_t i = 0; i < T; ++i) {
        int *t = &m->tri[3 * i];
        double x0 = m->nodes[2 * t[0]], y0 = m->nodes[2 * t[0] + 1];
        double x1 = m->nodes[2 * t[1]], y1 = m->nodes[2 * t[1] + 1];
        double x2 = m->nodes[2 * t[2]], y2 = m->nodes[2 * t[2] + 1];
        double a2 = (x1 - x0) * (y2 - y0) - (x2 - x0) * (y1 - y0);
        if (a2 < 0.0) {                       /* make the triangle counter-clockwise */
            int s = t[1]; t[1] = t[2]; t[2] = s;
            double sx = x1, sy = y1; x1 = x2; y1 = y2; x2 = sx; y2 = sy;
            a2 = -a2;
        }
        if (!(a2 > 0.0)) return -1;
        double area = 0.5 * a2;
        double la = hypot(x1 - x0, y1 - y0), lb = hypot(x2 - x1, y2 - y1), lc = hypot(x0 - x2, y0 - y2);
        m->area[i] = area;
        m->cx[i] = (x0 + x1 + x2) / 3.0;
        m->cy[i] = (y0 + y1 + y2) / 3.0;
        m->crad[i] = la * lb * lc / (4.0 * area);            /* circumradius */
        m->inrad[i] = 2.0 * area / (la + lb + lc);          /* inradius     */
        m->h[i] = fmax(m->crad[i], sqrt(area));             /* Eq. (17)     */
        /* means of dx^2, dx dy, dy^2 (scaled by h_i) over the cell */
        double mx[3] = {0.5 * (x0 + x1), 0.5 * (x1 + x2), 0.5 * (x2 + x0)};
        double my[3] = {0.5 * (y0 + y1), 0.5 * (y1 + y2), 0.5 * (y2 + y0)};
        double sxx = 0, sxy = 0, syy = 0;
        for (int q = 0; q < 3; ++q) {
            double dx = (mx[q] - m->cx[i]) / m->h[i], dy = (my[q] - m->cy[i]) / m->h[i];
            sxx += dx * dx; sxy += dx * dy; syy += dy * dy;
        }
        m->mxx[i] = sxx / 3.0; m->mxy[i] = sxy / 3.0; m->myy[i] = syy / 3.0;
        m->cface[3 * i] = m->cface[3 * i + 1] = m->cface[3 * i + 2] = -1;
        m->korder[i] = m->prm.second_order ? 1 : 2;   /* second-order variant: linear everywhere */
    }
    for (int64_t f = 0; f < F; ++f) {
        const int *fc = &m->face[5 * f];
        double ax = m->nodes[2 * fc[0]], ay = m->nodes[2 * fc[0] + 1];
        double bx = m->nodes[2 * fc[1]], by = m->nodes[2 * fc[1] + 1];
        double len = hypot(bx - ax, by - ay);
        if (!(len > 0.0)) return -2;
        double nx = (by - ay) / len, ny = -(bx - ax) / len;
        int l = fc[2];
        if (nx * (0.5 * (ax + bx) - m->cx[l]) + ny * (0.5 * (ay + by) - m->cy[l]) < 0.0) {
            nx = -nx; ny = -ny;                 /* normal points from l to r */
        }
        m->fnx[f] = nx; m->fny[f] = ny; m->flen[f] = len;
        /* two-point Gauss-Legendre on the face: s = 1/2 -+ 1/(2 sqrt 3) */
        double s0 = 0.5 - 0.5 / sqrt(3.0), s1 = 0.5 + 0.5 / sqrt(3.0);
        m->gx[2 * f] = ax + s0 * (bx - ax); m->gy[2 * f] = ay + s0 * (by - ay);
        m->gx[2 * f + 1] = ax + s1 * (bx - ax); m->gy[2 * f + 1] = ay + s1 * (by - ay);
        for (int side = 0; side < 2; ++side) {
            int c = fc[2 + side];
            if (c < 0) continue;
            int slot = 0;
            while (slot < 3 && m->cface[3 * c + slot] >= 0) ++slot;
            if (slot == 3) return -3;
            m->cface[3 * c + slot] = (int)f;
        }
        /* a cell touching a non-periodic boundary face is reconstructed at k = 1, Eq. (28) */
        if (fc[3] < 0) m->korder[l] = 1;
    }
    return 0;
}

/* Basis phi_{l,i} (Eq. (19)) at point (x, y) for cell i; out[5]. */
static void basis(const or_mesh *m, int i, double x, double y, double *out)
{
    double dx = (x - m->cx[i]) / m->h[i], dy = (y - m->cy[i]) / m->h[i];
    out[0] = dx;
    out[1] = dy;
    out[2] = 0.5 * (dx * dx - m->mxx[i]);
    out[3] = dx * dy - m->mxy[i];
    out[4] = 0.5 * (dy * dy - m->myy[i]);
}

/* d/dx and d/dy of the basis of cell i at (x, y); outx[5], outy[5]. */
static void basis_grad(const or_mesh *m, int i, double x, double y, double *outx, double *outy)
{
    double h = m->h[i];
    double dx = (x - m->cx[i]) / h, dy = (y - m->cy[i]) / h;
    outx[0] = 1.0 / h; outx[1] = 0.0;     outx[2] = dx / h; outx[3] = dy / h; outx[4] = 0.0;
    outy[0] = 0.0;     outy[1] = 1.0 / h; outy[2] = 0.0;    outy[3] = dx / h; outy[4] = dy / h;
}

/* Means over cell j, translated by (ox, oy), of the basis of cell c (value rows
 * and both first derivatives), by the three-edge-midpoint rule.  When c == j
 * the cell's own frame is used, so the translation is undone first. */
static void means_over(const or_mesh *m, int c, int j, double ox, double oy, int own,
                       double *v, double *gx, double *gy)
{
    const int *t = &m->tri[3 * j];
    double px[3], py[3];
    for (int q = 0; q < 3; ++q) {
        px[q] = m->nodes[2 * t[q]] + (own ? 0.0 : ox);
        py[q] = m->nodes[2 * t[q] + 1] + (own ? 0.0 : oy);
    }
    for (int l = 0; l < 5; ++l) v[l] = gx[l] = gy[l] = 0.0;
    for (int q = 0; q < 3; ++q) {
        double xm = 0.5 * (px[q] + px[(q + 1) % 3]), ym = 0.5 * (py[q] + py[(q + 1) % 3]);
        double b[5], bx[5], by[5];
        basis(m, c, xm, ym, b);
        basis_grad(m, c, xm, ym, bx, by);
        for (int l = 0; l < 5; ++l) { v[l] += b[l] / 3.0; gx[l] += bx[l] / 3.0; gy[l] += by[l] / 3.0; }
    }
}

typedef struct { int col; double v; } or_ent;

static int cmp_ent(const void *a, const void *b)
{
    const or_ent *x = a, *y = b;
    return (x->col > y->col) - (x->col < y->col);
}

int or_build_cls(or_mesh *m)
{
    const int T = (int)m->n_tri;
    const double w = m->prm.cls_w;
    m->ndof = 0;
    for (int i = 0; i < T; ++i) { m->dof_off[i] = m->ndof; m->ndof += ndof_of(m->korder[i]); }

    /* neighbours across interior and periodic faces (boundary faces give no equation) */
    for (int i = 0; i < T; ++i) {
        m->nb_cnt[i] = 0;
        for (int s = 0; s < 3; ++s) {
            int f = m->cface[3 * i + s];
            if (f < 0) continue;
            const int *fc = &m->face[5 * f];
            if (fc[3] < 0) continue;
            int j; double ox, oy;
            if (fc[2] == i) { j = fc[3]; ox = m->shift[2 * f]; oy = m->shift[2 * f + 1]; }
            else            { j = fc[2]; ox = -m->shift[2 * f]; oy = -m->shift[2 * f + 1]; }
            int k = m->nb_cnt[i]++;
            m->nb_cell[3 * i + k] = j; m->nb_dx[3 * i + k] = ox; m->nb_dy[3 * i + k] = oy;
        }
    }

    /* Blocks of the normal equations.  Cell i's equations about its neighbour j
     * are A_ij u_i - B_ij u_j = b_ij (rows p = 0, 1, 2 of Eq. (29)).
     * Per-cell least squares (default): each cell minimises its own equations,
     *   D_i = sum_j A_ij^T A_ij,  K_ij = -A_ij^T B_ij.
     * Global (cls_global, Eq. (33)): the sum of all cells' equations is
     * minimised, so u_i also enters its neighbours' equations through B_ji:
     *   D_i += sum_j B_ji^T B_ji,  K_ij -= B_ji^T A_ji  (symmetric). */
    int cap = 0;
    for (int i = 0; i < T; ++i) {
        int ni = ndof_of(m->korder[i]);
        cap += ni * ni;
        for (int k = 0; k < m->nb_cnt[i]; ++k) cap += ni * ndof_of(m->korder[m->nb_cell[3 * i + k]]);
    }
    or_ent *ent = malloc(sizeof(or_ent) * (size_t)(cap > 0 ? cap : 1));
    int *rowptr = calloc((size_t)m->ndof + 1, sizeof(int));
    int *col = malloc(sizeof(int) * (size_t)(cap > 0 ? cap : 1));
    double *val = malloc(sizeof(double) * (size_t)(cap > 0 ? cap : 1));
    double *Dall = calloc((size_t)T * 25, sizeof(double));
    double *Oall = calloc((size_t)T * 75, sizeof(double));   /* [i][slot][5][5], A^T B parts */
    if (!ent || !rowptr || !col || !val || !Dall || !Oall) {
        free(ent); free(rowptr); free(col); free(val); free(Dall); free(Oall);
        return -1;
    }
    for (int i = 0; i < T; ++i) {
        int ni = ndof_of(m->korder[i]);
        for (int k = 0; k < 15; ++k) m->a0[15 * i + k] = 0.0;
        for (int k = 0; k < m->nb_cnt[i]; ++k) {
            int j = m->nb_cell[3 * i + k];
            int nj = ndof_of(m->korder[j]);
            double ox = m->nb_dx[3 * i + k], oy = m->nb_dy[3 * i + k];
            double va[5], gxa[5], gya[5], vb[5], gxb[5], gyb[5];
            means_over(m, i, j, ox, oy, 0, va, gxa, gya);   /* basis of i over cell j */
            /* basis of j over its own cell: evaluated in j's own (untranslated) frame */
            means_over(m, j, j, 0.0, 0.0, 1, vb, gxb, gyb);
            /* rows p = 0 (value), 1 (x, y derivatives) and, with M = 2, 2 (xx, xy, yy),
             * each weighted by w_{i,p} = (w h_i)^p; the second derivatives of the
             * quadratic basis are the constants 1/h^2 on its last three entries */
            double A[6][5], B[6][5];
            double wp1 = w * m->h[i];                           /* w_{i,1} = (w h_i)^1 */
            double wp2 = wp1 * wp1;                             /* w_{i,2} = (w h_i)^2 */
            const int M = m->prm.cls_M, np = M == 0 ? 1 : (M == 1 ? 3 : 6);
            for (int l = 0; l < 5; ++l) {
                A[0][l] = va[l];  A[1][l] = wp1 * gxa[l]; A[2][l] = wp1 * gya[l];
                B[0][l] = vb[l];  B[1][l] = wp1 * gxb[l]; B[2][l] = wp1 * gyb[l];
                for (int p = 3; p < 6; ++p) { A[p][l] = 0.0; B[p][l] = 0.0; }
            }
            if (M == 2) {
                const double hi2 = m->h[i] * m->h[i], hj2 = m->h[j] * m->h[j];
                for (int p = 0; p < 3; ++p) {
                    if (ni == 5) A[3 + p][2 + p] = wp2 / hi2;
                    if (nj == 5) B[3 + p][2 + p] = wp2 / hj2;
                }
            }
            for (int l = 0; l < 5; ++l) m->a0[15 * i + 5 * k + l] = (l < ni) ? A[0][l] : 0.0;
            double *Di = &Dall[25 * i], *Oik = &Oall[75 * i + 25 * k];
            for (int r = 0; r < ni; ++r) {
                for (int c = 0; c < ni; ++c)
                    for (int p = 0; p < np; ++p) Di[5 * r + c] += A[p][r] * A[p][c];
                for (int c = 0; c < nj; ++c)
                    for (int p = 0; p < np; ++p) Oik[5 * r + c] += A[p][r] * B[p][c];
            }
            if (m->prm.cls_global) {
                /* the same equations seen from j: B^T B on D_j, B^T A on the block
                 * (j, i) of the slot of j that points back to i through this face */
                int kb = -1;
                for (int q = 0; q < m->nb_cnt[j]; ++q)
                    if (m->nb_cell[3 * j + q] == i && m->nb_dx[3 * j + q] == -ox && m->nb_dy[3 * j + q] == -oy) kb = q;
                if (kb < 0) {
                    free(ent); free(rowptr); free(col); free(val); free(Dall); free(Oall);
                    return -2;
                }
                double *Dj = &Dall[25 * j], *Oji = &Oall[75 * j + 25 * kb];
                for (int r = 0; r < nj; ++r) {
                    for (int c = 0; c < nj; ++c)
                        for (int p = 0; p < np; ++p) Dj[5 * r + c] += B[p][r] * B[p][c];
                    for (int c = 0; c < ni; ++c)
                        for (int p = 0; p < np; ++p) Oji[5 * r + c] += B[p][r] * A[p][c];
                }
            }
        }
    }
    int nnz = 0;
    for (int i = 0; i < T; ++i) {
        int ni = ndof_of(m->korder[i]);
        for (int r = 0; r < ni; ++r) {
            int row = m->dof_off[i] + r;
            int ne = 0;
            for (int c = 0; c < ni; ++c) { ent[ne].col = m->dof_off[i] + c; ent[ne].v = Dall[25 * i + 5 * r + c]; ++ne; }
            for (int k = 0; k < m->nb_cnt[i]; ++k) {
                int j = m->nb_cell[3 * i + k];
                int nj = ndof_of(m->korder[j]);
                for (int c = 0; c < nj; ++c) {
                    ent[ne].col = m->dof_off[j] + c;
                    ent[ne].v = -Oall[75 * i + 25 * k + 5 * r + c];
                    ++ne;
                }
            }
            qsort(ent, (size_t)ne, sizeof(or_ent), cmp_ent);
            rowptr[row] = nnz;
            for (int e = 0; e < ne; ++e) {               /* merge repeated columns */
                if (e > 0 && ent[e].col == ent[e - 1].col) { val[nnz - 1] += ent[e].v; continue; }
                col[nnz] = ent[e].col; val[nnz] = ent[e].v; ++nnz;
            }
        }
    }
    free(Dall);
    free(Oall);
    rowptr[m->ndof] = nnz;
    free(ent);
    m->K.n = m->ndof; m->K.nnz = nnz; m->K.rowptr = rowptr; m->K.col = col; m->K.val = val;
    return 0;
}

/* Right-hand side sum_j A_ij^T b_ij with b_ij = (ubar_j - ubar_i, 0, 0)
 * (Eq. (25)); only row 0 of A_ij meets the nonzero entry of b_ij. */
void or_cls_rhs_var(const or_mesh *m, const double *ubar, double *rhs)
{
    for (int64_t i = 0; i < m->n_tri; ++i) {
        int ni = ndof_of(m->korder[i]);
        for (int r = 0; r < ni; ++r) {
            double s = 0.0;
            for (int k = 0; k < m->nb_cnt[i]; ++k) {
                int j = m->nb_cell[3 * i + k];
                s += m->a0[15 * i + 5 * k + r] * (ubar[j] - ubar[i]);
            }
            rhs[m->dof_off[i] + r] = s;
        }
    }
}

/* ---------------------------------------------------------------------------
 * Reverse Cuthill-McKee on the cell adjacency graph (Sec. III.B).
 * Start: a pseudo-peripheral cell, found by repeated breadth-first search from
 * the lowest-degree cell, moving to the lowest-degree cell of the last level
 * while the eccentricity grows.  Neighbours are visited in increasing degree,
 * ties broken by index.  The Cuthill-McKee order is reversed at the end.
 */
static int bfs_levels(const or_mesh *m, const int *deg, int start, int *level, int *queue, int *last_out)
{
    const int T = (int)m->n_tri;
    for (int i = 0; i < T; ++i) level[i] = -1;
    int head = 0, tail = 0;
    queue[tail++] = start; level[start] = 0;
    int maxl = 0;
    while (head < tail) {
        int c = queue[head++];
        for (int k = 0; k < m->nb_cnt[c]; ++k) {
            int j = m->nb_cell[3 * c + k];
            if (level[j] < 0) { level[j] = level[c] + 1; if (level[j] > maxl) maxl = level[j]; queue[tail++] = j; }
        }
    }
    int best = -1;
    for (int h = 0; h < tail; ++h) {
        int c = queue[h];
        if (level[c] == maxl && (best < 0 || deg[c] < deg[best] || (deg[c] == deg[best] && c < best))) best = c;
    }
    *last_out = best;
    return maxl;
}

int or_build_rcm(or_mesh *m)
{
    const int T = (int)m->n_tri;
    int *deg = malloc(sizeof(int) * T), *level = malloc(sizeof(int) * T);
    int *queue = malloc(sizeof(int) * T), *order = malloc(sizeof(int) * T);
    char *seen = calloc((size_t)T, 1);
    if (!deg || !level || !queue || !order || !seen) return -1;
    for (int i = 0; i < T; ++i) deg[i] = m->nb_cnt[i];
    int n_out = 0;
    while (n_out < T) {
        int start = -1;
        for (int i = 0; i < T; ++i)
            if (!seen[i] && (start < 0 || deg[i] < deg[start])) start = i;
        /* pseudo-peripheral node within this component */
        int last, ecc = bfs_levels(m, deg, start, level, queue, &last);
        for (;;) {
            int last2, ecc2 = bfs_levels(m, deg, last, level, queue, &last2);
            if (ecc2 <= ecc) break;
            start = last; ecc = ecc2; last = last2;
        }
        /* Cuthill-McKee breadth-first order */
        int head = n_out, tail = n_out;
        order[tail++] = start; seen[start] = 1;
        while (head < tail) {
            int c = order[head++];
            int cand[3], nc = 0;
            for (int k = 0; k < m->nb_cnt[c]; ++k) {
                int j = m->nb_cell[3 * c + k];
                if (!seen[j]) { int dup = 0; for (int q = 0; q < nc; ++q) dup |= cand[q] == j; if (!dup) cand[nc++] = j; }
            }
            for (int a = 1; a < nc; ++a)              /* insertion sort by (degree, index) */
                for (int b = a; b > 0; --b) {
                    int x = cand[b - 1], y = cand[b];
                    if (deg[y] < deg[x] || (deg[y] == deg[x] && y < x)) { cand[b - 1] = y; cand[b] = x; }
                }
            for (int q = 0; q < nc; ++q) { seen[cand[q]] = 1; order[tail++] = cand[q]; }
        }
        n_out = tail;
    }
    for (int i = 0; i < T; ++i) m->perm[i] = order[T - 1 - i];   /* reverse */
    free(deg); free(level); free(queue); free(order); free(seen);

    /* dof permutation following the cell permutation */
    int p = 0;
    for (int i = 0; i < T; ++i) {
        int c = m->perm[i];
        int nc = ndof_of(m->korder[c]);
        for (int r = 0; r < nc; ++r) { m->dperm[p] = m->dof_off[c] + r; m->dinv[m->dof_off[c] + r] = p; ++p; }
    }
    /* permuted matrix Kp = P K P^T with sorted columns */
    const or_csr *K = &m->K;
    or_csr *Kp = &m->Kp;
    Kp->n = K->n; Kp->nnz = K->nnz;
    Kp->rowptr = malloc(sizeof(int) * (size_t)(K->n + 1));
    Kp->col = malloc(sizeof(int) * (size_t)K->nnz);
    Kp->val = malloc(sizeof(double) * (size_t)K->nnz);
    or_ent *ent = malloc(sizeof(or_ent) * 64);
    if (!Kp->rowptr || !Kp->col || !Kp->val || !ent) return -1;
    int nnz = 0;
    for (int r = 0; r < K->n; ++r) {
        int old = m->dperm[r];
        int ne = 0;
        for (int e = K->rowptr[old]; e < K->rowptr[old + 1]; ++e) {
            if (ne == 64) return -2;
            ent[ne].col = m->dinv[K->col[e]]; ent[ne].v = K->val[e]; ++ne;
        }
        qsort(ent, (size_t)ne, sizeof(or_ent), cmp_ent);
        Kp->rowptr[r] = nnz;
        for (int e = 0; e < ne; ++e) { Kp->col[nnz] = ent[e].col; Kp->val[nnz] = ent[e].v; ++nnz; }
    }
    Kp->rowptr[K->n] = nnz;
    free(ent);
    return 0;
}
