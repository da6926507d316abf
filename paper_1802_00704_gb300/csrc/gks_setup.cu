// Host set-up of a mesh handle: geometry, boundary order reduction, RCM order,
// CLS blocks, block ILU(0) factors, level sets, and the upload to HBM.
//
// Geometry-only data (Sec. III.A): the CLS operator depends on the mesh only,
// so it is assembled once here.  For a cell i and a face neighbour j (Eq. (29),
// M = 1 derivative order, weights w_{i,0} = 1 and w_{i,1} = w h_i) the rows of
// A_ij are
//   row 0: mean over cell j of phi_{l,i}                       (= a0 below)
//   row 1: w (1, 0, dx, dy, 0)      row 2: w (0, 1, 0, dx, dy)
// with (dx, dy) the centroid of j in i's scaled frame, and B_ij has only
// w (h_i/h_j) on the gradient entries of rows 1 and 2 (zero-mean basis).  The
// per-cell least-squares normal equations (Eqs. (32)-(33)) give
//   D_i u_i - sum_j O_ij u_j = sum_j A_ij^T b_ij,   D_i = sum_j A_ij^T A_ij,
//   O_ij = A_ij^T B_ij = w^2 (h_i/h_j) [e1 + dx e3 + dy e4 | e2 + dx e4 + dy e5],
// so an off-diagonal block is stored as three numbers (alpha, dx, dy).
// Means of quadratics over a triangle use its centroidal second moments
// (1/12) sum_k (p_k - c)(p_k - c)^T.
#include <algorithm>
#include <array>
#include <cmath>
#include <cstdarg>
#include <cstdio>
#include <cstring>
#include <limits>
#include <numeric>
#include <thread>

#include "gks_internal.h"

namespace gks {

static thread_local char g_err[512];

void set_error(const char *fmt, ...)
{
    va_list ap;
    va_start(ap, fmt);
    vsnprintf(g_err, sizeof(g_err), fmt, ap);
    va_end(ap);
}

const char *last_error() { return g_err; }

namespace {

struct HostCell {
    double area, cx, cy, crad, inrad, h, sxx, sxy, syy;   // s**: centroidal second moments (unscaled)
    int k;
    int nf;
    int face[3];
};

template <typename T>
gks_status dalloc(gks_mesh *m, T **p, size_t n)
{
    void *q = nullptr;
    size_t bytes = std::max<size_t>(n, 1) * sizeof(T);
    cudaError_t e = cudaMalloc(&q, bytes);
    if (e != cudaSuccess) {
        set_error("cudaMalloc(%zu) failed: %s", bytes, cudaGetErrorString(e));
        return e == cudaErrorMemoryAllocation ? GKS_ENOMEM : GKS_ECUDA;
    }
    m->allocations.push_back(q);
    m->device_bytes += (int64_t)bytes;
    *p = static_cast<T *>(q);
    return GKS_OK;
}

template <typename T>
gks_status upload(gks_mesh *m, T **p, const std::vector<T> &h)
{
    gks_status st = dalloc(m, p, h.size());
    if (st != GKS_OK) return st;
    GKS_CUDA(cudaMemcpy(*p, h.data(), h.size() * sizeof(T), cudaMemcpyHostToDevice));
    return GKS_OK;
}

// 5x5 inverse by Gauss-Jordan with partial pivoting (row-major).  Returns false if singular.
bool inv5(const double *a, double *out)
{
    double m[5][10];
    for (int r = 0; r < 5; ++r)
        for (int c = 0; c < 10; ++c) m[r][c] = c < 5 ? a[5 * r + c] : (c - 5 == r ? 1.0 : 0.0);
    for (int c = 0; c < 5; ++c) {
        int p = c;
        for (int r = c + 1; r < 5; ++r)
            if (std::fabs(m[r][c]) > std::fabs(m[p][c])) p = r;
        if (m[p][c] == 0.0) return false;
        if (p != c)
            for (int q = 0; q < 10; ++q) std::swap(m[p][q], m[c][q]);
        double d = 1.0 / m[c][c];
        for (int q = 0; q < 10; ++q) m[c][q] *= d;
        for (int r = 0; r < 5; ++r) {
            if (r == c || m[r][c] == 0.0) continue;
            double f = m[r][c];
            for (int q = 0; q < 10; ++q) m[r][q] -= f * m[c][q];
        }
    }
    for (int r = 0; r < 5; ++r)
        for (int c = 0; c < 5; ++c) out[5 * r + c] = m[r][5 + c];
    return true;
}

// Off-diagonal block O (5x5, row-major) from its three parameters.
void oblock(double alpha, double ex, double ey, double *O)
{
    std::fill(O, O + 25, 0.0);
    O[0 * 5 + 0] = alpha;
    O[1 * 5 + 1] = alpha;
    O[2 * 5 + 0] = alpha * ex;
    O[3 * 5 + 0] = alpha * ey;
    O[3 * 5 + 1] = alpha * ex;
    O[4 * 5 + 1] = alpha * ey;
}

// O += the transpose form alr [e1 (1, 0, exr, eyr, 0) + e2 (0, 1, 0, exr, eyr)]:
// what the global normal equations (Eq. (33)) add to the block (i, j) from j's
// own equations about i (alr = alpha_ji, (exr, eyr) = i's centroid in j's frame).
void oblock_rev(double alr, double exr, double eyr, double *O)
{
    O[0 * 5 + 0] += alr;
    O[0 * 5 + 2] += alr * exr;
    O[0 * 5 + 3] += alr * eyr;
    O[1 * 5 + 1] += alr;
    O[1 * 5 + 3] += alr * exr;
    O[1 * 5 + 4] += alr * eyr;
}

// Reverse Cuthill-McKee order (new -> old) of the cell graph given by adjacency lists.
// Start vertex of each component: a pseudo-peripheral vertex found by repeated
// breadth-first searches (George & Liu); neighbours are queued by increasing degree.
std::vector<int32_t> rcm_order(const std::vector<std::array<int32_t, 3>> &adj, const std::vector<int> &deg)
{
    const int64_t T = (int64_t)adj.size();
    std::vector<int32_t> order;
    order.reserve(T);
    std::vector<char> done(T, 0);
    std::vector<int32_t> level(T, -1), queue(T);
    auto bfs = [&](int32_t s, int32_t &far) {
        // returns eccentricity; far = min-degree vertex of the last level
        int64_t head = 0, tail = 0;
        queue[tail++] = s;
        level[s] = 0;
        int ecc = 0;
        while (head < tail) {
            int32_t c = queue[head++];
            for (int q = 0; q < deg[c]; ++q) {
                int32_t j = adj[c][q];
                if (level[j] < 0) {
                    level[j] = level[c] + 1;
                    ecc = std::max(ecc, level[j]);
                    queue[tail++] = j;
                }
            }
        }
        far = -1;
        for (int64_t q = 0; q < tail; ++q) {
            int32_t c = queue[q];
            if (level[c] == ecc && (far < 0 || deg[c] < deg[far] || (deg[c] == deg[far] && c < far))) far = c;
        }
        for (int64_t q = 0; q < tail; ++q) level[queue[q]] = -1;
        return ecc;
    };
    for (int64_t seed = 0; seed < T; ++seed) {
        if (done[seed]) continue;
        // first unvisited vertex, then walk to a pseudo-peripheral one
        int32_t s = (int32_t)seed;
        int32_t far;
        int ecc = bfs(s, far);
        for (int it = 0; it < 32; ++it) {
            int32_t far2;
            int ecc2 = bfs(far, far2);
            if (ecc2 <= ecc) break;
            s = far;
            ecc = ecc2;
            far = far2;
        }
        int64_t head = (int64_t)order.size();
        order.push_back(s);
        done[s] = 1;
        while (head < (int64_t)order.size()) {
            int32_t c = order[head++];
            int32_t cand[3];
            int nc = 0;
            for (int q = 0; q < deg[c]; ++q) {
                int32_t j = adj[c][q];
                if (!done[j]) {
                    done[j] = 1;
                    cand[nc++] = j;
                }
            }
            std::sort(cand, cand + nc, [&](int32_t a, int32_t b) { return deg[a] != deg[b] ? deg[a] < deg[b] : a < b; });
            for (int q = 0; q < nc; ++q) order.push_back(cand[q]);
        }
    }
    std::reverse(order.begin(), order.end());
    return order;
}

}  // namespace

namespace {

// Host data of one case in its own RCM order (local indices).
struct HostCase {
    int64_t T = 0, F = 0, nbf = 0, nk1 = 0, nnzb = 0, bw = 0;
    int32_t nlo = 0, nup = 0;
    std::vector<int32_t> perm, nb, cf, fl, fr, ftag, fperm, lev_lo, lev_up, kord;
    std::vector<double> area, iarea, h, mxx, mxy, myy, inrad, alpha, ex, ey, ox, oy, a0, D, P;
    std::vector<double> alr, exr, eyr, bdg;   // extended stencil only (empty otherwise)
    std::vector<double> fnx, fny, flen, gl, gr, bc;
};

// Geometry, boundary order reduction (Eq. (28)), RCM order, CLS blocks
// (Eq. (29)), block ILU(0) factors and levels of one case.
gks_status build_case(const CaseIn &in, double w, int second_order, int cls_global, int cls_M, HostCase &hc)
{
    const double *nodes = in.nodes, *face_shift = in.face_shift, *bc_state = in.bc_state;
    const int32_t *tris = in.tris, *faces = in.faces;
    const int64_t n_nodes = in.n_nodes, T = in.n_tri, F = in.n_face;
    if (!nodes || !tris || !faces || !face_shift || !bc_state || n_nodes <= 0 || T <= 0 || F <= 0 ||
        T > (int64_t)INT32_MAX / 8 || F > (int64_t)INT32_MAX / 8) {
        set_error("gks_mesh_create: null array or size out of range");
        return GKS_EINVAL;
    }
    // ---- cells: orientation, area, centroid, radii, length scale (Eq. (17))
    std::vector<HostCell> cell(T);
    for (int64_t i = 0; i < T; ++i) {
        const int32_t *t = tris + 3 * i;
        for (int q = 0; q < 3; ++q)
            if (t[q] < 0 || t[q] >= n_nodes) {
                set_error("gks_mesh_create: triangle %lld has node index %d out of range", (long long)i, t[q]);
                return GKS_EINVAL;
            }
        double px[3], py[3];
        for (int q = 0; q < 3; ++q) { px[q] = nodes[2 * t[q]]; py[q] = nodes[2 * t[q] + 1]; }
        double a2 = (px[1] - px[0]) * (py[2] - py[0]) - (px[2] - px[0]) * (py[1] - py[0]);
        if (!(std::fabs(a2) > 0.0) || !std::isfinite(a2)) {
            set_error("gks_mesh_create: triangle %lld is degenerate", (long long)i);
            return GKS_EINVAL;
        }
        HostCell &c = cell[i];
        c.area = 0.5 * std::fabs(a2);
        c.cx = (px[0] + px[1] + px[2]) / 3.0;
        c.cy = (py[0] + py[1] + py[2]) / 3.0;
        double e0 = std::hypot(px[1] - px[0], py[1] - py[0]);
        double e1 = std::hypot(px[2] - px[1], py[2] - py[1]);
        double e2 = std::hypot(px[0] - px[2], py[0] - py[2]);
        c.crad = e0 * e1 * e2 / (4.0 * c.area);
        c.inrad = 2.0 * c.area / (e0 + e1 + e2);
        c.h = std::max(c.crad, std::sqrt(c.area));
        c.sxx = c.sxy = c.syy = 0.0;
        for (int q = 0; q < 3; ++q) {
            double dx = px[q] - c.cx, dy = py[q] - c.cy;
            c.sxx += dx * dx / 12.0;
            c.sxy += dx * dy / 12.0;
            c.syy += dy * dy / 12.0;
        }
        c.k = second_order ? 1 : 2;     // the second-order variant is linear everywhere
        c.nf = 0;
        c.face[0] = c.face[1] = c.face[2] = -1;
    }

    // ---- faces: validation, incidence, boundary order reduction (Eq. (28))
    int64_t nbf = 0;
    for (int64_t f = 0; f < F; ++f) {
        const int32_t *fc = faces + 5 * f;
        bool bad = fc[0] < 0 || fc[0] >= n_nodes || fc[1] < 0 || fc[1] >= n_nodes || fc[2] < 0 || fc[2] >= T ||
                   fc[3] < -1 || fc[3] >= T || fc[4] < GKS_BC_INTERIOR || fc[4] > GKS_BC_NOSLIP || fc[2] == fc[3];
        bad = bad || ((fc[3] < 0) != (fc[4] >= GKS_BC_DIRICHLET));
        if (bad) {
            set_error("gks_mesh_create: face %lld is invalid (indices or tag)", (long long)f);
            return GKS_EINVAL;
        }
        for (int side = 0; side < 2; ++side) {
            int32_t c = fc[2 + side];
            if (c < 0) continue;
            if (cell[c].nf == 3) {
                set_error("gks_mesh_create: cell %d has more than three faces", c);
                return GKS_EINVAL;
            }
            cell[c].face[cell[c].nf++] = (int32_t)(2 * f + side);
        }
        if (fc[3] < 0) {
            cell[fc[2]].k = 1;
            ++nbf;
        }
    }

    // ---- cell graph and RCM order (Sec. III.B)
    std::vector<std::array<int32_t, 3>> adj(T);
    std::vector<int> deg(T, 0);
    for (int64_t i = 0; i < T; ++i)
        for (int q = 0; q < cell[i].nf; ++q) {
            int64_t f = cell[i].face[q] >> 1;
            int side = cell[i].face[q] & 1;
            int32_t j = faces[5 * f + 3 - side];   // the other cell
            if (j < 0) continue;
            bool dup = false;
            for (int p = 0; p < deg[i]; ++p) dup = dup || adj[i][p] == j;
            if (!dup) adj[i][deg[i]++] = j;
        }
    std::vector<int32_t> perm = rcm_order(adj, deg);   // internal -> caller
    std::vector<int32_t> inv(T);
    for (int64_t i = 0; i < T; ++i) inv[perm[i]] = (int32_t)i;

    // ---- CLS blocks in internal order
    std::vector<int32_t> h_nb(3 * T, -1), h_cf(3 * T, -1);
    std::vector<double> h_alpha(3 * T, 0.0), h_ex(3 * T, 0.0), h_ey(3 * T, 0.0), h_a0(15 * T, 0.0);
    // extended stencil: global normal equations (the reverse slot's coefficients alpha_ji and i's
    // centroid in j's frame) and second-derivative equations (the diagonal coupling beta on unknowns 3..5)
    std::vector<double> h_alr(3 * T, 0.0), h_exr(3 * T, 0.0), h_eyr(3 * T, 0.0), h_bdg(3 * T, 0.0);
    std::vector<double> h_ox(3 * T, 0.0), h_oy(3 * T, 0.0);
    std::vector<int32_t> h_kord(T, 2);
    std::vector<double> h_D(15 * T, 0.0), h_Dfull(25 * T, 0.0);
    std::vector<double> h_area(T), h_iarea(T), h_h(T), h_mxx(T), h_mxy(T), h_myy(T), h_inrad(T);
    int64_t nk1 = 0, nnzb = 0, bw = 0;
    for (int64_t i = 0; i < T; ++i) {
        const HostCell &c = cell[perm[i]];
        h_area[i] = c.area;
        h_iarea[i] = 1.0 / c.area;
        h_h[i] = c.h;
        h_mxx[i] = c.sxx / (c.h * c.h);
        h_mxy[i] = c.sxy / (c.h * c.h);
        h_myy[i] = c.syy / (c.h * c.h);
        h_inrad[i] = c.inrad;
        h_kord[i] = c.k;
        nk1 += c.k == 1;
    }
    for (int64_t i = 0; i < T; ++i) {
        const int32_t ci = perm[i];
        const HostCell &c = cell[ci];
        const int ni = c.k == 2 ? 5 : 2;
        double D[25] = {0};
        int slot = 0;
        for (int q = 0; q < c.nf; ++q) {
            int64_t f = c.face[q] >> 1;
            int side = c.face[q] & 1;
            int32_t cj = faces[5 * f + 3 - side];
            if (cj < 0) continue;
            // translation of j's coordinates next to i
            double ox = side == 0 ? face_shift[2 * f] : -face_shift[2 * f];
            double oy = side == 0 ? face_shift[2 * f + 1] : -face_shift[2 * f + 1];
            const HostCell &d = cell[cj];
            double dx = (d.cx + ox - c.cx) / c.h, dy = (d.cy + oy - c.cy) / c.h;
            double s2 = 1.0 / (c.h * c.h);
            double a0[5] = {dx, dy, 0.5 * (dx * dx + d.sxx * s2 - h_mxx[i]), dx * dy + d.sxy * s2 - h_mxy[i],
                            0.5 * (dy * dy + d.syy * s2 - h_myy[i])};
            // derivative rows of Eq. (29) up to order M: p = 1 (w (1, 0, dx, dy, 0), w (0, 1, 0, dx, dy));
            // p = 2 (w^2 e3, e4, e5 for a quadratic cell; the B rows (w h_i / h_j)^2 e3.. of a quadratic j)
            const double f1 = cls_M >= 1 ? 1.0 : 0.0;
            double r1[5] = {f1 * w, 0.0, f1 * w * dx, f1 * w * dy, 0.0};
            double r2[5] = {0.0, f1 * w, 0.0, f1 * w * dx, f1 * w * dy};
            for (int a = 0; a < ni; ++a)
                for (int b = 0; b < ni; ++b) D[5 * a + b] += a0[a] * a0[b] + r1[a] * r1[b] + r2[a] * r2[b];
            const double w4 = w * w * w * w;
            if (cls_M == 2 && c.k == 2) {
                for (int a = 2; a < 5; ++a) D[5 * a + a] += w4;
                if (d.k == 2) h_bdg[slot * T + i] = w4 * (c.h / d.h) * (c.h / d.h);
            }
            if (cls_global && cls_M >= 1) {
                // j's equations about i (Eq. (33)): their B rows (w h_j / h_i) e1, e2 act on u_i
                const double q = w * d.h / c.h;
                D[0] += q * q;
                D[6] += q * q;
                h_alr[slot * T + i] = w * w * d.h / c.h;
                h_exr[slot * T + i] = d.k == 2 ? (c.cx - ox - d.cx) / d.h : 0.0;
                h_eyr[slot * T + i] = d.k == 2 ? (c.cy - oy - d.cy) / d.h : 0.0;
                if (cls_M == 2 && c.k == 2) {
                    // and their second-derivative B rows (w h_j / h_i)^2 e3.. on a quadratic i
                    const double q2 = q * q;
                    for (int a = 2; a < 5; ++a) D[5 * a + a] += q2 * q2;
                    if (d.k == 2) h_bdg[slot * T + i] += w4 * (d.h / c.h) * (d.h / c.h);
                }
            }
            int32_t j = inv[cj];
            h_nb[slot * T + i] = j;
            h_alpha[slot * T + i] = cls_M >= 1 ? w * w * c.h / d.h : 0.0;
            h_ex[slot * T + i] = c.k == 2 ? dx : 0.0;
            h_ey[slot * T + i] = c.k == 2 ? dy : 0.0;
            h_ox[slot * T + i] = dx;
            h_oy[slot * T + i] = dy;
            for (int l = 0; l < 5; ++l) h_a0[(slot * 5 + l) * T + i] = l < ni ? a0[l] : 0.0;
            bw = std::max<int64_t>(bw, std::llabs((long long)(j - i)));
            ++slot;
            ++nnzb;
        }
        for (int a = ni; a < 5; ++a) D[5 * a + a] = 1.0;    // padding of k = 1 cells
        int u = 0;
        for (int a = 0; a < 5; ++a)
            for (int b = a; b < 5; ++b) h_D[(u++) * T + i] = D[5 * a + b];
        std::copy(D, D + 25, &h_Dfull[25 * i]);
        ++nnzb;
    }

    // ---- block ILU(0) in internal (RCM) order: only diagonal blocks change,
    // Dt_i = D_i - sum_{k<i} O_ik Dt_k^{-1} O_ki, because no two face
    // neighbours of a triangle are face neighbours of each other.
    std::vector<double> h_P(25 * T, 0.0), Pinv(25 * T, 0.0);
    for (int64_t i = 0; i < T; ++i) {
        double Dt[25];
        std::copy(&h_Dfull[25 * i], &h_Dfull[25 * i] + 25, Dt);
        for (int s = 0; s < 3; ++s) {
            int32_t k = h_nb[s * T + i];
            if (k < 0 || k >= i) continue;
            double Oik[25];
            oblock(h_alpha[s * T + i], h_ex[s * T + i], h_ey[s * T + i], Oik);
            if (cls_global) oblock_rev(h_alr[s * T + i], h_exr[s * T + i], h_eyr[s * T + i], Oik);
            for (int a = 2; a < 5; ++a) Oik[5 * a + a] += h_bdg[s * T + i];
            for (int s2 = 0; s2 < 3; ++s2) {
                if (h_nb[s2 * T + k] != (int32_t)i) continue;
                double Oki[25], tmp[25];
                oblock(h_alpha[s2 * T + k], h_ex[s2 * T + k], h_ey[s2 * T + k], Oki);
                if (cls_global) oblock_rev(h_alr[s2 * T + k], h_exr[s2 * T + k], h_eyr[s2 * T + k], Oki);
                for (int a = 2; a < 5; ++a) Oki[5 * a + a] += h_bdg[s2 * T + k];
                const double *Pk = &Pinv[25 * k];
                for (int a = 0; a < 5; ++a)
                    for (int b = 0; b < 5; ++b) {
                        double sacc = 0.0;
                        for (int q = 0; q < 5; ++q) sacc += Pk[5 * a + q] * Oki[5 * q + b];
                        tmp[5 * a + b] = sacc;
                    }
                for (int a = 0; a < 5; ++a)
                    for (int b = 0; b < 5; ++b) {
                        double sacc = 0.0;
                        for (int q = 0; q < 5; ++q) sacc += Oik[5 * a + q] * tmp[5 * q + b];
                        Dt[5 * a + b] -= sacc;
                    }
            }
        }
        if (!inv5(Dt, &Pinv[25 * i])) {
            set_error("gks_mesh_create: singular ILU(0) pivot block at cell %d", perm[i]);
            return GKS_EINVAL;
        }
    }
    for (int64_t i = 0; i < T; ++i)
        for (int q = 0; q < 25; ++q) h_P[q * T + i] = Pinv[25 * i + q];

    // ---- level sets of the two triangular solves
    std::vector<int32_t> lev(T, 0);
    int32_t nlo = 0, nup = 0;
    for (int64_t i = 0; i < T; ++i) {
        int32_t l = 0;
        for (int s = 0; s < 3; ++s) {
            int32_t k = h_nb[s * T + i];
            if (k >= 0 && k < i) l = std::max(l, lev[k] + 1);
        }
        lev[i] = l;
        nlo = std::max(nlo, l + 1);
    }
    hc.lev_lo = lev;
    hc.nlo = nlo;
    for (int64_t i = T - 1; i >= 0; --i) {
        int32_t l = 0;
        for (int s = 0; s < 3; ++s) {
            int32_t k = h_nb[s * T + i];
            if (k > i) l = std::max(l, lev[k] + 1);
        }
        lev[i] = l;
        nup = std::max(nup, l + 1);
    }
    // lev[] now holds the backward levels (rows with higher indices first)
    hc.lev_up = lev;
    hc.nup = nup;

    // ---- faces in internal order (sorted by the lower internal cell index)
    std::vector<int64_t> forder(F);
    std::iota(forder.begin(), forder.end(), 0);
    auto fkey = [&](int64_t f) {
        int32_t l = inv[faces[5 * f + 2]];
        int32_t r = faces[5 * f + 3] >= 0 ? inv[faces[5 * f + 3]] : l;
        return std::min(l, r);
    };
    std::stable_sort(forder.begin(), forder.end(), [&](int64_t a, int64_t b) { return fkey(a) < fkey(b); });
    std::vector<int32_t> h_fl(F), h_fr(F), h_ftag(F), h_fperm(F);
    std::vector<double> h_fnx(F), h_fny(F), h_flen(F), h_gl(4 * F), h_gr(4 * F, 0.0), h_bc(4 * F);
    std::vector<int32_t> finv(F);
    const double s0 = 0.5 - 0.5 / std::sqrt(3.0), s1 = 0.5 + 0.5 / std::sqrt(3.0);
    for (int64_t q = 0; q < F; ++q) {
        int64_t f = forder[q];
        finv[f] = (int32_t)q;
        const int32_t *fc = faces + 5 * f;
        h_fperm[q] = (int32_t)f;
        h_fl[q] = inv[fc[2]];
        h_fr[q] = fc[3] >= 0 ? inv[fc[3]] : -1;
        h_ftag[q] = fc[4];
        double ax = nodes[2 * fc[0]], ay = nodes[2 * fc[0] + 1], bx = nodes[2 * fc[1]], by = nodes[2 * fc[1] + 1];
        double len = std::hypot(bx - ax, by - ay);
        if (!(len > 0.0)) {
            set_error("gks_mesh_create: face %lld has zero length", (long long)f);
            return GKS_EINVAL;
        }
        double nx = (by - ay) / len, ny = -(bx - ax) / len;
        const HostCell &cl = cell[fc[2]];
        if (nx * (0.5 * (ax + bx) - cl.cx) + ny * (0.5 * (ay + by) - cl.cy) < 0.0) {
            nx = -nx;
            ny = -ny;
        }
        h_fnx[q] = nx;
        h_fny[q] = ny;
        h_flen[q] = len;
        double gx[2] = {ax + s0 * (bx - ax), ax + s1 * (bx - ax)};
        double gy[2] = {ay + s0 * (by - ay), ay + s1 * (by - ay)};
        for (int g = 0; g < 2; ++g) {
            h_gl[(2 * g) * F + q] = (gx[g] - cl.cx) / cl.h;
            h_gl[(2 * g + 1) * F + q] = (gy[g] - cl.cy) / cl.h;
            if (fc[3] >= 0) {
                const HostCell &cr = cell[fc[3]];
                h_gr[(2 * g) * F + q] = (gx[g] - face_shift[2 * f] - cr.cx) / cr.h;
                h_gr[(2 * g + 1) * F + q] = (gy[g] - face_shift[2 * f + 1] - cr.cy) / cr.h;
            }
        }
        for (int v = 0; v < 4; ++v) h_bc[v * F + q] = bc_state[4 * f + v];
    }
    for (int64_t i = 0; i < T; ++i) {
        const HostCell &c = cell[perm[i]];
        for (int q = 0; q < c.nf; ++q) {
            int64_t f = c.face[q] >> 1;
            h_cf[q * T + i] = (finv[f] << 1) | (c.face[q] & 1);
        }
    }

    hc.T = T;
    hc.F = F;
    hc.nbf = nbf;
    hc.nk1 = nk1;
    hc.nnzb = nnzb;
    hc.bw = bw;
    hc.perm = std::move(perm);
    hc.nb = std::move(h_nb);
    hc.cf = std::move(h_cf);
    hc.area = std::move(h_area);
    hc.iarea = std::move(h_iarea);
    hc.h = std::move(h_h);
    hc.mxx = std::move(h_mxx);
    hc.mxy = std::move(h_mxy);
    hc.myy = std::move(h_myy);
    hc.inrad = std::move(h_inrad);
    hc.alpha = std::move(h_alpha);
    if (cls_global || cls_M == 2) {
        hc.alr = std::move(h_alr);
        hc.exr = std::move(h_exr);
        hc.eyr = std::move(h_eyr);
        hc.bdg = std::move(h_bdg);
    }
    hc.ex = std::move(h_ex);
    hc.ey = std::move(h_ey);
    hc.ox = std::move(h_ox);
    hc.oy = std::move(h_oy);
    hc.kord = std::move(h_kord);
    hc.a0 = std::move(h_a0);
    hc.D = std::move(h_D);
    hc.P = std::move(h_P);
    hc.fl = std::move(h_fl);
    hc.fr = std::move(h_fr);
    hc.ftag = std::move(h_ftag);
    hc.fperm = std::move(h_fperm);
    hc.fnx = std::move(h_fnx);
    hc.fny = std::move(h_fny);
    hc.flen = std::move(h_flen);
    hc.gl = std::move(h_gl);
    hc.gr = std::move(h_gr);
    hc.bc = std::move(h_bc);
    return GKS_OK;
}

// Copy rows [k][n] of a case array into rows [k][N] of the global array at column off.
template <typename V>
void place(const std::vector<V> &src, int64_t n, int k, std::vector<V> &dst, int64_t N, int64_t off)
{
    for (int q = 0; q < k; ++q) std::copy(src.begin() + q * n, src.begin() + (q + 1) * n, dst.begin() + q * N + off);
}

}  // namespace

gks_status build_batch(gks_mesh *m, const CaseIn *cases, int32_t n_cases)
{
    if (!cases || n_cases <= 0) {
        set_error("gks_mesh_create: no case");
        return GKS_EINVAL;
    }
    const gks_config &cfg = m->cfg;
    std::vector<HostCase> hcs(n_cases);
    {
        // cases are independent: build them on all host threads
        std::atomic<int32_t> next{0};
        std::atomic<int> failed{-1};
        std::vector<gks_status> st(n_cases, GKS_OK);
        std::vector<std::string> msg(n_cases);
        unsigned nt = std::max(1u, std::min<unsigned>(std::thread::hardware_concurrency(), (unsigned)n_cases));
        auto work = [&]() {
            for (int32_t c; (c = next.fetch_add(1)) < n_cases;) {
                st[c] = build_case(cases[c], cfg.cls_w, cfg.second_order, cfg.cls_global, cfg.cls_M, hcs[c]);
                if (st[c] != GKS_OK) {
                    msg[c] = last_error();
                    int expect = -1;
                    failed.compare_exchange_strong(expect, c);
                }
            }
        };
        std::vector<std::thread> pool;
        for (unsigned q = 1; q < nt; ++q) pool.emplace_back(work);
        work();
        for (auto &t : pool) t.join();
        if (failed.load() >= 0) {
            const int c = failed.load();
            set_error("case %d: %s", c, msg[c].c_str());
            return st[c];
        }
    }
    // ---- layout: cases one after the other, each padded to whole blocks when batched
    const bool pad = n_cases > 1;
    std::vector<int64_t> coff(n_cases + 1, 0), foff(n_cases + 1, 0), ccell(n_cases + 1, 0), cface(n_cases + 1, 0);
    for (int32_t c = 0; c < n_cases; ++c) {
        const int64_t Tc = hcs[c].T;
        coff[c + 1] = coff[c] + (pad ? (Tc + kBlock - 1) / kBlock * kBlock : Tc);
        foff[c + 1] = foff[c] + hcs[c].F;
        ccell[c + 1] = ccell[c] + Tc;
        cface[c + 1] = cface[c] + hcs[c].F;
    }
    const int64_t T = coff[n_cases], F = foff[n_cases];
    if (T > (int64_t)INT32_MAX / 2 || F > (int64_t)INT32_MAX / 2) {
        set_error("gks_mesh_create: too many cells or faces");
        return GKS_EINVAL;
    }
    const int64_t nblk = (T + kBlock - 1) / kBlock;
    std::vector<int32_t> h_perm(T, -1), h_nb(3 * T, -1), h_cf(3 * T, -1), h_blk_case(nblk, 0), h_case_blk(n_cases + 1);
    std::vector<double> h_area(T, 1.0), h_iarea(T, 1.0), h_h(T, 1.0), h_mxx(T, 0.0), h_mxy(T, 0.0), h_myy(T, 0.0);
    std::vector<double> h_inrad(T, std::numeric_limits<double>::infinity());
    std::vector<double> h_alpha(3 * T, 0.0), h_ex(3 * T, 0.0), h_ey(3 * T, 0.0), h_a0(15 * T, 0.0);
    std::vector<double> h_ox(3 * T, 0.0), h_oy(3 * T, 0.0);
    // extended stencil (global normal equations or second-derivative equations)
    const bool ext = cfg.cls_global || cfg.cls_M == 2;
    std::vector<double> h_alr(ext ? 3 * T : 0, 0.0), h_exr(h_alr.size(), 0.0), h_eyr(h_alr.size(), 0.0);
    std::vector<double> h_bdg(h_alr.size(), 0.0);
    std::vector<int32_t> h_kord(T, 2);
    std::vector<double> h_D(15 * T, 0.0), h_P(25 * T, 0.0);
    std::vector<int32_t> h_fl(F), h_fr(F), h_ftag(F), h_fperm(F), h_face_case(F);
    std::vector<double> h_fnx(F), h_fny(F), h_flen(F), h_gl(4 * F), h_gr(4 * F), h_bc(4 * F);
    // padding cells: identity diagonal and pivot blocks, no neighbours, no faces
    for (int64_t i = 0; i < T; ++i) {
        h_D[0 * T + i] = h_D[5 * T + i] = h_D[9 * T + i] = h_D[12 * T + i] = h_D[14 * T + i] = 1.0;
        for (int a = 0; a < 5; ++a) h_P[(6 * a) * T + i] = 1.0;
    }
    int32_t nlo = 0, nup = 0;
    m->n_tri = m->n_face = m->n_bface = m->n_k1 = m->nnzb = m->bandwidth = 0;
    m->case_tri.assign(n_cases, 0);
    m->case_face.assign(n_cases, 0);
    for (int32_t c = 0; c < n_cases; ++c) {
        HostCase &hc = hcs[c];
        const int64_t Tc = hc.T, Fc = hc.F, o = coff[c], fo = foff[c];
        h_case_blk[c] = (int32_t)(o / kBlock);
        for (int64_t b = o / kBlock; b < (coff[c + 1] + kBlock - 1) / kBlock; ++b) h_blk_case[b] = c;
        for (int64_t i = 0; i < Tc; ++i) {
            h_perm[o + i] = (int32_t)(ccell[c] + hc.perm[i]);
            for (int s = 0; s < 3; ++s) {
                const int32_t j = hc.nb[s * Tc + i];
                h_nb[s * T + o + i] = j >= 0 ? (int32_t)(o + j) : -1;
                const int32_t f = hc.cf[s * Tc + i];
                h_cf[s * T + o + i] = f >= 0 ? (int32_t)(((fo + (f >> 1)) << 1) | (f & 1)) : -1;
            }
        }
        place(hc.area, Tc, 1, h_area, T, o); place(hc.iarea, Tc, 1, h_iarea, T, o); place(hc.h, Tc, 1, h_h, T, o);
        place(hc.mxx, Tc, 1, h_mxx, T, o); place(hc.mxy, Tc, 1, h_mxy, T, o); place(hc.myy, Tc, 1, h_myy, T, o);
        place(hc.inrad, Tc, 1, h_inrad, T, o);
        place(hc.alpha, Tc, 3, h_alpha, T, o); place(hc.ex, Tc, 3, h_ex, T, o); place(hc.ey, Tc, 3, h_ey, T, o);
        place(hc.ox, Tc, 3, h_ox, T, o); place(hc.oy, Tc, 3, h_oy, T, o); place(hc.kord, Tc, 1, h_kord, T, o);
        if (ext) {
            place(hc.alr, Tc, 3, h_alr, T, o); place(hc.exr, Tc, 3, h_exr, T, o); place(hc.eyr, Tc, 3, h_eyr, T, o);
            place(hc.bdg, Tc, 3, h_bdg, T, o);
        }
        place(hc.a0, Tc, 15, h_a0, T, o); place(hc.D, Tc, 15, h_D, T, o); place(hc.P, Tc, 25, h_P, T, o);
        for (int64_t f = 0; f < Fc; ++f) {
            h_fl[fo + f] = (int32_t)(o + hc.fl[f]);
            h_fr[fo + f] = hc.fr[f] >= 0 ? (int32_t)(o + hc.fr[f]) : -1;
            h_ftag[fo + f] = hc.ftag[f];
            h_fperm[fo + f] = (int32_t)(cface[c] + hc.fperm[f]);
            h_face_case[fo + f] = c;
        }
        place(hc.fnx, Fc, 1, h_fnx, F, fo); place(hc.fny, Fc, 1, h_fny, F, fo); place(hc.flen, Fc, 1, h_flen, F, fo);
        place(hc.gl, Fc, 4, h_gl, F, fo); place(hc.gr, Fc, 4, h_gr, F, fo); place(hc.bc, Fc, 4, h_bc, F, fo);
        nlo = std::max(nlo, hc.nlo);
        nup = std::max(nup, hc.nup);
        m->n_tri += Tc;
        m->n_face += Fc;
        m->n_bface += hc.nbf;
        m->n_k1 += hc.nk1;
        m->nnzb += hc.nnzb;
        m->bandwidth = std::max(m->bandwidth, hc.bw);
        m->case_tri[c] = Tc;
        m->case_face[c] = Fc;
    }
    h_case_blk[n_cases] = (int32_t)nblk;
    // level sets: the rows of every case at level l are solved together
    auto bucket = [&](int32_t nlev, bool lower, std::vector<int32_t> &rows, std::vector<int32_t> &ptr) {
        ptr.assign(nlev + 1, 0);
        for (int32_t c = 0; c < n_cases; ++c)
            for (int64_t i = 0; i < hcs[c].T; ++i) ++ptr[(lower ? hcs[c].lev_lo[i] : hcs[c].lev_up[i]) + 1];
        for (int32_t l = 0; l < nlev; ++l) ptr[l + 1] += ptr[l];
        std::vector<int32_t> fill(ptr.begin(), ptr.end() - 1);
        rows.assign(ptr[nlev], 0);
        for (int32_t c = 0; c < n_cases; ++c)
            for (int64_t i = 0; i < hcs[c].T; ++i)
                rows[fill[lower ? hcs[c].lev_lo[i] : hcs[c].lev_up[i]]++] = (int32_t)(coff[c] + i);
    };
    std::vector<int32_t> rows_lo, rows_up;
    bucket(nlo, true, rows_lo, m->lvl_lo_ptr);
    bucket(nup, false, rows_up, m->lvl_up_ptr);
    hcs.clear();

    // ---- upload
    m->n_case = n_cases;
    DeviceMesh &d = m->d;
    d.T = T;
    d.F = F;
    d.ncase = n_cases;
    gks_status st;
#define UP(ptr, vec) \
    if ((st = upload(m, &d.ptr, vec)) != GKS_OK) return st
    UP(area, h_area); UP(inv_area, h_iarea); UP(h, h_h); UP(mxx, h_mxx); UP(mxy, h_mxy); UP(myy, h_myy);
    UP(inrad, h_inrad); UP(nb, h_nb); UP(alpha, h_alpha); UP(ex, h_ex); UP(ey, h_ey); UP(a0, h_a0);
    UP(D, h_D); UP(P, h_P); UP(cf, h_cf); UP(perm, h_perm); UP(lvl_lo, rows_lo); UP(lvl_up, rows_up);
    UP(fl, h_fl); UP(fr, h_fr); UP(ftag, h_ftag); UP(fperm, h_fperm); UP(fnx, h_fnx); UP(fny, h_fny);
    UP(flen, h_flen); UP(gl, h_gl); UP(gr, h_gr); UP(bc, h_bc);
    UP(blk_case, h_blk_case); UP(case_blk, h_case_blk); UP(face_case, h_face_case);
    if (ext) {
        UP(alr, h_alr); UP(exr, h_exr); UP(eyr, h_eyr); UP(bdg, h_bdg);
    }

    if (cfg.limiter) {
        UP(ox, h_ox); UP(oy, h_oy); UP(kord, h_kord);
    }
    if (cfg.precision == GKS_MIXED) {
        auto f32 = [](const std::vector<double> &v) { return std::vector<float>(v.begin(), v.end()); };
        UP(D32, f32(h_D)); UP(P32, f32(h_P)); UP(alpha32, f32(h_alpha)); UP(ex32, f32(h_ex)); UP(ey32, f32(h_ey));
        if (ext) {
            UP(alr32, f32(h_alr)); UP(exr32, f32(h_exr)); UP(eyr32, f32(h_eyr)); UP(bdg32, f32(h_bdg));
        }
        if (cfg.ilu_fp16) {
            // FP16 copies of the ILU(0) factors if every value fits FP16's normal range
            // (smaller ones round to FP16's subnormals, far below the block's scale)
            bool fits = true;
            auto f16 = [&](const std::vector<double> &v) {
                std::vector<__half> o(v.size());
                for (size_t q = 0; q < v.size(); ++q) {
                    if (!(std::fabs(v[q]) <= 6.0e4)) fits = false;
                    o[q] = __double2half(v[q]);
                }
                return o;
            };
            std::vector<__half> p16 = f16(h_P), a16 = f16(h_alpha), x16 = f16(h_ex), y16 = f16(h_ey);
            std::vector<__half> ar16 = f16(h_alr), xr16 = f16(h_exr), yr16 = f16(h_eyr), b16 = f16(h_bdg);
            if (fits) {
                UP(P16, p16); UP(alpha16, a16); UP(ex16, x16); UP(ey16, y16);
                if (ext) {
                    UP(alr16, ar16); UP(exr16, xr16); UP(eyr16, yr16); UP(bdg16, b16);
                }
            }
        }
        std::vector<float> h_ih32(T);
        for (int64_t i = 0; i < T; ++i) h_ih32[i] = float(1.0 / h_h[i]);
        UP(ih32, h_ih32);
        // FP32 pairs of the geometry the double-FP32 flux reads
        auto pairs = [](std::vector<const std::vector<double> *> rows, double scale) {
            const size_t n = rows[0]->size(), nr = rows.size();
            std::vector<float> o(2 * nr * n);
            for (size_t r = 0; r < nr; ++r)
                for (size_t q = 0; q < n; ++q) {
                    const double v = scale * (*rows[r])[q];
                    o[r * n + q] = float(v);
                    o[(nr + r) * n + q] = float(v - double(o[r * n + q]));
                }
            return o;
        };
        auto rows4 = [](const std::vector<double> &g, int64_t n) {
            std::vector<std::vector<double>> r(4);
            for (int q = 0; q < 4; ++q) r[q].assign(g.begin() + q * n, g.begin() + (q + 1) * n);
            return r;
        };
        {
            const std::vector<std::vector<double>> glr = rows4(h_gl, F), grr = rows4(h_gr, F);
            UP(m2, pairs({&h_mxx, &h_mxy, &h_myy}, 1.0));
            UP(gl2, pairs({&glr[0], &glr[1], &glr[2], &glr[3]}, 1.0));
            UP(gr2, pairs({&grr[0], &grr[1], &grr[2], &grr[3]}, 1.0));
            UP(fn2, pairs({&h_fnx, &h_fny}, 1.0));
            UP(flen2, pairs({&h_flen}, 0.5));
        }
        if (cfg.basis_fp32) {
            // FP32 pairs of the operator: v = hi + lo to 2^-48 for v = 0 or 2^-74 <= |v| <= 2^30
            // (the bound on |v| keeps the parts of x the residual drops negligible)
            bool in_range = true;
            auto pair = [&](double v, float &hi, float &lo) {
                const double a = std::fabs(v);
                if (v != 0.0 && !(a >= 0x1p-74 && a <= 0x1p30)) in_range = false;
                hi = float(v);
                lo = float(v - double(hi));
            };
            std::vector<float> h_D2(30 * T), h_S2(18 * T), h_SR2(ext ? 18 * T : 0), h_SB2(ext ? 6 * T : 0);
            for (int64_t i = 0; i < T; ++i) {
                for (int q = 0; q < 15; ++q) pair(h_D[q * T + i], h_D2[q * T + i], h_D2[(15 + q) * T + i]);
                for (int s = 0; s < 3; ++s) {
                    const double sa = h_nb[s * T + i] >= 0 ? -h_alpha[s * T + i] : 0.0;
                    const double o[3] = {sa, sa * h_ex[s * T + i], sa * h_ey[s * T + i]};
                    for (int q = 0; q < 3; ++q)
                        pair(o[q], h_S2[(3 * s + q) * T + i], h_S2[(9 + 3 * s + q) * T + i]);
                    if (ext) {
                        const double sr = h_nb[s * T + i] >= 0 ? -h_alr[s * T + i] : 0.0;
                        const double r[3] = {sr, sr * h_exr[s * T + i], sr * h_eyr[s * T + i]};
                        for (int q = 0; q < 3; ++q)
                            pair(r[q], h_SR2[(3 * s + q) * T + i], h_SR2[(9 + 3 * s + q) * T + i]);
                        pair(h_nb[s * T + i] >= 0 ? -h_bdg[s * T + i] : 0.0, h_SB2[s * T + i], h_SB2[(3 + s) * T + i]);
                    }
                }
            }
            if (in_range) {
                UP(D2, h_D2); UP(S2, h_S2);
                if (ext) {
                    UP(SR2, h_SR2); UP(SB2, h_SB2);
                }
                // pairs of the right-hand-side weights for the double-FP32 right-hand side
                // (0 or 2^-50 <= |a0| <= 2^50: the low parts stay normal FP32 and the
                // scaled squares of the norm stay below 2^128)
                bool a0_range = true;
                std::vector<float> h_a0p(30 * T);
                for (int64_t q = 0; q < 15 * T; ++q) {
                    const double v = h_a0[q], a = std::fabs(v);
                    if (v != 0.0 && !(a >= 0x1p-50 && a <= 0x1p50)) a0_range = false;
                    h_a0p[q] = float(v);
                    h_a0p[15 * T + q] = float(v - double(h_a0p[q]));
                }
                if (a0_range) UP(a0p, h_a0p);
            }
        }
    }
#undef UP

    // ---- work buffers
    Work &k = m->wk;
    k.m = cfg.gmres_m;
    k.m_alloc = cfg.gmres_m;
    k.nblk = (int)nblk;
    k.ns = 4 * n_cases;
    const int mm = k.m;
    const int64_t ns = k.ns;
#define AL(ptr, n) \
    if ((st = dalloc(m, &k.ptr, (size_t)(n))) != GKS_OK) return st
    AL(w, 4 * T); AL(w_old, 4 * T); AL(x, 20 * T); AL(b, 20 * T); AL(r, 20 * T); AL(t2, 20 * T); AL(t3, 20 * T);
    if (cfg.basis_fp32) {
        AL(V32, (size_t)(mm + 1) * 20 * T);
    } else {
        AL(V, (size_t)(mm + 1) * 20 * T);
    }
    AL(flux, 4 * F);
    if (cfg.precision == GKS_MIXED) {
        AL(t2_32, 20 * T); AL(t3_32, 20 * T); AL(r32, 20 * T); AL(Z32, (size_t)mm * 20 * T);
    } else {
        AL(Z, (size_t)mm * 20 * T);
    }
    AL(part, (size_t)nblk * 4 * (mm + 2)); AL(dpart, (size_t)nblk * 4);
    if (cfg.limiter) {
        AL(xl, 20 * T); AL(lflag, T);
    }
    AL(x_prev, 20 * T); AL(x_prev2, 20 * T);   // extrapolated warm start (also for the autotuner)
    if (cfg.precision == GKS_MIXED) {
        AL(x2, 40 * T);
        k.x32 = k.x2;
        AL(w2, 8 * T);
        AL(y32, ns * mm);
    }
    AL(H, ns * (mm + 1) * mm); AL(cs, ns * mm); AL(sn, ns * mm); AL(g, ns * (mm + 1)); AL(y, ns * mm);
    AL(hcol, ns * (mm + 2)); AL(hco, ns * (mm + 2)); AL(vn, ns * (mm + 1)); AL(bnorm, ns); AL(beta, ns); AL(ctl, kCtlFields * ns); AL(flags, 4);
    AL(sexp, 2 * ns);
    AL(dt, n_cases); AL(tcase, n_cases); AL(tfinal, n_cases); AL(done, n_cases); AL(scal, 8); AL(status, n_cases);
    AL(nstep, n_cases); AL(last_dt, n_cases); AL(iters_acc, ns); AL(nsolve, 1); AL(run_ctl, 4);
    AL(sf_ctl, 4);
    GKS_CUDA(cudaDeviceGetAttribute(&k.sm_count, cudaDevAttrMultiProcessorCount, m->device));
    if (cfg.precond == GKS_PC_ILU_EXACT) AL(sf_flag, T);
#undef AL
    GKS_CUDA(cudaMemset(k.sf_ctl, 0, sizeof(int32_t) * 4));
    if (k.sf_flag) GKS_CUDA(cudaMemset(k.sf_flag, 0, sizeof(int32_t) * T));
    GKS_CUDA(cudaMemset(k.nsolve, 0, sizeof(int64_t)));
    GKS_CUDA(cudaMemset(k.run_ctl, 0, sizeof(int64_t) * 4));
    GKS_CUDA(cudaMemset(k.x, 0, sizeof(double) * 20 * T));
    GKS_CUDA(cudaMemset(k.bnorm, 0, sizeof(double) * ns));
    GKS_CUDA(cudaMemset(k.ctl, 0, sizeof(int32_t) * kCtlFields * ns));
    GKS_CUDA(cudaMemset(k.sexp, 0, sizeof(int32_t) * 2 * ns));
    GKS_CUDA(cudaMemset(k.status, 0, sizeof(int32_t) * n_cases));
    GKS_CUDA(cudaMemset(k.done, 0, sizeof(int32_t) * n_cases));
    {
        // padding cells hold a harmless uniform state
        std::vector<double> w0(4 * T, 0.0);
        for (int64_t i = 0; i < T; ++i) {
            w0[i] = 1.0;
            w0[3 * T + i] = 2.5;
        }
        GKS_CUDA(cudaMemcpy(k.w, w0.data(), sizeof(double) * 4 * T, cudaMemcpyHostToDevice));
    }
    GKS_CUDA(cudaMallocHost(&k.h_flags, sizeof(int32_t) * 4));
    GKS_CUDA(cudaMallocHost(&k.h_scal, sizeof(double) * 8));
    GKS_CUDA(cudaMallocHost(&k.h_step, sizeof(double) * 9));
    GKS_CUDA(cudaMallocHost(&k.h_stepi, sizeof(int32_t) * 5));
    return GKS_OK;
}

void free_mesh(gks_mesh *m)
{
    if (m->graphs) {
        destroy_graph_execs(m->graphs);
        if (m->graphs->cap) cudaStreamDestroy(m->graphs->cap);
        if (m->graphs->ctr) cudaFree(m->graphs->ctr);
        if (m->graphs->h_ctr) cudaFreeHost(m->graphs->h_ctr);
        if (m->graphs->h_run) cudaFreeHost(m->graphs->h_run);
        delete m->graphs;
        m->graphs = nullptr;
    }
    for (void *p : m->allocations) cudaFree(p);
    m->allocations.clear();
    if (m->wk.h_flags) cudaFreeHost(m->wk.h_flags);
    if (m->wk.h_scal) cudaFreeHost(m->wk.h_scal);
    if (m->wk.h_step) cudaFreeHost(m->wk.h_step);
    if (m->wk.h_stepi) cudaFreeHost(m->wk.h_stepi);
    m->wk.h_flags = nullptr;
    m->wk.h_scal = nullptr;
    m->wk.h_step = nullptr;
    m->wk.h_stepi = nullptr;
}

}  // namespace gks
