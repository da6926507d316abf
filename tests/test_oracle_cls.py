"""Pins of the oracle's geometry, CLS system (Sec. III.A) and linear solver
(Sec. III.B) against exact properties: closed cells, quadratic exactness,
zero coefficients for constant data, a dense direct solve, and the O(h^3)
reconstruction error of a quadratic reconstruction."""
import math

import numpy as np
import pytest

from paper_1802_00704_gb300 import inputs as I


def _walled(n, seed=11):
    st = np.array([1.0, 0.0, 0.0, 2.5])
    bc = {s: (I.TAG_DIRICHLET, st) for s in ("left", "right", "bottom", "top")}
    return I.split_quad_mesh(n, n, 1.0, 1.0, seed=seed, bc=bc)


def test_geometry_closed_cells(oracle_mod):
    c = I.advection_case(8)
    om = oracle_mod.OracleMesh(c.mesh)
    cg, fg = om.cell_geometry(), om.face_geometry()
    assert abs(cg["area"].sum() - 4.0) < 1e-13
    acc = np.zeros((om.T, 2))
    for f, (n0, n1, l, r, tag) in enumerate(c.mesh.faces):
        v = fg["len"][f] * np.array([fg["nx"][f], fg["ny"][f]])
        acc[l] += v
        acc[r] -= v
    assert np.abs(acc).max() < 1e-14
    # circumradius: equal distance from the circumcentre to the three vertices
    p = c.mesh.nodes[c.mesh.tris]
    for i in range(0, om.T, 17):
        a, b, q = p[i]
        d = 2 * (a[0] * (b[1] - q[1]) + b[0] * (q[1] - a[1]) + q[0] * (a[1] - b[1]))
        ux = ((a @ a) * (b[1] - q[1]) + (b @ b) * (q[1] - a[1]) + (q @ q) * (a[1] - b[1])) / d
        uy = ((a @ a) * (q[0] - b[0]) + (b @ b) * (a[0] - q[0]) + (q @ q) * (b[0] - a[0])) / d
        R = math.hypot(a[0] - ux, a[1] - uy)
        assert abs(cg["crad"][i] - R) < 1e-13
        assert abs(cg["h"][i] - max(R, math.sqrt(cg["area"][i]))) < 1e-13 * R


def _quad(x, y):
    return 0.7 + 0.3 * x - 0.2 * y + 0.45 * x * x - 0.35 * x * y + 0.25 * y * y


def _exact_coef(cg, T):
    coef = np.zeros((5, T))
    h, cx, cy = cg["h"], cg["cx"], cg["cy"]
    coef[0] = h * (0.3 + 0.9 * cx - 0.35 * cy)
    coef[1] = h * (-0.2 - 0.35 * cx + 0.5 * cy)
    coef[2] = h * h * 0.9
    coef[3] = h * h * (-0.35)
    coef[4] = h * h * 0.5
    return coef


@pytest.mark.parametrize("M", [1, 2])
@pytest.mark.parametrize("glob", [0, 1])
def test_cls_operator_exact_for_quadratics(oracle_mod, glob, M):
    """The exact coefficients of a global quadratic satisfy every equation of a
    cell that can hold it (k = 2); per cell that zeroes the rows of k = 2 cells,
    in the global system (cls_global, Eq. (33)) the rows of k = 2 cells whose
    neighbours are k = 2 too (their equations enter through B_ji).  With M = 2
    (second-derivative equations) a k = 1 neighbour cannot match the second
    derivatives either, so the same selection applies per cell."""
    m = _walled(8)
    om = oracle_mod.OracleMesh(m, cls_global=glob, cls_M=M)
    cg = om.cell_geometry()
    qbar = I.cell_average(m, lambda x, y: _quad(x, y)[None])[0]
    w = np.stack([qbar, qbar, qbar, qbar + 3.0])
    rp, col, val, off = om.cls_matrix()
    rhs = om.cls_rhs(w)[0]
    ex = _exact_coef(cg, om.T)
    x = np.zeros(om.ndof)
    k = cg["k"].astype(int)
    for i in range(om.T):
        n = 5 if k[i] == 2 else 2
        x[off[i]:off[i] + n] = ex[:n, i]
    Kx = np.array([val[rp[r]:rp[r + 1]] @ x[col[rp[r]:rp[r + 1]]] for r in range(om.ndof)])
    res = Kx - rhs
    nbrs = [set() for _ in range(om.T)]
    for (_, _, l, r, _) in m.faces:
        if r >= 0:
            nbrs[l].add(r)
            nbrs[r].add(l)
    keep = [i for i in range(om.T) if k[i] == 2 and (not (glob or M == 2) or all(k[j] == 2 for j in nbrs[i]))]
    interior_rows = np.concatenate([np.arange(off[i], off[i] + 5) for i in keep])
    assert len(interior_rows) > 0
    assert np.abs(res[interior_rows]).max() < 1e-13
    boundary_rows = np.setdiff1d(np.arange(om.ndof), interior_rows)
    assert np.abs(res[boundary_rows]).max() > 1e-6        # k = 1 cells cannot hold a quadratic


@pytest.mark.parametrize("glob", [0, 1])
def test_constant_data_gives_zero_coefficients(oracle_mod, glob):
    c = I.advection_case(6)
    om = oracle_mod.OracleMesh(c.mesh, cls_global=glob)
    w = np.ones((4, om.T)) * np.array([[1.2], [0.3], [-0.1], [3.0]])
    coef, it, rr, bad = om.cls_solve(w)
    assert bad == 0 and np.all(coef == 0.0)


@pytest.mark.parametrize("M", [1, 2])
@pytest.mark.parametrize("glob", [0, 1])
@pytest.mark.parametrize("kind", ["periodic4", "periodic8", "walled6"])
def test_gmres_matches_dense_lu(oracle_mod, kind, glob, M):
    if kind.startswith("periodic"):
        c = I.advection_case(int(kind[-1]), k=1, amp=0.3)
        m, w = c.mesh, c.w0
    else:
        m = _walled(6)
        w = I.cell_average(m, lambda x, y: np.stack([1 + 0.2 * np.sin(3 * x + y), np.cos(x - 2 * y),
                                                     0.1 * x * y, 2.5 + np.exp(0.3 * x)]))
    om = oracle_mod.OracleMesh(m, cls_global=glob, cls_M=M)
    coef, it, rr, bad = om.cls_solve(w)
    ref = om.cls_dense(w)
    assert bad == 0 and np.all(rr < 1e-13)
    assert np.abs(coef - ref).max() <= 1e-11 * np.abs(ref).max()


def test_rcm_is_a_permutation_and_narrows_bandwidth(oracle_mod):
    c = I.advection_case(16, seed=3)
    om = oracle_mod.OracleMesh(c.mesh)
    p = om.rcm_perm()
    assert np.array_equal(np.sort(p), np.arange(om.T))
    inv = np.empty_like(p)
    inv[p] = np.arange(om.T)
    f = c.mesh.faces
    nat = np.abs(f[:, 2] - f[:, 3]).max()
    rcm = np.abs(inv[f[:, 2]] - inv[f[:, 3]]).max()
    assert rcm < nat


def test_reconstruction_error_is_third_order(oracle_mod):
    """Pointwise error of the reconstructed polynomial at face Gauss points for
    smooth periodic data is O(h^3) (k = 2, Eq. (19))."""
    errs = []
    for n in (8, 16, 32):
        c = I.advection_case(n, k=1, amp=0.2)
        om = oracle_mod.OracleMesh(c.mesh)
        coef, it, rr, bad = om.cls_solve(c.w0)
        fg = om.face_geometry()
        e = 0.0
        for f in range(0, om.F, max(1, om.F // 200)):
            l = c.mesh.faces[f, 2]
            for g in range(2):
                x, y = fg["gauss"][f, g]
                val = om.eval_cell(c.w0, coef, l, x, y)[0, 0]
                e = max(e, abs(val - (1 + 0.2 * math.sin(math.pi * (x + y)))))
        errs.append(e)
    assert errs[0] / errs[1] > 6 and errs[1] / errs[2] > 6, errs


def _dense(om):
    rp, col, val, off = om.cls_matrix()
    K = np.zeros((om.ndof, om.ndof))
    for r in range(om.ndof):
        K[r, col[rp[r]:rp[r + 1]]] = val[rp[r]:rp[r + 1]]
    return K


@pytest.mark.parametrize("M", [1, 2])
@pytest.mark.parametrize("kind", ["walled6", "periodic5"])
def test_global_cls_is_symmetric_positive_definite(oracle_mod, kind, M):
    """cls_global: the normal equations of all equations together are C^T C,
    symmetric and positive definite (Eq. (33)); the default per-cell equations
    are not symmetric.  Both have the same sparsity (face neighbours)."""
    m = _walled(6) if kind == "walled6" else I.advection_case(5, seed=4).mesh
    Kg = _dense(oracle_mod.OracleMesh(m, cls_global=1, cls_M=M))
    Kp = _dense(oracle_mod.OracleMesh(m, cls_M=M))
    scale = np.abs(Kg).max()
    assert np.abs(Kg - Kg.T).max() <= 1e-14 * scale
    assert np.linalg.eigvalsh(0.5 * (Kg + Kg.T)).min() > 1e-10 * scale
    assert np.abs(Kp - Kp.T).max() > 1e-3 * np.abs(Kp).max()
    assert np.array_equal(Kg != 0, (Kg != 0) | (Kp != 0)) or np.array_equal(Kg != 0, Kp != 0)


def test_value_equations_only_for_the_linear_variant(oracle_mod):
    """cls_M = 0 with k_i = 1 everywhere (second-order variant): only the value
    equations, so each cell's gradient is its own least-squares fit to the
    neighbours' averages, uncoupled (no off-diagonal blocks), and exact for a
    linear field in every cell.  Every cell needs two neighbours (a y-periodic
    strip; a corner triangle with one neighbour would leave its gradient
    undetermined).  Without the linear variant the value equations cannot
    determine the five quadratic coefficients, which is refused."""
    c = I.riemann_strip_case(12, 4, left=(1.0, 0.0, 0.0, 1.0), right=(1.0, 0.0, 0.0, 1.0))
    m = c.mesh
    om = oracle_mod.OracleMesh(m, cls_M=0, second_order=1)
    K = _dense(om)
    rp, col, val, off = om.cls_matrix()
    tol = 1e-13 * np.abs(K).max()        # the zero-mean basis' means vanish up to rounding
    for i in range(om.T):
        blk = K[off[i]:off[i] + 2]
        assert np.abs(blk[:, :off[i]]).max(initial=0.0) <= tol and np.abs(blk[:, off[i] + 2:]).max(initial=0.0) <= tol
    cg = om.cell_geometry()
    qbar = I.cell_average(m, lambda x, y: (0.4 + 0.8 * x + 0.0 * y)[None])[0]
    w = np.stack([qbar, qbar, qbar, qbar + 3.0])
    coef, it, rr, bad = om.cls_solve(w)
    assert bad == 0
    assert np.allclose(coef[0, 0], 0.8 * cg["h"], rtol=1e-10, atol=1e-13)
    assert np.allclose(coef[0, 1], 0.0, atol=1e-12)
    with pytest.raises(Exception):
        oracle_mod.OracleMesh(m, cls_M=0)
