"""Pins of the oracle's shock detector and DWBAP limiter (Sec. III.C): smooth
data are not flagged and keep their coefficients; the limited scheme runs the
Sod problem (Eq. (44)) to t = 0.2 with positive states, and its distance to the
exact Riemann solution (Rankine-Hugoniot and isentropic relations, solved by
Newton iteration on the star pressure) shrinks under mesh refinement."""
import os

import numpy as np

from paper_1802_00704_gb300 import inputs as I
from tests.exact_riemann import exact_riemann


def test_exact_riemann_solver_star_state():
    # Sod star region against the tabulated five-digit values (tests/golden)
    gold = os.path.join(os.path.dirname(__file__), "golden", "sod_star_state.txt")
    ref = dict((k, float(v)) for k, v in (l.split() for l in open(gold) if l.strip() and not l.startswith("#")))
    us = ref["u_star"]
    x = np.array([0.5 + us * 0.2 - 1e-4, 0.5 + us * 0.2 + 1e-4])
    r, u, p = exact_riemann(x, 0.2, (1.0, 0.0, 1.0), (0.125, 0.0, 0.1))
    assert np.all(np.abs(p - ref["p_star"]) < 1e-5) and np.all(np.abs(u - us) < 1e-5)
    assert abs(r[0] - ref["rho_star_left"]) < 1e-5 and abs(r[1] - ref["rho_star_right"]) < 1e-5


def test_smooth_data_not_limited(oracle_mod):
    c = I.advection_case(16)
    om = oracle_mod.OracleMesh(c.mesh, limiter=1)
    coef, _, _, _ = om.cls_solve(c.w0)
    lim, flag = om.limit(c.w0, coef)
    assert np.all(flag == 0) and np.array_equal(lim, coef)


def _sod_l1(oracle_mod, nx, ny):
    c = I.sod_case(nx, ny)
    om = oracle_mod.OracleMesh(c.mesh, limiter=1)
    w = c.w0.copy()
    t = 0.0
    while t < 0.2 - 1e-14:
        dt = min(om.cfl_dt(w), 0.2 - t)
        info = om.step(w, dt)
        assert info.status == 0
        t += dt
    cg = om.cell_geometry()
    ex = exact_riemann(cg["cx"], 0.2, (1.0, 0.0, 1.0), (0.125, 0.0, 0.1))
    p = 0.4 * (w[3] - 0.5 * (w[1] ** 2 + w[2] ** 2) / w[0])
    assert np.all(w[0] > 0) and np.all(p > 0)
    area = cg["area"]
    return np.sum(area * np.abs(w[0] - ex[0])) / area.sum()


def test_limited_sod_converges_to_exact_riemann(oracle_mod):
    e1 = _sod_l1(oracle_mod, 40, 3)
    e2 = _sod_l1(oracle_mod, 80, 6)
    assert e2 < e1 / 1.4 and e2 < 0.01, (e1, e2)


def test_limiter_flags_only_near_the_jump(oracle_mod):
    c = I.sod_case(100, 4)
    om = oracle_mod.OracleMesh(c.mesh, limiter=1)
    coef, _, _, _ = om.cls_solve(c.w0)
    lim, flag = om.limit(c.w0, coef)
    cx = om.cell_geometry()["cx"]
    assert flag.sum() > 0
    assert np.all(np.abs(cx[flag > 0] - 0.5) < 0.05)
    assert np.array_equal(lim[:, :, flag == 0], coef[:, :, flag == 0])


def test_robust_mode_keeps_strong_contacts_positive(oracle_mod):
    # density ratio 10 at pressure ratio 2 (the strong end of the batched Riemann
    # strips): the plain DWBAP lets a cell average go negative within a few steps,
    # the robust mode (first order in the flagged cells) keeps every state physical
    left, right = (10.0, 0.0, 0.0, 2.0), (1.0, 0.0, 0.0, 1.0)

    def run(mode, steps=40):
        c = I.riemann_strip_case(60, 4, left=left, right=right, seed=5)
        om = oracle_mod.OracleMesh(c.mesh, limiter=mode)
        w = c.w0.copy()
        for n in range(steps):
            if om.step(w).status != 0:
                return n
            p = 0.4 * (w[3] - 0.5 * (w[1] ** 2 + w[2] ** 2) / w[0])
            if not (np.all(w[0] > 0) and np.all(p > 0)):
                return n
        return steps

    assert run(2) == 40
    assert run(1) < 40


def test_robust_mode_converges_to_exact_riemann(oracle_mod):
    def l1(nx, ny):
        c = I.riemann_strip_case(nx, ny, left=(10.0, 0.0, 0.0, 2.0), right=(1.0, 0.0, 0.0, 1.0), seed=9)
        om = oracle_mod.OracleMesh(c.mesh, limiter=2)
        w, t = c.w0.copy(), 0.0
        while t < 0.1 - 1e-14:
            dt = min(om.cfl_dt(w), 0.1 - t)
            assert om.step(w, dt).status == 0
            t += dt
        cg = om.cell_geometry()
        ex = exact_riemann(cg["cx"], 0.1, (10.0, 0.0, 2.0), (1.0, 0.0, 1.0))
        return np.sum(cg["area"] * np.abs(w[0] - ex[0])) / cg["area"].sum()
    e1, e2 = l1(40, 3), l1(80, 6)
    assert e2 < e1 / 1.3, (e1, e2)


def test_char_basis_diagonalises_the_euler_jacobian(oracle_mod):
    """The eigenvectors used for characteristic limiting: L R = I and
    R diag(q_n - c, q_n, q_n, q_n + c) L equals the Jacobian of the Euler flux
    along n (central differences of the flux)."""
    g = 1.4
    W = np.array([1.3, 1.3 * 0.4, -1.3 * 0.7, 2.5 / 0.4 + 0.5 * 1.3 * (0.4 ** 2 + 0.7 ** 2)])

    def flux(W, nx, ny):
        rho, u, v = W[0], W[1] / W[0], W[2] / W[0]
        p = (g - 1) * (W[3] - 0.5 * rho * (u * u + v * v))
        qn = u * nx + v * ny
        return np.array([rho * qn, rho * u * qn + p * nx, rho * v * qn + p * ny, (W[3] + p) * qn])

    for nx, ny in [(1.0, 0.0), (0.0, 1.0), (0.6, 0.8)]:
        R, L = oracle_mod.char_basis(W, g, nx, ny)
        A = np.zeros((4, 4))
        for k in range(4):
            d = np.zeros(4)
            d[k] = 1e-6 * max(1.0, abs(W[k]))
            A[:, k] = (flux(W + d, nx, ny) - flux(W - d, nx, ny)) / (2 * d[k])
        rho, u, v = W[0], W[1] / W[0], W[2] / W[0]
        c = np.sqrt(g * (g - 1) * (W[3] - 0.5 * rho * (u * u + v * v)) / rho)
        qn = u * nx + v * ny
        assert np.max(np.abs(L @ R - np.eye(4))) < 1e-14
        assert np.max(np.abs(R @ np.diag([qn - c, qn, qn, qn + c]) @ L - A)) < 1e-8


def test_characteristic_limiting_on_sod(oracle_mod):
    """DWBAP in characteristic variables: smooth data untouched, and the Sod
    run stays physical and converges to the exact solution under refinement."""
    c = I.advection_case(16)
    om = oracle_mod.OracleMesh(c.mesh, limiter=1, limit_char=1)
    coef, _, _, _ = om.cls_solve(c.w0)
    lim, flag = om.limit(c.w0, coef)
    assert np.all(flag == 0) and np.array_equal(lim, coef)

    def l1(nx, ny):
        c = I.sod_case(nx, ny)
        om = oracle_mod.OracleMesh(c.mesh, limiter=1, limit_char=1)
        w, t = c.w0.copy(), 0.0
        while t < 0.2 - 1e-14:
            dt = min(om.cfl_dt(w), 0.2 - t)
            assert om.step(w, dt).status == 0
            t += dt
        p = 0.4 * (w[3] - 0.5 * (w[1] ** 2 + w[2] ** 2) / w[0])
        assert np.all(w[0] > 0) and np.all(p > 0)
        cg = om.cell_geometry()
        ex = exact_riemann(cg["cx"], 0.2, (1.0, 0.0, 1.0), (0.125, 0.0, 0.1))
        return np.sum(cg["area"] * np.abs(w[0] - ex[0])) / cg["area"].sum()

    e1, e2 = l1(40, 3), l1(80, 6)
    assert e2 < e1 / 1.4 and e2 < 0.01, (e1, e2)
