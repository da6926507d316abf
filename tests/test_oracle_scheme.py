"""Pins of the oracle's full step (Eq. (6)): free-stream preservation,
conservation on periodic meshes, third-order convergence on the advected
density wave (Eqs. (41)-(42), restated diagonally), and invariance under
rotation and translation of the whole problem."""
import math

import numpy as np
import pytest

from paper_1802_00704_gb300 import inputs as I


def _uniform(T, rho, u, v, p, gamma=1.4):
    return np.ascontiguousarray(np.stack([np.full(T, rho), np.full(T, rho * u), np.full(T, rho * v),
                                          np.full(T, p / (gamma - 1) + 0.5 * rho * (u * u + v * v))]))


def test_free_stream_preserved(oracle_mod):
    c = I.advection_case(8, seed=7)
    om = oracle_mod.OracleMesh(c.mesh)
    w = _uniform(om.T, 1.3, 0.9, -0.6, 0.7)
    w0 = w.copy()
    for _ in range(3):
        info = om.step(w)
        assert info.status == 0
    assert np.abs(w - w0).max() < 1e-13 * np.abs(w0).max()


def test_free_stream_with_dirichlet_boundaries(oracle_mod):
    st = I.prim_to_cons(np.float64(1.3), np.float64(0.9), np.float64(-0.6), np.float64(0.7), 1.4)
    bc = {s: (I.TAG_DIRICHLET, st) for s in ("left", "right", "bottom", "top")}
    m = I.split_quad_mesh(6, 5, 1.0, 0.8, seed=2, bc=bc)
    om = oracle_mod.OracleMesh(m)
    w = _uniform(om.T, 1.3, 0.9, -0.6, 0.7)
    w0 = w.copy()
    om.step(w)
    assert np.abs(w - w0).max() < 1e-13 * np.abs(w0).max()


def test_conservation_periodic(oracle_mod):
    c = I.advection_case(12, k=2, amp=0.2)
    om = oracle_mod.OracleMesh(c.mesh)
    area = om.cell_geometry()["area"]
    w = c.w0.copy()
    tot0 = (w * area).sum(axis=1)
    for _ in range(10):
        assert om.step(w).status == 0
    tot = (w * area).sum(axis=1)
    assert np.all(np.abs(tot - tot0) <= 1e-13 * np.abs(tot0).max())


def _advect(oracle_mod, n, tf):
    c = I.advection_case(n)
    om = oracle_mod.OracleMesh(c.mesh)
    w = c.w0.copy()
    t = 0.0
    while t < tf - 1e-14:
        dt = min(om.cfl_dt(w), tf - t)
        assert om.step(w, dt).status == 0
        t += dt
    ex = I.advection_exact_density(c, tf)
    area = om.cell_geometry()["area"]
    l1 = np.sum(area * np.abs(w[0] - ex)) / area.sum()
    l2 = math.sqrt(np.sum(area * (w[0] - ex) ** 2) / area.sum())
    return l1, l2


def test_advection_third_order(oracle_mod):
    """L1 and L2 density errors at t = 0.1 on 20^2, 40^2 and 80^2 jittered
    meshes; the paper states that the designed (third) order is reached
    (Sec. IV.A).  Both refinements must show it: one ratio alone cannot tell an
    order-3 scheme from a lucky pre-asymptotic ratio (measured: 2.83 and 2.95
    in L1)."""
    e = [_advect(oracle_mod, n, 0.1) for n in (20, 40, 80)]
    for a, b in zip(e, e[1:]):
        o1 = math.log(a[0] / b[0], 2)
        o2 = math.log(a[1] / b[1], 2)
        assert o1 > 2.7 and o2 > 2.7, (e, o1, o2)


def _rotated_mesh(mesh, th, shift=(0.0, 0.0)):
    R = np.array([[math.cos(th), -math.sin(th)], [math.sin(th), math.cos(th)]])
    m2 = I.Mesh(nodes=mesh.nodes @ R.T + np.array(shift), tris=mesh.tris, faces=mesh.faces,
                face_shift=mesh.face_shift @ R.T, bc_state=mesh.bc_state)
    return m2, R


def test_rotation_and_translation_invariance(oracle_mod):
    c = I.advection_case(8, k=1, amp=0.2)
    w = c.w0.copy()
    w[2] *= 0.3                                    # break the u = v symmetry
    w[3] = 2.5 + 0.5 * (w[1] ** 2 + w[2] ** 2) / w[0]
    om = oracle_mod.OracleMesh(c.mesh)
    dt = 0.8 * om.cfl_dt(w)
    wa = w.copy()
    om.step(wa, dt)
    th = 0.7321
    m2, R = _rotated_mesh(c.mesh, th, shift=(3.1, -1.7))
    om2 = oracle_mod.OracleMesh(m2)
    wb = w.copy()
    wb[1:3] = R @ w[1:3]
    om2.step(wb, dt)
    wa_rot = wa.copy()
    wa_rot[1:3] = R @ wa[1:3]
    scale = np.abs(wa).max(axis=1, keepdims=True)
    assert np.all(np.abs(wb - wa_rot) <= 1e-12 * scale)


def test_weak_riemann_strip_runs_with_boundaries(oracle_mod):
    c = I.riemann_strip_case(40, 4, left=(1.1, 0.0, 0.0, 1.1), right=(1.0, 0.0, 0.0, 1.0))
    om = oracle_mod.OracleMesh(c.mesh)
    w = c.w0.copy()
    for _ in range(5):
        info = om.step(w)
        assert info.status == 0
    assert np.all(w[0] > 0)
    # the boundary cells (Dirichlet faces) are reconstructed at k = 1, Eq. (28)
    k = om.cell_geometry()["k"]
    bcell = c.mesh.faces[c.mesh.faces[:, 3] < 0, 2]
    assert np.all(k[bcell] == 1) and (k == 2).sum() == om.T - len(np.unique(bcell))


def test_sod_without_limiter_reports_nonphysical_state(oracle_mod):
    """Unlimited quadratic reconstruction across the Sod jump (Eq. (44))
    undershoots to negative density at Gauss points; the step reports it
    instead of producing NaNs (the paper applies its limiter there)."""
    c = I.sod_case(40, 4)
    om = oracle_mod.OracleMesh(c.mesh)
    w = c.w0.copy()
    assert om.step(w).status == 1


def test_acoustic_pulse_third_vs_second_order(oracle_mod):
    """Acoustic pressure pulse (Sec. IV): the error against the exact linear
    acoustics solution (Hankel integral, checked at t = 0 below) is smaller for
    the third-order scheme and falls faster under refinement than for the
    second-order variant (k_i = 1 everywhere)."""
    import math
    from tests.acoustic_exact import pulse_pressure, pulse_pressure_cell_average
    eta = np.linspace(0.0, 0.4, 9)
    alpha = math.log(2.0) / 0.04 ** 2
    assert np.max(np.abs(pulse_pressure(eta, 0.0) - (1.0 + 0.01 * np.exp(-alpha * eta ** 2)))) < 1e-13
    tend = 0.05

    def err(n, second):
        c = I.acoustic_pulse_case(n)
        om = oracle_mod.OracleMesh(c.mesh, second_order=second)
        w, t = c.w0.copy(), 0.0
        while t < tend - 1e-14:
            dt = min(om.cfl_dt(w), tend - t)
            assert om.step(w, dt).status == 0
            t += dt
        area = om.cell_geometry()["area"]
        p = 0.4 * (w[3] - 0.5 * (w[1] ** 2 + w[2] ** 2) / w[0])
        ex = pulse_pressure_cell_average(c.mesh.nodes, c.mesh.tris, tend)
        return np.sum(area * np.abs(p - ex)) / area.sum()

    e3 = [err(n, 0) for n in (20, 40)]
    e2 = [err(n, 1) for n in (20, 40)]
    r3, r2 = math.log2(e3[0] / e3[1]), math.log2(e2[0] / e2[1])
    assert e3[1] < e2[1] and r3 > 2.1 and r3 > r2 + 0.4, (e3, e2, r3, r2)
