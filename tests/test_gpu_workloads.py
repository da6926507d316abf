"""The benchmark's workloads run end to end on the GPU: the run control's
steady-residual stop on the viscous cavity against the same rule applied to
the oracle's steps, the third-order convergence sweep of the advected density
wave (Sec. IV.A) on 40^2..320^2 meshes, the mixed path over 100 steps of the
800-triangle wave against the oracle, and one FP64 step of the
1,000,000-triangle shock-vortex workload against one oracle step."""
import math

import numpy as np
import pytest

from paper_1802_00704_gb300 import inputs as I
from tests.gpu_util import dev, host, needs_gpu, torch

pytestmark = [pytest.mark.gpu, needs_gpu]


@pytest.fixture(scope="module")
def O():
    from oracle import oracle
    oracle.build()
    return oracle


@pytest.fixture(scope="module")
def G():
    from paper_1802_00704_gb300 import build, gks
    build.build()
    return gks


def _steady_res(w_new, w_old, area, dt):
    """The run control's steady residual of one step: the largest over the
    four variables of sqrt(sum |Omega| (w^{n+1} - w^n)^2) / dt."""
    return max(math.sqrt(np.sum(area * (w_new[v] - w_old[v]) ** 2)) / dt for v in range(4))


@pytest.mark.parametrize("precision", ["fp64", "mixed"])
def test_run_stops_at_the_oracle_steady_residual(O, G, precision):
    """gks_run(steady_tol) on a 12 x 12 cavity (isothermal no-slip walls,
    Re 1000, Pr 0.72) stops at the first step whose residual, relative to the
    first step's, is below the tolerance; the same rule written here around the
    oracle's steps picks the same step, and the reported residual matches."""
    c = I.cavity_case(12)
    om = O.OracleMesh(c.mesh, mu=c.mu, prandtl=0.72)
    area = om.cell_geometry()["area"]
    w = c.w0.copy()
    rel, r0 = [], None
    for _ in range(300):
        w_old = w.copy()
        info = om.step(w)
        assert info.status == 0
        r = _steady_res(w, w_old, area, info.dt)
        r0 = r if r0 is None else r0
        rel.append(r / r0)
    rel = np.array(rel)
    # a tolerance the residual crosses for the first time at step n (1-based):
    # the last new minimum (by 0.5 %) of the relative residual over these steps
    # (acoustic waves make it oscillate on its way down; measured: step 120)
    n = None
    for q in range(20, 300):
        if rel[q] < 0.995 * rel[:q].min():
            n = q + 1
            tol = math.sqrt(rel[q] * rel[:q].min())
    assert n is not None and n > 50, rel
    kw = dict(precision=G.MIXED, basis_fp32=1) if precision == "mixed" else {}
    m = G.GksMesh(c.mesh, mu=c.mu, prandtl=0.72, **kw)
    wg = dev(c.w0)
    info = m.run(wg, max_steps=1000, steady_tol=tol)
    assert info["status"] == 0
    assert info["steps"] == n, (info["steps"], n)
    assert abs(info["steady_res"] / rel[n - 1] - 1.0) <= 1e-5, (info["steady_res"], rel[n - 1])


def _advect_gpu(G, n, tf, **kw):
    c = I.advection_case(n)
    m = G.GksMesh(c.mesh, **kw)
    w = dev(c.w0)
    info = m.run(w, t_final=tf, max_steps=10 ** 6)
    assert info["status"] == 0 and abs(info["t"] - tf) <= 1e-12
    ex = I.advection_exact_density(c, tf)
    p = c.mesh.nodes[c.mesh.tris]
    area = 0.5 * np.abs((p[:, 1, 0] - p[:, 0, 0]) * (p[:, 2, 1] - p[:, 0, 1]) -
                        (p[:, 2, 0] - p[:, 0, 0]) * (p[:, 1, 1] - p[:, 0, 1]))
    rho = host(w)[0]
    l1 = np.sum(area * np.abs(rho - ex)) / area.sum()
    l2 = math.sqrt(np.sum(area * (rho - ex) ** 2) / area.sum())
    return l1, l2


@pytest.mark.parametrize("precision", ["fp64", "mixed"])
def test_advection_order_sweep(G, precision):
    """The density wave to t = 0.1 on jittered 40^2, 80^2, 160^2 and 320^2
    meshes (121 to 1,372 steps): L1 and L2 errors against the exact cell
    averages fall at order >= 2.7 at every refinement (the paper's designed
    third order, Sec. IV.A; measured 2.95, 2.93, 2.82 in L1 on both paths).
    Over longer times the order falls at the finest meshes (t = 2: 2.58, 2.21,
    1.28): an error term linear in h grows with time there, as the inviscid
    collision time tau = 0.01 dt of Eq. (39), which scales with h, would make."""
    kw = dict(precision=G.MIXED, basis_fp32=1) if precision == "mixed" else {}
    e = [_advect_gpu(G, n, 0.1, **kw) for n in (40, 80, 160, 320)]
    for a, b in zip(e, e[1:]):
        o1, o2 = math.log2(a[0] / b[0]), math.log2(a[1] / b[1])
        assert o1 >= 2.7 and o2 >= 2.7, (e, o1, o2)


def test_order_over_a_full_period_without_the_inviscid_collision_time(G):
    """Over a full period (t = 2) the inviscid collision time tau = 0.01 dt of
    Eq. (39) adds a numerical viscosity that scales with h, and the measured
    order falls at fine meshes (2.58, 2.21, 1.28 from 40^2 to 320^2).  With the
    viscous form tau = mu / p (Eq. (40)) and mu = 1e-12 that term is gone and
    the scheme is third order over the whole period (measured 3.01, 2.98, 3.00):
    the loss is the collision time's, not the reconstruction's or the flux's."""
    e = [_advect_gpu(G, n, 2.0, precision=G.MIXED, basis_fp32=1, mu=1e-12)[0] for n in (40, 80, 160)]
    orders = [math.log2(a / b) for a, b in zip(e, e[1:])]
    assert min(orders) >= 2.8, (e, orders)
    inviscid = [_advect_gpu(G, n, 2.0, precision=G.MIXED, basis_fp32=1)[0] for n in (80, 160)]
    assert math.log2(inviscid[0] / inviscid[1]) < 2.5 and inviscid[1] > 2.0 * e[2], (inviscid, e)


@pytest.mark.parametrize("basis_fp32", [0, 1])
def test_mixed_100_steps_against_oracle(O, G, basis_fp32):
    """Config 1 (800 triangles) for 100 steps on the mixed path: relative L1
    within 1e-8 of the FP64 oracle on every conserved variable, and the
    relative max per cell within 1e-7."""
    c = I.advection_case(20)
    om = O.OracleMesh(c.mesh)
    area = om.cell_geometry()["area"]
    wo = c.w0.copy()
    m = G.GksMesh(c.mesh, precision=G.MIXED, basis_fp32=basis_fp32)
    w = dev(c.w0)
    for _ in range(100):
        dt = om.cfl_dt(wo)
        assert om.step(wo, dt).status == 0
        assert m.step(w, dt)["status"] == 0
    got = host(w)
    l1 = np.sum(area * np.abs(got - wo), axis=1) / np.sum(area * np.abs(wo), axis=1)
    mx = np.max(np.abs(got - wo), axis=1) / np.max(np.abs(wo), axis=1)
    assert np.all(l1 <= 1e-8) and np.all(mx <= 1e-7), (l1, mx)


def test_fullsize_fp64_step_against_oracle(O, G):
    """One FP64 step of the 1,000,000-triangle shock-vortex workload (the
    benchmark's mesh) against one oracle step from the same state: every cell
    within 1e-10 relative of the largest value of its variable."""
    c = I.shock_vortex_case(1000, 500)
    om = O.OracleMesh(c.mesh)
    wo = c.w0.copy()
    dt = om.cfl_dt(wo)
    assert om.step(wo, dt).status == 0
    m = G.GksMesh(c.mesh)
    w = dev(c.w0)
    assert m.step(w, dt)["status"] == 0
    got = host(w)
    err = np.max(np.abs(got - wo), axis=1) / np.max(np.abs(wo), axis=1)
    assert np.all(err <= 1e-10), err


def test_fp64_flux_option_is_the_fp64_point_flux(G):
    """flux_lead = 2: the mixed solver with the FP64 path's flux kernel; the
    point flux equals the FP64 path's bit for bit (viscous, Prandtl 0.72)."""
    rng = np.random.default_rng(5)
    n = 2000
    w = np.zeros((2, n, 6, 4))
    for s in range(2):
        rho = rng.uniform(0.5, 2.0, n)
        U, V, p = rng.uniform(-1, 1, n), rng.uniform(-1, 1, n), rng.uniform(0.5, 2.0, n)
        w[s, :, 0] = np.stack([rho, rho * U, rho * V, p / 0.4 + 0.5 * rho * (U * U + V * V)], axis=1)
        w[s, :, 1:] = rng.normal(0.0, 0.05, (n, 5, 4))
    kw = dict(mu=2e-3, prandtl=0.72)
    a = host(G.point_flux(dev(w[0]), dev(w[1]), 0.004, precision=G.MIXED, flux_lead=2, **kw))
    b = host(G.point_flux(dev(w[0]), dev(w[1]), 0.004, precision=G.FP64, **kw))
    assert np.array_equal(a, b)


def test_viscous_cavity_mixed_solver_with_fp64_flux(G):
    """The lid-driven cavity (Re 1000, Pr 0.72, isothermal no-slip walls) for 60
    steps: with the FP64 flux (flux_lead = 2) the mixed path differs from the FP64
    path only by the CLS solve's tolerance, within 1e-10 relative L1 on every
    conserved variable; the default double-FP32 lead with FP32 slope terms moves
    the momenta further (their viscous stress is carried in FP32)."""
    c = I.cavity_case(24)
    p = c.mesh.nodes[c.mesh.tris]
    area = 0.5 * np.abs((p[:, 1, 0] - p[:, 0, 0]) * (p[:, 2, 1] - p[:, 0, 1]) -
                        (p[:, 2, 0] - p[:, 0, 0]) * (p[:, 1, 1] - p[:, 0, 1]))
    out = {}
    for name, kw in (("fp64", {}), ("fp64_flux", dict(precision=G.MIXED, flux_lead=2)),
                     ("pairs", dict(precision=G.MIXED, flux_lead=1))):
        m = G.GksMesh(c.mesh, mu=c.mu, prandtl=0.72, **kw)
        w = dev(c.w0)
        assert m.run(w, max_steps=60)["status"] == 0
        out[name] = host(w)
    ref = out["fp64"]
    l1 = {k: np.sum(area * np.abs(out[k] - ref), axis=1) / np.sum(area * np.abs(ref), axis=1)
          for k in ("fp64_flux", "pairs")}
    assert np.all(l1["fp64_flux"] <= 1e-10), l1
    assert l1["pairs"][1:3].max() > l1["fp64_flux"][1:3].max(), l1
