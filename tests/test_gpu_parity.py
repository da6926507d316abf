"""Parity of the CUDA path (through the C ABI) with the CPU oracle, element by
element, on seeded inputs that span several thread blocks and a ragged tail.
Tolerances: FP64 path within 1e-10 relative max per variable after one step
and 1e-8 after 100 steps; kernel-level parity (point flux, face flux with the
same coefficients) within 1e-12; reconstruction coefficients within 1e-9
(both GMRES solves stop at relative residuals <= 1e-12, and the coefficient
error is the residual times the condition number of the CLS operator)."""
import numpy as np
import pytest

from paper_1802_00704_gb300 import inputs as I
from tests.gpu_util import dev, host, needs_gpu, rel_max, torch

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


def _walled(nx, ny, seed=11):
    st = I.prim_to_cons(np.float64(1.0), np.float64(0.2), np.float64(-0.1), np.float64(1.0), 1.4)
    bc = {s: (I.TAG_DIRICHLET, st) for s in ("left", "right", "bottom", "top")}
    m = I.split_quad_mesh(nx, ny, 1.0, 0.8, seed=seed, bc=bc)
    w = I.cell_average(m, lambda x, y: I.prim_to_cons(1 + 0.2 * np.sin(3 * x + y), 0.2 + 0.1 * np.cos(2 * y),
                                                      -0.1 + 0.05 * x, 1 + 0.1 * np.cos(x - y), 1.4))
    return I.Case("walled", m, w)


CASES = {
    "advection20": lambda: I.advection_case(20),
    "advection_k3_17": lambda: I.advection_case(17, k=3, amp=0.1, seed=9),
    "walled13x9": lambda: _walled(13, 9),
    "shock_vortex40x20": lambda: I.shock_vortex_case(40, 20),
    "weak_riemann60x4": lambda: I.riemann_strip_case(60, 4, left=(1.2, 0.0, 0.0, 1.3), right=(1.0, 0.0, 0.0, 1.0)),
}


# --------------------------------------------------------------------------- point flux

def _random_states(rng, n, jump=0.0):
    """Face-frame row blocks (n, 6, 4) of physical states with derivatives."""
    rho = 0.5 + rng.random(n)
    u = rng.uniform(-1.5, 1.5, n)
    v = rng.uniform(-1.0, 1.0, n)
    p = 0.3 + rng.random(n) * (1.0 + jump)
    w = np.zeros((n, 6, 4))
    w[:, 0] = np.stack([rho, rho * u, rho * v, p / 0.4 + 0.5 * rho * (u * u + v * v)], 1)
    w[:, 1:] = 0.2 * rng.standard_normal((n, 5, 4)) * w[:, :1]
    return w


@pytest.mark.parametrize("mu,tau2,jump,dt", [(0.0, 0, 0.0, 0.01), (0.0, 1, 2.0, 0.003), (1e-3, 0, 0.0, 0.002),
                                             (0.05, 0, 0.0, 0.002), (2e-5, 1, 0.5, 0.02)])
def test_point_flux_matches_oracle(O, G, mu, tau2, jump, dt):
    rng = np.random.default_rng(17)
    n = 300
    wl, wr = _random_states(rng, n, jump), _random_states(rng, n, jump)
    got = host(G.point_flux(dev(wl), dev(wr), dt, mu=mu, tau2_exact=tau2))
    ref = np.stack([O.point_flux(wl[q], wr[q], dt, mu=mu, tau2_exact=tau2)[0] for q in range(n)])
    scale = np.max(np.abs(ref), axis=0)
    assert np.all(np.max(np.abs(got - ref), axis=0) <= 1e-12 * scale), np.max(np.abs(got - ref), axis=0) / scale


@pytest.mark.parametrize("precision", ["fp64", "mixed"])
def test_prandtl_point_flux_matches_oracle(O, G, precision):
    """Prandtl-corrected energy flux (Pr = 0.72, viscous collision time) against
    the oracle, which takes the heat flux as the moment of (1/2)(u - U)|c|^2
    directly: 1e-12 of each flux scale in FP64, 1e-7 in mixed precision."""
    rng = np.random.default_rng(23)
    n = 200
    wl, wr = _random_states(rng, n, 0.3), _random_states(rng, n, 0.3)
    if precision == "mixed":
        for q in (wl, wr):
            q[:, 1:] *= 0.1
    dt, mu = 0.004, 2e-3
    got = host(G.point_flux(dev(wl), dev(wr), dt, mu=mu, prandtl=0.72,
                            precision=G.MIXED if precision == "mixed" else G.FP64))
    ref = np.stack([O.point_flux(wl[q], wr[q], dt, mu=mu, prandtl=0.72)[0] for q in range(n)])
    base = np.stack([O.point_flux(wl[q], wr[q], dt, mu=mu)[0] for q in range(n)])
    assert np.max(np.abs(ref[:, 3] - base[:, 3])) > 1e-6 * np.max(np.abs(ref[:, 3]))   # the correction acts
    scale = np.max(np.abs(ref), axis=0)
    tol = 1e-12 if precision == "fp64" else 1e-7
    assert np.all(np.max(np.abs(got - ref), axis=0) <= tol * scale), np.max(np.abs(got - ref), axis=0) / scale


# --------------------------------------------------------------------------- reconstruction and flux

@pytest.mark.parametrize("name", list(CASES))
@pytest.mark.parametrize("pc", ["exact", "sweep", "levels", "bjacobi"])
def test_cls_matches_oracle(O, G, name, pc):
    """Every preconditioner (the sync-free exact ILU solves, the sweeps, the
    exact solves launched level by level, the block-diagonal inverse) solves
    the same system to the same tolerance: the oracle's coefficients."""
    c = CASES[name]()
    om = O.OracleMesh(c.mesh)
    ref, _, rr, bad = om.cls_solve(c.w0)
    assert bad == 0
    pcs = {"exact": G.PC_ILU_EXACT, "sweep": G.PC_ILU_SWEEP, "levels": G.PC_ILU_LEVELS, "bjacobi": G.PC_BJACOBI}
    m = G.GksMesh(c.mesh, precond=pcs[pc])
    coef, info = m.cls_reconstruct(dev(c.w0))
    assert info["converged"] == 1 and max(info["relres"]) <= 1e-12
    got = host(coef)
    for v in range(4):
        if np.max(np.abs(ref[v])) == 0.0:
            assert np.all(got[v] == 0.0)
        else:
            assert rel_max(got[v], ref[v]) <= 1e-9, (v, rel_max(got[v], ref[v]))


@pytest.mark.parametrize("name", list(CASES))
def test_face_flux_matches_oracle(O, G, name):
    c = CASES[name]()
    om = O.OracleMesh(c.mesh)
    coef, _, _, _ = om.cls_solve(c.w0)
    dt = 0.7 * om.cfl_dt(c.w0)
    ref = om.face_flux(c.w0, coef, dt)
    m = G.GksMesh(c.mesh)
    got, st = m.flux(dev(c.w0), dev(coef), dt)
    got = host(got)
    assert np.all(rel_max(got, ref, axis=1) <= 1e-12), rel_max(got, ref, axis=1)


# --------------------------------------------------------------------------- full steps

@pytest.mark.parametrize("name", list(CASES))
@pytest.mark.parametrize("pc", ["exact", "sweep"])
def test_one_step_matches_oracle(O, G, name, pc):
    c = CASES[name]()
    om = O.OracleMesh(c.mesh)
    wo = c.w0.copy()
    dt = om.cfl_dt(wo)
    info_o = om.step(wo, dt)
    assert info_o.status == 0
    m = G.GksMesh(c.mesh, precond=G.PC_ILU_EXACT if pc == "exact" else G.PC_ILU_SWEEP)
    w = dev(c.w0)
    info = m.step(w, dt)
    assert info["status"] == 0 and abs(info["dt"] - dt) == 0.0
    err = rel_max(host(w), wo, axis=1)
    assert np.all(err <= 1e-10), err


def test_cfl_dt_matches_oracle(O, G):
    c = CASES["shock_vortex40x20"]()
    om = O.OracleMesh(c.mesh)
    m = G.GksMesh(c.mesh)
    assert abs(m.cfl_dt(dev(c.w0)) - om.cfl_dt(c.w0)) <= 1e-14 * om.cfl_dt(c.w0)


def test_hundred_steps_match_oracle(O, G):
    """Config-1 workload: 20 x 20 jittered periodic advection, 100 CFL steps."""
    c = I.advection_case(20)
    om = O.OracleMesh(c.mesh)
    wo = c.w0.copy()
    m = G.GksMesh(c.mesh)
    w = dev(c.w0)
    for _ in range(100):
        io = om.step(wo)
        ig = m.step(w)
        assert io.status == 0 and ig["status"] == 0
    err = rel_max(host(w), wo, axis=1)
    assert np.all(err <= 1e-8), err


def test_run_matches_steps(G):
    c = I.advection_case(12, k=2)
    m1 = G.GksMesh(c.mesh)
    m2 = G.GksMesh(c.mesh)
    w1, w2 = dev(c.w0), dev(c.w0)
    info = m1.run(w1, t_final=0.05, max_steps=10000)
    t = 0.0
    while t < 0.05 * (1 - 1e-14):
        dt = min(m2.cfl_dt(w2), 0.05 - t)
        m2.step(w2, dt)
        t += dt
    assert abs(info["t"] - 0.05) < 1e-14
    assert np.array_equal(host(w1), host(w2))


@pytest.mark.parametrize("prandtl", [1.0, 0.72])
def test_viscous_noslip_cavity_matches_oracle(O, G, prandtl):
    c = I.cavity_case(10)
    om = O.OracleMesh(c.mesh, mu=c.mu, prandtl=prandtl)
    wo = c.w0.copy()
    m = G.GksMesh(c.mesh, mu=c.mu, prandtl=prandtl)
    w = dev(c.w0)
    for _ in range(5):
        dt = om.cfl_dt(wo)
        assert om.step(wo, dt).status == 0
        assert m.step(w, dt)["status"] == 0
    wg = host(w)
    assert np.all(rel_max(wg, wo, axis=1) <= 1e-10)
    err = rel_max(wg - c.w0, wo - c.w0, axis=1)          # the flow starts at rest: compare the change too
    assert np.all(err[[1, 2]] <= 1e-9), err


# --------------------------------------------------------------------------- invariants on the GPU

def test_free_stream_and_conservation_on_gpu(G):
    c = I.advection_case(16, k=2)
    m = G.GksMesh(c.mesh)
    T = c.mesh.n_tri
    rho, u, v, p = 1.3, 0.9, -0.6, 0.7
    w0 = np.stack([np.full(T, rho), np.full(T, rho * u), np.full(T, rho * v),
                   np.full(T, p / 0.4 + 0.5 * rho * (u * u + v * v))])
    w = dev(w0)
    for _ in range(3):
        m.step(w)
    assert rel_max(host(w), w0) < 1e-13
    from oracle import oracle
    area = oracle.OracleMesh(c.mesh).cell_geometry()["area"]
    w = dev(c.w0)
    tot0 = (c.w0 * area).sum(axis=1)
    for _ in range(10):
        m.step(w)
    tot = (host(w) * area).sum(axis=1)
    assert np.all(np.abs(tot - tot0) <= 1e-13 * np.abs(tot0).max())


def test_deterministic_repeat(G):
    c = I.shock_vortex_case(30, 15)
    outs = []
    for _ in range(2):
        m = G.GksMesh(c.mesh)
        w = dev(c.w0)
        for _ in range(3):
            m.step(w)
        outs.append(host(w))
    assert np.array_equal(outs[0], outs[1])


# --------------------------------------------------------------------------- kinetic interface slopes

@pytest.mark.parametrize("precision", ["fp64", "mixed"])
@pytest.mark.parametrize("prandtl", [1.0, 0.72])
def test_kinetic_interface_slopes_point_flux_matches_oracle(O, G, precision, prandtl):
    """slope0_mode = 1 (interface derivatives by kinetic weighting) against the
    oracle's own construction of the same half-space moments: 1e-12 of each
    flux scale in FP64, 1e-7 in mixed precision; the mode changes the flux of
    discontinuous states."""
    rng = np.random.default_rng(31)
    n = 200
    wl, wr = _random_states(rng, n, 0.5), _random_states(rng, n, 0.5)
    if precision == "mixed":
        for q in (wl, wr):
            q[:, 1:] *= 0.1
    dt, mu = 0.004, 1e-3
    got = host(G.point_flux(dev(wl), dev(wr), dt, mu=mu, prandtl=prandtl, slope0_mode=1,
                            precision=G.MIXED if precision == "mixed" else G.FP64))
    ref = np.stack([O.point_flux(wl[q], wr[q], dt, mu=mu, prandtl=prandtl, slope0_mode=1)[0] for q in range(n)])
    base = np.stack([O.point_flux(wl[q], wr[q], dt, mu=mu, prandtl=prandtl)[0] for q in range(n)])
    assert np.max(np.abs(ref - base)) > 1e-6 * np.max(np.abs(ref))
    scale = np.max(np.abs(ref), axis=0)
    tol = 1e-12 if precision == "fp64" else 1e-7
    assert np.all(np.max(np.abs(got - ref), axis=0) <= tol * scale), np.max(np.abs(got - ref), axis=0) / scale


@pytest.mark.parametrize("name", ["shock_vortex40x20", "walled13x9", "weak_riemann60x4"])
def test_kinetic_interface_slopes_steps_match_oracle(O, G, name):
    """Ten FP64 steps with slope0_mode = 1 stay within 1e-10 relative max of the
    oracle's."""
    c = CASES[name]()
    om = O.OracleMesh(c.mesh, slope0_mode=1)
    m = G.GksMesh(c.mesh, slope0_mode=1)
    wo, w = c.w0.copy(), dev(c.w0)
    for _ in range(10):
        dt = om.cfl_dt(wo)
        assert om.step(wo, dt).status == 0
        assert m.step(w, dt)["status"] == 0
    assert np.all(rel_max(host(w), wo, axis=1) <= 1e-10), rel_max(host(w), wo, axis=1)


# --------------------------------------------------------------------------- global CLS normal equations

@pytest.mark.parametrize("name", list(CASES))
@pytest.mark.parametrize("mode", ["fp64_exact", "fp64_sweep", "mixed"])
def test_global_cls_matches_oracle(O, G, name, mode):
    """cls_global (Eq. (33), C^T C u = C^T b) against the oracle's assembly of the
    same global equations: coefficients within 1e-9 relative max in FP64 (exact
    and sweep ILU) and in mixed precision (FP32 basis, FP16 ILU factors,
    double-FP32 residual); the solution differs from the per-cell equations'."""
    c = CASES[name]()
    om = O.OracleMesh(c.mesh, cls_global=1)
    ref, _, rr, bad = om.cls_solve(c.w0)
    assert bad == 0
    kw = dict(cls_global=1)
    if mode == "mixed":
        kw.update(precision=G.MIXED, basis_fp32=1, ilu_fp16=1)
    else:
        kw.update(precond=G.PC_ILU_EXACT if mode == "fp64_exact" else G.PC_ILU_SWEEP)
    m = G.GksMesh(c.mesh, **kw)
    coef, info = m.cls_reconstruct(dev(c.w0))
    assert info["converged"] == 1 and max(info["relres"]) <= 1e-12
    got = host(coef)
    for v in range(4):
        if np.max(np.abs(ref[v])) == 0.0:
            assert np.all(got[v] == 0.0)
        else:
            assert rel_max(got[v], ref[v]) <= 1e-9, (v, rel_max(got[v], ref[v]))
    per_cell, _, _, _ = O.OracleMesh(c.mesh).cls_solve(c.w0)
    assert np.max(np.abs(per_cell - ref)) > 1e-6 * np.max(np.abs(ref))


@pytest.mark.parametrize("name", ["shock_vortex40x20", "walled13x9"])
def test_global_cls_steps_match_oracle(O, G, name):
    c = CASES[name]()
    om = O.OracleMesh(c.mesh, cls_global=1)
    m = G.GksMesh(c.mesh, cls_global=1)
    wo, w = c.w0.copy(), dev(c.w0)
    for _ in range(5):
        dt = om.cfl_dt(wo)
        assert om.step(wo, dt).status == 0
        assert m.step(w, dt)["status"] == 0
    assert np.all(rel_max(host(w), wo, axis=1) <= 1e-10), rel_max(host(w), wo, axis=1)


# --------------------------------------------------------------------------- derivative order of the CLS equations

@pytest.mark.parametrize("name", ["advection20", "shock_vortex40x20", "walled13x9"])
@pytest.mark.parametrize("glob", [0, 1])
@pytest.mark.parametrize("mode", ["fp64", "mixed"])
def test_second_derivative_equations_match_oracle(O, G, name, glob, mode):
    """cls_M = 2 (second-derivative equations of Eq. (29) for quadratic cells),
    per cell and global, against the oracle's assembly: coefficients within 1e-9
    relative max in FP64 and in mixed precision."""
    c = CASES[name]()
    om = O.OracleMesh(c.mesh, cls_M=2, cls_global=glob)
    ref, _, rr, bad = om.cls_solve(c.w0)
    assert bad == 0
    kw = dict(cls_M=2, cls_global=glob)
    if mode == "mixed":
        kw.update(precision=G.MIXED, basis_fp32=1, ilu_fp16=1)
    m = G.GksMesh(c.mesh, **kw)
    coef, info = m.cls_reconstruct(dev(c.w0))
    assert info["converged"] == 1 and max(info["relres"]) <= 1e-12
    got = host(coef)
    for v in range(4):
        if np.max(np.abs(ref[v])) == 0.0:
            assert np.all(got[v] == 0.0)
        else:
            assert rel_max(got[v], ref[v]) <= 1e-9, (v, rel_max(got[v], ref[v]))


def test_value_equations_second_order_variant_matches_oracle(O, G):
    """cls_M = 0 with the second-order variant (values only, k_i = 1) on a
    y-periodic strip: coefficients and five steps match the oracle; M = 0 with
    quadratic cells is refused."""
    c = CASES["weak_riemann60x4"]()
    om = O.OracleMesh(c.mesh, cls_M=0, second_order=1)
    ref, _, _, bad = om.cls_solve(c.w0)
    assert bad == 0
    m = G.GksMesh(c.mesh, cls_M=0, second_order=1)
    coef, info = m.cls_reconstruct(dev(c.w0))
    got = host(coef)
    for v in range(4):
        if np.max(np.abs(ref[v])) > 0:
            assert rel_max(got[v], ref[v]) <= 1e-9
    wo, w = c.w0.copy(), dev(c.w0)
    for _ in range(5):
        dt = om.cfl_dt(wo)
        assert om.step(wo, dt).status == 0
        assert m.step(w, dt)["status"] == 0
    assert np.all(rel_max(host(w), wo, axis=1) <= 1e-10)
    with pytest.raises(G.GksError):
        G.GksMesh(c.mesh, cls_M=0)
