"""Full-size check on the 1,000,000-triangle shock-vortex workload (1000 x 500
jittered split quads), in the launch configuration the benchmark times:
sampled outputs against the oracle and properties that hold at any size."""
import numpy as np
import pytest

from paper_1802_00704_gb300 import inputs as I
from tests.gpu_util import dev, host, needs_gpu, rel_max, torch

pytestmark = [pytest.mark.gpu, needs_gpu]


@pytest.fixture(scope="module")
def big():
    from oracle import oracle
    from paper_1802_00704_gb300 import build, gks
    oracle.build()
    build.build()
    c = I.shock_vortex_case(1000, 500)
    return c, oracle.OracleMesh(c.mesh), gks.GksMesh(c.mesh), gks


def test_fullsize_reconstruction_residual(big):
    import scipy.sparse as sps
    c, om, g, G = big
    coef, info = g.cls_reconstruct(dev(c.w0))
    assert info["converged"] == 1
    x = host(coef)
    rp, col, val, off = om.cls_matrix()
    K = sps.csr_matrix((val, col, rp), shape=(om.ndof, om.ndof))
    rhs = om.cls_rhs(c.w0)
    k = om.cell_geometry()["k"].astype(int)
    for v in range(4):
        xv = np.zeros(om.ndof)
        two = k == 2
        for l in range(5):
            sel = two if l >= 2 else np.ones_like(two)
            xv[off[sel] + l] = x[v, l, sel]
        assert np.all(x[v, 2:, ~two] == 0.0)
        r = K @ xv - rhs[v]
        assert np.linalg.norm(r) <= 1e-10 * np.linalg.norm(rhs[v]), (v, np.linalg.norm(r) / np.linalg.norm(rhs[v]))


def test_fullsize_sampled_fluxes_and_balance(big):
    c, om, g, G = big
    w = dev(c.w0)
    coef, _ = g.cls_reconstruct(w)
    dt = g.cfl_dt(w)
    flux, st = g.flux(w, coef, dt)
    fl = host(flux)
    rng = np.random.default_rng(704)
    ids = np.unique(np.concatenate([rng.integers(0, c.mesh.n_face, 3000),
                                    np.nonzero(c.mesh.faces[:, 3] < 0)[0][::7]]))
    ref = om.face_flux_subset(c.w0, host(coef), dt, ids)
    scale = np.max(np.abs(fl), axis=1, keepdims=True)
    assert np.all(np.abs(fl[:, ids] - ref) <= 1e-12 * scale)
    # one step: the change of the totals equals minus the boundary fluxes
    area = om.cell_geometry()["area"]
    w1 = dev(c.w0)
    g.reset_warm_start()
    info = g.step(w1, dt)
    assert info["status"] == 0
    d_tot = ((host(w1) - c.w0) * area).sum(axis=1)
    bnd = c.mesh.faces[:, 3] < 0
    out = fl[:, bnd].sum(axis=1)
    tot = (np.abs(c.w0) * area).sum(axis=1)
    assert np.all(np.abs(d_tot + out) <= 1e-12 * tot), (d_tot, out)


def test_fullsize_mixed_path_as_benchmarked(big):
    """The mixed path with the knobs the benchmark's tuner picks (2 sweeps,
    quadratic warm start, inner tolerance 1e-4) and its FP32 Krylov basis: 4 steps stay within 1e-8
    relative L1 of the FP64 path, and sampled mixed face fluxes agree with the
    oracle to 1e-7 of the largest flux."""
    c, om, g, G = big
    area = om.cell_geometry()["area"]
    mx = G.GksMesh(c.mesh, precision=G.MIXED, ilu_sweeps=2, warm_extrap=2, inner_rtol=1e-4, basis_fp32=1)
    g.reset_warm_start()
    wm, wf = dev(c.w0), dev(c.w0)
    for _ in range(4):
        dt = g.cfl_dt(wf)
        assert mx.step(wm, dt)["status"] == 0
        assert g.step(wf, dt)["status"] == 0
    a, b = host(wm), host(wf)
    l1 = np.sum(area * np.abs(a - b), axis=1) / np.sum(area * np.abs(b), axis=1)
    assert np.all(l1 <= 1e-8), l1
    coef, _ = mx.cls_reconstruct(dev(c.w0))
    dt = g.cfl_dt(dev(c.w0))
    fl = host(mx.flux(dev(c.w0), coef, dt)[0])
    ids = np.random.default_rng(11).integers(0, c.mesh.n_face, 2000)
    ref = om.face_flux_subset(c.w0, host(coef), dt, ids)
    scale = np.max(np.abs(fl), axis=1, keepdims=True)
    assert np.all(np.abs(fl[:, ids] - ref) <= 1e-7 * scale)


def test_config5_batch_50_steps_against_oracle_and_fp64():
    """The 512-case batch (19.8M triangles, log-uniform 1e3-2e5 per case,
    advection and Riemann strips with ratios 2-10) in the benchmark's launch
    configuration (mixed, FP32 Krylov basis, robust limiter, GMRES(12)) for the
    configuration's 50 steps: every case physical; the six smallest cases equal
    the oracle's own 50 steps to 1e-8 relative L1 per conserved variable; and
    every case of the batch equals the FP64 batch's state to 1e-8 relative L1."""
    from oracle import oracle
    from paper_1802_00704_gb300 import build, gks
    oracle.build()
    build.build()
    cases = I.batch_cases(512, workers=16)
    w0 = np.ascontiguousarray(np.concatenate([c.w0 for c in cases], axis=1))
    offs = np.concatenate([[0], np.cumsum([c.mesh.n_tri for c in cases])])
    states = {}
    for prec in ("mixed", "fp64"):
        kw = dict(precision=gks.MIXED, basis_fp32=1) if prec == "mixed" else dict(precision=gks.FP64)
        b = gks.GksMesh.batch([c.mesh for c in cases], limiter=2, gmres_m=12, **kw)
        w = dev(w0)
        r = b.batch_run(w, max_steps=50)
        assert r["n_failed"] == 0 and r["steps"] == 50, (prec, r["n_failed"], r["steps"])
        states[prec] = host(w)
        del b
    wm, wf = states["mixed"], states["fp64"]
    for q, c in enumerate(cases):
        p = c.mesh.nodes[c.mesh.tris]
        area = 0.5 * np.abs((p[:, 1, 0] - p[:, 0, 0]) * (p[:, 2, 1] - p[:, 0, 1]) -
                            (p[:, 2, 0] - p[:, 0, 0]) * (p[:, 1, 1] - p[:, 0, 1]))
        a, f = wm[:, offs[q]:offs[q + 1]], wf[:, offs[q]:offs[q + 1]]
        l1 = np.sum(area * np.abs(a - f), axis=1) / np.sum(area * np.abs(f), axis=1)
        assert np.all(l1 <= 1e-8), (q, l1)
    for q in np.argsort([c.mesh.n_tri for c in cases])[:6]:
        c = cases[q]
        om = oracle.OracleMesh(c.mesh, limiter=2)
        wo = c.w0.copy()
        for _ in range(50):
            assert om.step(wo).status == 0
        area = om.cell_geometry()["area"]
        got = wm[:, offs[q]:offs[q + 1]]
        l1 = np.sum(area * np.abs(got - wo), axis=1) / np.sum(area * np.abs(wo), axis=1)
        assert np.all(l1 <= 1e-8), (q, l1)
