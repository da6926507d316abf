"""Mixed-precision path (GKS_MIXED) against the FP64 oracle.

The CLS coefficients still reach the FP64 tolerance (iterative refinement
with FP64 residuals), so they match as tightly as the FP64 path.  The flux
computes only slope-carrying terms in FP32; their size relative to the flux
is of order dt |grad W| / |W|, so the error budget of a state after n steps is
about n * 6e-8 * CFL * (h |grad W| / |W|) relative, far below the 1e-8
relative L1 target.  Relative L1 is sum |Omega| |q - q_ref| / sum |Omega| |q_ref|
per conserved variable."""
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


def rel_l1(a, b, area):
    return np.sum(area * np.abs(a - b), axis=1) / np.sum(area * np.abs(b), axis=1)


def test_mixed_point_flux_close_to_oracle(O, G):
    rng = np.random.default_rng(5)
    n = 200
    from tests.test_gpu_parity import _random_states
    wl, wr = _random_states(rng, n), _random_states(rng, n)
    for q in (wl, wr):                          # smooth-flow sized derivatives
        q[:, 1:] *= 0.1
    dt = 0.004
    got = host(G.point_flux(dev(wl), dev(wr), dt, precision=G.MIXED))
    ref = np.stack([O.point_flux(wl[q], wr[q], dt)[0] for q in range(n)])
    scale = np.max(np.abs(ref), axis=0)
    err = np.max(np.abs(got - ref), axis=0) / scale
    assert np.all(err <= 1e-7), err


@pytest.mark.parametrize("basis_fp32", [0, 1])
@pytest.mark.parametrize("name", ["advection20", "shock_vortex40x20", "walled13x9"])
def test_mixed_cls_reaches_fp64_tolerance(O, G, name, basis_fp32):
    from tests.test_gpu_parity import CASES
    c = CASES[name]()
    om = O.OracleMesh(c.mesh)
    ref, _, _, _ = om.cls_solve(c.w0)
    m = G.GksMesh(c.mesh, precision=G.MIXED, basis_fp32=basis_fp32)
    coef, info = m.cls_reconstruct(dev(c.w0))
    assert info["converged"] == 1 and max(info["relres"]) <= 1e-12
    got = host(coef)
    for v in range(4):
        if np.max(np.abs(ref[v])) > 0:
            assert rel_max(got[v], ref[v]) <= 1e-9


@pytest.mark.parametrize("basis_fp32", [0, 1])
@pytest.mark.parametrize("name,steps", [("advection20", 20), ("shock_vortex40x20", 20)])
def test_mixed_steps_within_1e8_l1(O, G, name, steps, basis_fp32):
    from tests.test_gpu_parity import CASES
    c = CASES[name]()
    om = O.OracleMesh(c.mesh)
    area = om.cell_geometry()["area"]
    wo = c.w0.copy()
    m = G.GksMesh(c.mesh, precision=G.MIXED, basis_fp32=basis_fp32)
    w = dev(c.w0)
    for _ in range(steps):
        dt = om.cfl_dt(wo)
        assert om.step(wo, dt).status == 0
        assert m.step(w, dt)["status"] == 0
    err = rel_l1(host(w), wo, area)
    assert np.all(err <= 1e-8), err
    # and the change over the run is resolved well beyond that
    dchg = rel_l1(host(w) - c.w0, wo - c.w0, area)
    assert np.all(dchg[np.abs(wo - c.w0).max(axis=1) > 1e-12] <= 1e-5), dchg


def test_mixed_exact_ilu_and_sweeps_agree(G):
    c = I.shock_vortex_case(30, 15)
    out = []
    for pc in (G.PC_ILU_EXACT, G.PC_ILU_SWEEP):
        m = G.GksMesh(c.mesh, precision=G.MIXED, precond=pc)
        w = dev(c.w0)
        for _ in range(3):
            m.step(w)
        out.append(host(w))
    assert rel_max(out[0], out[1]) <= 1e-11


def test_fp32_basis_needs_mixed_precision(G):
    c = I.advection_case(6)
    with pytest.raises(G.GksError):
        G.GksMesh(c.mesh, precision=G.FP64, basis_fp32=1)


def test_fp32_basis_batch_matches_single_runs(G):
    cases = [I.advection_case(9, k=2), I.shock_vortex_case(24, 12), I.sod_case(60, 4)]
    b = G.GksMesh.batch([c.mesh for c in cases], precision=G.MIXED, basis_fp32=1, limiter=1)
    w = dev(np.ascontiguousarray(np.concatenate([c.w0 for c in cases], axis=1)))
    r = b.batch_run(w, max_steps=4)
    assert r["n_failed"] == 0
    wh, o = host(w), 0
    for c in cases:
        m = G.GksMesh(c.mesh, precision=G.MIXED, basis_fp32=1, limiter=1)
        ws = dev(c.w0)
        m.run(ws, max_steps=4)
        assert rel_max(wh[:, o:o + c.mesh.n_tri], host(ws)) <= 1e-13, c.name
        o += c.mesh.n_tri
