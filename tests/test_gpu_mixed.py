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


def _true_relres(om, w, coef):
    """||b - K x|| / ||b|| per variable in FP64 from the oracle's CLS matrix."""
    import scipy.sparse as sp
    rp, col, val, off = om.cls_matrix()
    n = len(rp) - 1
    K = sp.csr_matrix((val, col, rp), shape=(n, n))
    b = om.cls_rhs(w)
    nd = np.diff(np.append(off, n))
    X = np.zeros((4, n))
    for i in range(len(off)):
        X[:, off[i]:off[i] + nd[i]] = coef[:, :nd[i], i]
    out = []
    for v in range(4):
        bn = np.linalg.norm(b[v])
        out.append(np.linalg.norm(b[v] - K @ X[v]) / bn if bn > 0 else 0.0)
    return np.array(out)


@pytest.mark.parametrize("name", ["advection20", "shock_vortex40x20", "walled13x9"])
def test_refinement_residual_matches_fp64_residual(O, G, name):
    """The mixed mode's refinement residual (double-FP32 arithmetic with the FP32
    basis) certifies the FP64 tolerance: the relative residual the solve reports
    equals the FP64 residual of the returned coefficients, computed from the
    oracle's matrix, to 1e-14 of |b|, and that residual is below 1e-12."""
    from tests.test_gpu_parity import CASES
    c = CASES[name]()
    om = O.OracleMesh(c.mesh)
    m = G.GksMesh(c.mesh, precision=G.MIXED, basis_fp32=1)
    coef, info = m.cls_reconstruct(dev(c.w0))
    assert info["converged"] == 1
    true = _true_relres(om, c.w0, host(coef))
    rep = np.array(info["relres"])
    assert np.all(true <= 1.01e-12), true
    assert np.all(np.abs(rep - true) <= 1e-14), (rep, true)


@pytest.mark.parametrize("where", ["everywhere", "left_half"])
def test_tiny_variable_keeps_fp32_basis_accurate(O, G, where):
    """A variable of size 1e-30 (rho v of a nearly one-dimensional flow) is
    below the range of the double-FP32 split (such cells take the FP64
    operator) and its squares below FP32's range: the first basis vector is
    stored scaled by a power of two near 1/|b|, so the solve still reaches the
    FP64 tolerance and matches the oracle."""
    c = I.advection_case(20, seed=9)
    w = c.w0.copy()
    rng = np.random.default_rng(3)
    tiny = 1e-30 * (0.5 + rng.random(w.shape[1]))
    if where == "everywhere":
        w[2] = tiny
    else:
        cx = O.OracleMesh(c.mesh).cell_geometry()["cx"]
        w[2] = np.where(cx < 0.5, tiny, 1e-3 * (0.5 + rng.random(w.shape[1])))
    om = O.OracleMesh(c.mesh)
    ref, _, _, _ = om.cls_solve(w)
    m = G.GksMesh(c.mesh, precision=G.MIXED, basis_fp32=1)
    coef, info = m.cls_reconstruct(dev(w))
    assert info["converged"] == 1 and max(info["relres"]) <= 1e-12, info
    got = host(coef)
    for v in range(4):
        assert rel_max(got[v], ref[v]) <= 1e-9, (v, rel_max(got[v], ref[v]))
    assert np.all(_true_relres(om, w, got) <= 1.01e-12)


def test_warm_start_far_from_new_system(O, G):
    """A warm start from a flow whose rho v is 1e50 times larger than the new
    one: the first residual is 1e48 times |b|, and the FP32 basis stores it
    scaled by the larger of |b| and the previous |b| (the warm start's own
    scale), not overflowing; later restarts rescale by the cycle's estimate.
    The solve meets the FP64 tolerance and matches the oracle's solve from zero."""
    c = I.advection_case(20, seed=4)
    rng = np.random.default_rng(8)
    m = G.GksMesh(c.mesh, precision=G.MIXED, basis_fp32=1)
    _, info1 = m.cls_reconstruct(dev(c.w0))     # warm start with rho v of order one
    assert info1["converged"] == 1
    w2 = c.w0.copy()
    w2[2] = 1e-50 * (0.5 + rng.random(w2.shape[1]))
    om = O.OracleMesh(c.mesh)
    ref, _, _, _ = om.cls_solve(w2)
    coef, info = m.cls_reconstruct(dev(w2))
    assert info["converged"] == 1 and max(info["relres"]) <= 1e-12, info
    got = host(coef)
    for v in range(4):
        assert rel_max(got[v], ref[v]) <= 1e-9, (v, rel_max(got[v], ref[v]))


@pytest.mark.parametrize("name", ["advection20", "shock_vortex40x20", "walled13x9"])
def test_fp16_ilu_factors_reach_fp64_tolerance(O, G, name):
    """ilu_fp16: the FP32 preconditioner reads FP16 copies of the ILU(0) factors.
    A fixed preconditioner: the solve still meets the FP64 tolerance, matches the
    oracle's coefficients to 1e-9, and needs at most one more Arnoldi iteration
    per variable than with FP32 factors; with FP16 asked for in FP64 mode the
    configuration is refused."""
    from tests.test_gpu_parity import CASES
    c = CASES[name]()
    om = O.OracleMesh(c.mesh)
    ref, _, _, _ = om.cls_solve(c.w0)
    its = []
    for f16 in (0, 1):
        m = G.GksMesh(c.mesh, precision=G.MIXED, basis_fp32=1, ilu_fp16=f16)
        coef, info = m.cls_reconstruct(dev(c.w0))
        assert info["converged"] == 1 and max(info["relres"]) <= 1e-12
        got = host(coef)
        for v in range(4):
            if np.max(np.abs(ref[v])) > 0:
                assert rel_max(got[v], ref[v]) <= 1e-9
        its.append(info["iters"])
    assert all(b <= a + 1 for a, b in zip(*its)), its
    with pytest.raises(G.GksError):
        G.GksMesh(c.mesh, precision=G.FP64, ilu_fp16=1)


def test_fp16_ilu_factors_steps_within_1e8_l1(O, G):
    c = I.shock_vortex_case(40, 20)
    area = O.OracleMesh(c.mesh).cell_geometry()["area"]
    om = O.OracleMesh(c.mesh)
    m = G.GksMesh(c.mesh, precision=G.MIXED, basis_fp32=1, ilu_fp16=1, warm_extrap=2)
    wo, w = c.w0.copy(), dev(c.w0)
    for _ in range(20):
        dt = om.cfl_dt(wo)
        assert om.step(wo, dt).status == 0
        assert m.step(w, dt)["status"] == 0
    assert np.all(rel_l1(host(w), wo, area) <= 1e-8), rel_l1(host(w), wo, area)
