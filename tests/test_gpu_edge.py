"""Edge cases of the CUDA path: tiny and ragged meshes, boundary-only cells,
zero right-hand sides, error reporting (non-physical state, GMRES cap,
invalid input, unsupported option)."""
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


@pytest.mark.parametrize("nx,ny", [(3, 3), (5, 3), (3, 7)])
def test_tiny_periodic_meshes(O, G, nx, ny):
    m = I.split_quad_mesh(nx, ny, 2.0, 1.0, seed=4, periodic_x=True, periodic_y=True)
    w0 = I.cell_average(m, lambda x, y: I.prim_to_cons(1 + 0.1 * np.sin(np.pi * x), 0.5 + 0 * x, 0.2 + 0 * x,
                                                        1 + 0 * x, 1.4))
    om = O.OracleMesh(m)
    wo = w0.copy()
    dt = om.cfl_dt(wo)
    om.step(wo, dt)
    g = G.GksMesh(m, precond=G.PC_ILU_EXACT)
    w = dev(w0)
    g.step(w, dt)
    assert np.all(rel_max(host(w), wo, axis=1) <= 1e-10)


def test_mostly_boundary_cells(O, G):
    st = I.prim_to_cons(np.float64(1.0), np.float64(0.3), np.float64(0.0), np.float64(1.0), 1.4)
    bc = {s: (I.TAG_DIRICHLET, st) for s in ("left", "right", "bottom", "top")}
    m = I.split_quad_mesh(3, 3, 1.0, 1.0, seed=8, bc=bc)
    w0 = I.cell_average(m, lambda x, y: I.prim_to_cons(1 + 0.1 * x * y, 0.3 + 0 * x, 0 * x, 1 + 0.05 * y, 1.4))
    om = O.OracleMesh(m)
    k = om.cell_geometry()["k"]
    assert (k == 1).sum() > (k == 2).sum()
    wo = w0.copy()
    dt = om.cfl_dt(wo)
    om.step(wo, dt)
    g = G.GksMesh(m)
    assert g.stats()["n_k1"] == int((k == 1).sum())
    w = dev(w0)
    g.step(w, dt)
    assert np.all(rel_max(host(w), wo, axis=1) <= 1e-10)


def test_zero_rhs_gives_exact_zero_coefficients(G):
    c = I.advection_case(9)
    g = G.GksMesh(c.mesh)
    T = c.mesh.n_tri
    w = dev(np.stack([np.full(T, 1.1), np.full(T, 0.2), np.full(T, -0.3), np.full(T, 2.7)]))
    coef, info = g.cls_reconstruct(w)
    assert info["iters"] == [0, 0, 0, 0] and torch.count_nonzero(coef).item() == 0


def test_nonphysical_state_is_reported(G):
    c = I.sod_case(40, 4)
    g = G.GksMesh(c.mesh)
    w = dev(c.w0)
    info = g.step(w, check=False)
    assert info["status"] == G.GKS_ENONPHYS


def test_gmres_cap_is_reported(G):
    c = I.advection_case(10)
    g = G.GksMesh(c.mesh, gmres_maxit=1)
    coef, info = g.cls_reconstruct(dev(c.w0), check=False)
    assert info["status"] == G.GKS_ENOCONV and info["converged"] == 0 and max(info["iters"]) == 1


def test_invalid_inputs_are_rejected(G):
    c = I.advection_case(5)
    bad = c.mesh.faces.copy()
    bad[3, 2] = c.mesh.n_tri + 5
    m2 = I.Mesh(c.mesh.nodes, c.mesh.tris, bad, c.mesh.face_shift, c.mesh.bc_state)
    with pytest.raises(G.GksError) as e:
        G.GksMesh(m2)
    assert e.value.status == G.GKS_EINVAL
    bad = c.mesh.faces.copy()
    bad[0, 4] = 9                      # tag out of range
    with pytest.raises(G.GksError):
        G.GksMesh(I.Mesh(c.mesh.nodes, c.mesh.tris, bad, c.mesh.face_shift, c.mesh.bc_state))
    with pytest.raises(G.GksError) as e:
        G.GksMesh(c.mesh, precision=7)
    assert e.value.status == G.GKS_EINVAL
    with pytest.raises(G.GksError) as e:
        G.GksMesh(c.mesh, precond=9)
    assert e.value.status == G.GKS_EINVAL
    with pytest.raises(G.GksError) as e:
        G.GksMesh(c.mesh, gmres_m=0)
    assert e.value.status == G.GKS_EINVAL


def test_level_structure_is_reported(G):
    c = I.advection_case(20)
    s = G.GksMesh(c.mesh).stats()
    assert s["n_tri"] == 800 and s["n_face"] == 1200 and s["nnzb"] == 800 + 2400
    assert 1 < s["levels_lower"] < 800 and 1 < s["levels_upper"] < 800
