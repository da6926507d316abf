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
