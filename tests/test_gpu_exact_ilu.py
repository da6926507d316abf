"""The exact block-ILU(0) preconditioner of Sec. III.B (triangular solves on
the RCM order, not sweeps) applied by sync-free kernels: one launch per
relation, rows taken in RCM order by block tickets, each row waiting (bounded)
for its neighbours' ready tags.  Its rows do the arithmetic of the
level-by-level launches, so the two agree bit for bit; a wait that runs out
is reported as GKS_ETIMEOUT instead of hanging."""
import numpy as np
import pytest

from paper_1802_00704_gb300 import inputs as I
from tests.gpu_util import dev, host, needs_gpu

pytestmark = [pytest.mark.gpu, needs_gpu]


@pytest.fixture(scope="module")
def G():
    from paper_1802_00704_gb300 import build, gks
    build.build()
    return gks


def _steps(G, mesh, w0, pc, prec, n, **kw):
    m = G.GksMesh(mesh, precond=pc, precision=prec, **kw)
    w = dev(w0)
    its = [m.step(w, 2e-4)["iters"] for _ in range(n)]
    return host(w), its


@pytest.mark.parametrize("precision", ["fp64", "mixed"])
@pytest.mark.parametrize("case", ["shock_vortex", "advection", "walled_global"])
def test_sync_free_solves_equal_the_level_launches(G, precision, case):
    """Three steps with the sync-free exact solves and with one launch per
    level: the same states and GMRES iterations, bit for bit (per-cell and
    global normal equations, FP64 and the mixed FP32 preconditioner)."""
    prec = G.MIXED if precision == "mixed" else G.FP64
    kw = {}
    if case == "shock_vortex":
        c = I.shock_vortex_case(40, 20)
    elif case == "advection":
        c = I.advection_case(12, k=2)
    else:
        c = I.advection_case(10, k=1)
        kw = {"cls_global": 1}
    a = _steps(G, c.mesh, c.w0, G.PC_ILU_EXACT, prec, 3, **kw)
    b = _steps(G, c.mesh, c.w0, G.PC_ILU_LEVELS, prec, 3, **kw)
    assert np.array_equal(a[0], b[0])
    assert a[1] == b[1]


def test_sync_free_solves_on_a_batch(G):
    """Cases of a batch share the launches; each case's rows wait only on its
    own rows: the batch equals the level launches on the same batch."""
    cases = [I.advection_case(12, k=2), I.shock_vortex_case(30, 15), I.advection_case(7, seed=5)]
    w0 = np.ascontiguousarray(np.concatenate([c.w0 for c in cases], axis=1))
    res = []
    for pc in (G.PC_ILU_EXACT, G.PC_ILU_LEVELS):
        b = G.GksMesh.batch([c.mesh for c in cases], precond=pc, precision=G.MIXED)
        w = dev(w0)
        r = b.batch_run(w, max_steps=3)
        assert r["n_failed"] == 0
        res.append((host(w), r["gmres_iters"]))
    assert np.array_equal(res[0][0], res[1][0]) and res[0][1] == res[1][1]


def test_sync_free_solves_in_the_run_graph(G):
    """gks_run with the exact solves as one graph launch equals the host loop."""
    c = I.shock_vortex_case(30, 15)
    out = []
    for mode in (0, 1):
        m = G.GksMesh(c.mesh, precond=G.PC_ILU_EXACT, precision=G.MIXED, no_graphs=mode)
        w = dev(c.w0)
        info = m.run(w, max_steps=4)
        out.append((host(w), info["gmres_iters"]))
    assert np.array_equal(out[0][0], out[1][0]) and out[0][1] == out[1][1]


def test_exact_preconditioner_needs_fewer_iterations_than_the_diagonal(G):
    """The exact ILU(0) solve is a stronger preconditioner than one sweep, and
    both are stronger than the block-diagonal inverse."""
    c = I.shock_vortex_case(40, 20)
    it = {}
    for name, pc in (("exact", G.PC_ILU_EXACT), ("sweep1", G.PC_ILU_SWEEP), ("bjacobi", G.PC_BJACOBI)):
        m = G.GksMesh(c.mesh, precond=pc, ilu_sweeps=1)
        _, info = m.cls_reconstruct(dev(c.w0))
        assert info["converged"] == 1
        it[name] = sum(info["iters"])
    assert it["exact"] <= it["sweep1"] < it["bjacobi"]


def test_bounded_wait_gives_up_on_a_flag_nothing_sets(G):
    """The wait of the sync-free solves on its own: on a flag that nothing sets
    it gives up after its limit and says so; on a set flag it returns at once."""
    to, ns = G.probe_wait(2_000_000, False)
    assert to and 2_000_000 <= ns < 1_000_000_000
    to, ns = G.probe_wait(1_000_000_000, True)
    assert not to and ns < 1_000_000
