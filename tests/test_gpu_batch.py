"""Batched cases: several independent meshes of uneven size in one handle.
Each case must advance exactly as it does alone (the kernels cover all cases
at once, reductions are segmented per case and the GMRES masks are per case
and variable, so the arithmetic per case is the same), cases keep their own
time steps and end times, and a failing case does not stop the others."""
import numpy as np
import pytest

from paper_1802_00704_gb300 import inputs as I
from tests.gpu_util import dev, host, needs_gpu, rel_max, torch

pytestmark = [pytest.mark.gpu, needs_gpu]


@pytest.fixture(scope="module")
def G():
    from paper_1802_00704_gb300 import build, gks
    build.build()
    return gks


def _cases():
    st = I.prim_to_cons(np.float64(1.0), np.float64(0.2), np.float64(-0.1), np.float64(1.0), 1.4)
    bc = {s: (I.TAG_DIRICHLET, st) for s in ("left", "right", "bottom", "top")}
    m3 = I.split_quad_mesh(11, 7, 1.0, 0.8, seed=3, bc=bc)
    w3 = I.cell_average(m3, lambda x, y: I.prim_to_cons(1 + 0.2 * np.sin(3 * x + y), 0.2 + 0 * x, -0.1 + 0 * x,
                                                        1 + 0.1 * np.cos(x - y), 1.4))
    return [I.advection_case(12, k=2), I.shock_vortex_case(30, 15), I.Case("walled", m3, w3),
            I.advection_case(7, seed=5)]


def _concat(cases):
    return np.ascontiguousarray(np.concatenate([c.w0 for c in cases], axis=1))


def _split(w, cases):
    out, o = [], 0
    for c in cases:
        out.append(w[:, o:o + c.mesh.n_tri])
        o += c.mesh.n_tri
    return out


@pytest.mark.parametrize("precision", ["fp64", "mixed"])
def test_batch_cases_match_single_runs(G, precision):
    cases = _cases()
    prec = G.MIXED if precision == "mixed" else G.FP64
    b = G.GksMesh.batch([c.mesh for c in cases], precision=prec)
    assert b.stats()["n_case"] == len(cases)
    w = dev(_concat(cases))
    r = b.batch_run(w, max_steps=4)
    assert r["n_failed"] == 0 and r["steps"] == 4
    got = _split(host(w), cases)
    for c, g in zip(cases, got):
        m = G.GksMesh(c.mesh, precision=prec)
        ws = dev(c.w0)
        m.run(ws, max_steps=4)
        assert rel_max(g, host(ws)) <= 1e-13, c.name


def test_batch_end_times_per_case(G):
    cases = _cases()[:3]
    b = G.GksMesh.batch([c.mesh for c in cases])
    w = dev(_concat(cases))
    tf = np.array([0.004, 0.0015, 0.003])
    r = b.batch_run(w, t_final=tf, max_steps=10000)
    assert np.all(np.abs(r["t"] - tf) <= 1e-15 * tf) and r["n_finished"] == 3
    for c, g, t in zip(cases, _split(host(w), cases), tf):
        m = G.GksMesh(c.mesh)
        ws = dev(c.w0)
        info = m.run(ws, t_final=t, max_steps=10000)
        assert abs(info["t"] - t) <= 1e-15 * t
        assert rel_max(g, host(ws)) <= 1e-13


def test_failing_case_does_not_stop_the_others(G):
    good = I.advection_case(9)
    bad = I.sod_case(40, 4)                       # unlimited quadratic reconstruction goes non-physical
    b = G.GksMesh.batch([good.mesh, bad.mesh])
    w = dev(_concat([good, bad]))
    r = b.batch_run(w, max_steps=3)
    assert list(r["status"]) == [G.GKS_OK, G.GKS_ENONPHYS] and r["n_failed"] == 1
    m = G.GksMesh(good.mesh)
    ws = dev(good.w0)
    m.run(ws, max_steps=3)
    assert rel_max(_split(host(w), [good, bad])[0], host(ws)) <= 1e-13


def test_many_small_cases(G):
    cases = [I.advection_case(3 + (q % 9), k=1 + q % 3, seed=100 + q) for q in range(40)]
    b = G.GksMesh.batch([c.mesh for c in cases], precision=G.MIXED, gmres_m=12)
    w = dev(_concat(cases))
    r = b.batch_run(w, max_steps=2)
    assert r["n_failed"] == 0
    for c, g in list(zip(cases, _split(host(w), cases)))[::7]:
        m = G.GksMesh(c.mesh, precision=G.MIXED, gmres_m=12)
        ws = dev(c.w0)
        m.run(ws, max_steps=2)
        assert rel_max(g, host(ws)) <= 1e-13


def test_single_mesh_entry_points_refuse_batches(G):
    cases = _cases()[:2]
    b = G.GksMesh.batch([c.mesh for c in cases])
    w = dev(_concat(cases))
    with pytest.raises(G.GksError):
        b.step(w)
    with pytest.raises(G.GksError):
        b.cfl_dt_noalloc(w, torch.zeros(1, dtype=torch.float64, device="cuda"))


@pytest.mark.parametrize("precision", ["fp64", "mixed"])
def test_finished_case_keeps_its_warm_start_history(G, precision):
    """Extrapolated warm start in a batch whose cases finish at different times
    (the history buffers rotate for every case; a finished case exchanges its
    two buffers' contents so that it keeps its history): a second run of the
    batch reaches, per case, the states of a single run that stopped and
    resumed at the same times (1e-10: both solves meet 1e-12, from guesses that
    may differ in rounding)."""
    cases = _cases()[:3]
    prec = G.MIXED if precision == "mixed" else G.FP64
    kw = dict(precision=prec, warm_extrap=2, basis_fp32=int(precision == "mixed"))
    b = G.GksMesh.batch([c.mesh for c in cases], **kw)
    w = dev(_concat(cases))
    t1 = np.array([0.004, 0.0015, 0.003])
    t2 = np.array([0.006, 0.005, 0.0045])
    r1 = b.batch_run(w, t_final=t1, max_steps=10000)
    r2 = b.batch_run(w, t_final=t2, max_steps=10000)
    assert r1["n_finished"] == 3 and r2["n_finished"] == 3 and r2["n_failed"] == 0
    for c, g, ta, tb in zip(cases, _split(host(w), cases), t1, t2):
        m = G.GksMesh(c.mesh, **kw)
        ws = dev(c.w0)
        m.run(ws, t_final=ta, max_steps=10000)
        m.run(ws, t_final=tb, max_steps=10000)
        assert rel_max(g, host(ws)) <= 1e-10, c.name
