"""Solver options that change how the CLS system is solved but not what it
solves: the extrapolated warm start (initial guess 2 x_{n-1} - x_{n-2}) must
reach the same tolerance, so the states stay within the FP64 parity bounds of
the oracle, with no more GMRES iterations than the plain warm start."""
import numpy as np
import pytest

from paper_1802_00704_gb300 import inputs as I
from tests.gpu_util import dev, host, needs_gpu, rel_max

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


@pytest.mark.parametrize("order", [1, 2])
@pytest.mark.parametrize("precision", ["fp64", "mixed"])
def test_extrapolated_warm_start_matches_oracle(O, G, precision, order):
    c = I.shock_vortex_case(40, 20)
    om = O.OracleMesh(c.mesh)
    prec = G.MIXED if precision == "mixed" else G.FP64
    plain = G.GksMesh(c.mesh, precision=prec)
    extrap = G.GksMesh(c.mesh, precision=prec, warm_extrap=order)
    wo, wp, we = c.w0.copy(), dev(c.w0), dev(c.w0)
    its_p = its_e = 0
    for n in range(30):
        info = om.step(wo)
        assert info.status == 0
        its_p += max(plain.step(wp, info.dt)["iters"])
        r = extrap.step(we, info.dt)
        its_e += max(r["iters"])
        assert max(r["relres"]) <= 1e-12
    assert np.all(rel_max(host(we), wo, axis=1) <= 1e-8)
    assert rel_max(host(we), host(wp)) <= 1e-10
    assert its_e <= its_p, (its_e, its_p)


def test_warm_start_reset_forgets_the_history(G):
    c = I.advection_case(12)
    m = G.GksMesh(c.mesh, warm_extrap=2)
    w = dev(c.w0)
    for _ in range(3):
        m.step(w)
    m.reset_warm_start()
    # after the reset the handle repeats what a fresh one does, bit for bit
    fresh = G.GksMesh(c.mesh, warm_extrap=2)
    wa, wb = dev(c.w0), dev(c.w0)
    for _ in range(4):
        ia = m.step(wa, 1e-3)
        ib = fresh.step(wb, 1e-3)
        assert ia["iters"] == ib["iters"]
    assert np.array_equal(host(wa), host(wb))


@pytest.mark.parametrize("precision", ["fp64", "mixed"])
def test_autotune_keeps_the_state_and_the_results(G, precision):
    c = I.shock_vortex_case(60, 30)
    prec = G.MIXED if precision == "mixed" else G.FP64
    w = dev(c.w0)
    tuned = G.GksMesh(c.mesh, precision=prec)
    r = tuned.autotune(w, trial_steps=2)
    assert np.array_equal(host(w), c.w0)                   # the caller's state is untouched
    assert r["ilu_sweeps"] in (1, 2, 3) and r["warm_extrap"] in (0, 1, 2) and r["ilu_sweeps_bwd"] in (-1, 1, 2)
    # sweeps (1, 2, 3) with the same number backward, (2, 3) with one backward sweep and
    # 1 with a backward pair
    # (x warm start x inner tolerance in mixed precision), then restarts 16 and 8,
    # then (mixed, double-FP32 flux) the two other launch shapes of the flux kernel
    assert r["n_candidates"] == (54 + 2 + 2 if precision == "mixed" else 18 + 2) and r["n_failed"] == 0
    assert r["gmres_m"] in (30, 16, 8) and r["flux_variant"] in ((0, 1, 2) if precision == "mixed" else (0,))
    assert 0 < r["ms_per_step"] <= r["ms_per_step_before"]
    if precision == "fp64":
        assert r["inner_rtol"] == 1e-6
    plain = G.GksMesh(c.mesh, precision=prec)
    wt, wp = dev(c.w0), dev(c.w0)
    for _ in range(6):
        dt = plain.cfl_dt(wp)
        a = tuned.step(wt, dt)
        plain.step(wp, dt)
        assert max(a["relres"]) <= 1e-12
    assert rel_max(host(wt), host(wp)) <= 1e-10


def test_autotune_on_a_batch(G):
    cases = [I.advection_case(14, k=2), I.shock_vortex_case(30, 15), I.sod_case(50, 4)]
    w0 = np.ascontiguousarray(np.concatenate([c.w0 for c in cases], axis=1))
    b = G.GksMesh.batch([c.mesh for c in cases], precision=G.MIXED, limiter=1)
    r = b.autotune(dev(w0), trial_steps=2)
    assert r["n_failed"] == 0
    # a fresh handle with the knobs the tuner chose (a shorter restart changes the
    # iterates within the GMRES tolerance, which the limiter's flags can amplify)
    ref = G.GksMesh.batch([c.mesh for c in cases], precision=G.MIXED, limiter=1, ilu_sweeps=r["ilu_sweeps"],
                          ilu_sweeps_bwd=r["ilu_sweeps_bwd"], warm_extrap=r["warm_extrap"],
                          inner_rtol=r["inner_rtol"], gmres_m=r["gmres_m"], flux_shape=r["flux_variant"])
    wa, wb = dev(w0), dev(w0)
    assert b.batch_run(wa, max_steps=5)["n_failed"] == 0
    ref.batch_run(wb, max_steps=5)
    assert rel_max(host(wa), host(wb)) <= 1e-10


@pytest.mark.parametrize("precision", ["fp64", "mixed"])
@pytest.mark.parametrize("basis_fp32", [0, 1])
def test_device_control_and_graphs_equal_direct_launches(G, precision, basis_fp32):
    """The CLS solve runs as one CUDA graph whose while / if nodes take the
    GMRES decisions on the device (no_graphs = 0), as kernels launched one by
    one with the host reading the stop flags (1), or as per-step graph replays
    under host control (2).  Same kernels, same order: the states and iteration
    counts agree bit for bit; 1 and 2 count the same launches, and the device
    control launches one condition kernel more per GMRES cycle."""
    if precision == "fp64" and basis_fp32:
        pytest.skip("the FP32 basis belongs to the mixed mode")
    prec = G.MIXED if precision == "mixed" else G.FP64
    c = I.shock_vortex_case(40, 20)
    out, counts, cycles, work = [], [], [], []
    for mode in (0, 1, 2):
        m = G.GksMesh(c.mesh, precision=prec, warm_extrap=2, no_graphs=mode, basis_fp32=basis_fp32)
        w = dev(c.w0)
        m.profile_begin([])
        l0 = G.launch_count()
        its = [m.step(w, 2e-4)["iters"] for _ in range(6)]
        counts.append(G.launch_count() - l0)
        p = m.profile_end()
        cycles.append(p["residuals"] - 6)
        work.append((p["arnoldi"], p["arnoldi_jsum"], p["precond"], p["residuals"]))
        out.append((host(w), its))
    for q in (1, 2):
        assert np.array_equal(out[0][0], out[q][0])
        assert out[0][1] == out[q][1]
        assert work[0] == work[q]
    assert counts[1] == counts[2]
    assert cycles[0] > 0 and counts[0] == counts[1] + cycles[0]


@pytest.mark.parametrize("precision", ["fp64", "mixed"])
def test_run_graph_equals_the_host_step_loop(G, precision):
    """gks_run with graphs on is one launch of a graph whose while node the
    device ends once every case is done or max_steps loops ran (no_graphs = 0);
    with 2 the host enqueues the same steps, the solve as per-part graph
    replays, and looks at the done flags every 16 loops; with 1 every kernel is
    launched one by one.  Same kernels in the same order, the warm-start
    history rotated by the device's solve count in all three: states and run
    results agree exactly, for a run that stops at max_steps and one that
    stops at its end time.  On the max_steps run the solver work agrees too;
    1 and 2 count the same launches, and the graph adds one condition kernel
    per GMRES cycle and per loop, and one per launch.  (After an end time the
    host loop may enqueue up to 15 loops in which every case is masked, which
    change nothing; the graph stops at once.)"""
    prec = G.MIXED if precision == "mixed" else G.FP64
    c = I.shock_vortex_case(40, 20)
    res = []
    for mode in (0, 2, 1):
        m = G.GksMesh(c.mesh, precision=prec, warm_extrap=2, no_graphs=mode)
        w = dev(c.w0)
        m.profile_begin([])
        l0 = G.launch_count()
        a = m.run(w, max_steps=7)
        n = G.launch_count() - l0
        p = m.profile_end()
        tf = 3.5 * m.cfl_dt(w)
        b = m.run(w, t_final=tf, max_steps=10000)
        assert a["steps"] == 7 and b["steps"] >= 3 and abs(b["t"] - tf) <= 1e-15 * tf
        res.append((host(w), a, b, n, (p["arnoldi"], p["arnoldi_jsum"], p["precond"], p["residuals"])))
    for q in (1, 2):
        assert np.array_equal(res[0][0], res[q][0])
        assert res[0][1] == res[q][1] and res[0][2] == res[q][2] and res[0][4] == res[q][4]
    assert res[1][3] == res[2][3]
    cycles = res[0][4][3] - 7
    assert cycles > 0 and res[0][3] == res[1][3] + cycles + 7 + 1


@pytest.mark.parametrize("precision", ["fp64", "mixed"])
def test_cfl_step_as_a_graph_launch_equals_the_host_step(G, precision):
    """gks_step with the CFL step runs as one launch of the step-loop graph (one
    synchronisation); with no_graphs = 1 it takes the host path.  Same kernels:
    the states and every field of the step info agree exactly, also for a step
    taken after a run that ended the case at its end time (the step clears the
    done flag, so the solve runs)."""
    prec = G.MIXED if precision == "mixed" else G.FP64
    c = I.shock_vortex_case(40, 20)
    res = []
    for mode in (0, 1):
        m = G.GksMesh(c.mesh, precision=prec, warm_extrap=2, no_graphs=mode)
        w = dev(c.w0)
        infos = [m.step(w) for _ in range(4)]
        tf = 2.5 * infos[-1]["dt"]
        m.run(w, t_final=tf, max_steps=100)
        infos.append(m.step(w))
        res.append((host(w), infos))
    assert np.array_equal(res[0][0], res[1][0])
    for a, b in zip(res[0][1], res[1][1]):
        assert a == b
    assert min(res[0][1][-1]["iters"]) > 0 and res[0][1][-1]["dt"] > 0.0


def test_batch_run_graph_equals_the_host_step_loop(G):
    """The batched run as one graph launch and as the host loop: cases with
    their own end times finish at different loops (the graph keeps stepping the
    others under the per-case masks), and every case's state, time and step
    count agree exactly."""
    cases = [I.advection_case(12, k=2), I.shock_vortex_case(30, 15), I.advection_case(7, seed=5)]
    tf = np.array([0.004, 0.0015, 0.003])
    res = []
    for mode in (0, 2):
        b = G.GksMesh.batch([c.mesh for c in cases], precision=G.MIXED, no_graphs=mode)
        w = dev(np.ascontiguousarray(np.concatenate([c.w0 for c in cases], axis=1)))
        r = b.batch_run(w, t_final=tf, max_steps=10000)
        assert r["n_failed"] == 0 and r["n_finished"] == 3
        res.append((host(w), r))
    assert np.array_equal(res[0][0], res[1][0])
    for k in ("t", "status"):
        assert np.array_equal(res[0][1][k], res[1][1][k])
    assert res[0][1]["steps"] == res[1][1]["steps"] and res[0][1]["gmres_iters"] == res[1][1]["gmres_iters"]


@pytest.mark.parametrize("mode", [0, 1])
def test_iteration_cap_stops_solve_the_same_way(G, mode):
    """gmres_maxit below what the tolerance needs: the solve stops at the cap
    under device and host control alike, reports it (GKS_ENOCONV with the
    iterations and relative residuals of the cap), and leaves the same state."""
    c = I.shock_vortex_case(30, 15)
    res = []
    for no_graphs in (mode, 1):
        m = G.GksMesh(c.mesh, gmres_maxit=3, no_graphs=no_graphs)
        w = dev(c.w0)
        r = m.step(w, 2e-4, check=False)
        assert r["status"] == G.GKS_ENOCONV
        assert max(r["iters"]) == 3 and max(r["relres"]) > 1e-12
        res.append((host(w), r["iters"], r["relres"]))
    assert np.array_equal(res[0][0], res[1][0])
    assert res[0][1] == res[1][1] and res[0][2] == res[1][2]


def test_graphs_follow_knob_changes(G):
    """Knobs baked into the captured kernel arguments (sweeps, warm start, inner
    tolerance, restart length, flux launch shape) drop the graphs when they
    change: after the autotuner has run every candidate, the handle steps
    exactly like a fresh handle built with the knobs it picked and launching its
    kernels one by one."""
    c = I.shock_vortex_case(30, 15)
    m = G.GksMesh(c.mesh, precision=G.MIXED)
    r = m.autotune(dev(c.w0), trial_steps=1)
    ref = G.GksMesh(c.mesh, precision=G.MIXED, ilu_sweeps=r["ilu_sweeps"], ilu_sweeps_bwd=r["ilu_sweeps_bwd"],
                    warm_extrap=r["warm_extrap"], inner_rtol=r["inner_rtol"], gmres_m=r["gmres_m"],
                    flux_shape=r["flux_variant"], no_graphs=1)
    wa, wb = dev(c.w0), dev(c.w0)
    for _ in range(5):
        assert m.step(wa, 2e-4)["iters"] == ref.step(wb, 2e-4)["iters"]
    assert np.array_equal(host(wa), host(wb))


def test_profiler_classes_cover_the_step(G):
    """Every kernel class of a mixed step is timed: flux, operator, ILU,
    Gram-Schmidt, update, FP64 residual, correction and the small kernels; the
    work counters agree with the residuals and Arnoldi iterations run."""
    c = I.shock_vortex_case(40, 20)
    m = G.GksMesh(c.mesh, precision=G.MIXED, basis_fp32=1, warm_extrap=2)
    w = dev(c.w0)
    m.step(w, 2e-4)
    m.profile_begin(range(G.PROF_CLASSES))
    for _ in range(3):
        m.step(w, 2e-4)
    p = m.profile_end()
    assert len(p["n"]) == G.PROF_CLASSES == 8
    assert all(n > 0 for n in p["n"]) and all(t > 0.0 for t in p["ms"]), p
    assert p["arnoldi"] > 0 and p["precond"] == p["arnoldi"]
    # one residual at the start of each solve and one after every cycle
    assert p["residuals"] >= 2 * 3 and p["n"][G.PROF_RESID] == p["residuals"]


@pytest.mark.parametrize("bwd", [0, 1, 3])
def test_backward_sweeps_knob_reaches_tolerance(O, G, bwd):
    """ilu_sweeps_bwd: a fixed preconditioner with a different number of backward
    sweeps; the solve still meets the FP64 tolerance and the oracle's
    coefficients (1e-9) in FP64 and mixed precision."""
    c = I.shock_vortex_case(40, 20)
    ref, _, _, _ = O.OracleMesh(c.mesh).cls_solve(c.w0)
    for prec in (G.FP64, G.MIXED):
        m = G.GksMesh(c.mesh, precision=prec, ilu_sweeps=2, ilu_sweeps_bwd=bwd)
        coef, info = m.cls_reconstruct(dev(c.w0))
        assert info["converged"] == 1 and max(info["relres"]) <= 1e-12
        got = host(coef)
        for v in range(4):
            assert rel_max(got[v], ref[v]) <= 1e-9


@pytest.mark.parametrize("cls_global", [0, 1])
@pytest.mark.parametrize("precision", ["fp64", "mixed"])
def test_fused_first_ilu_pass_is_the_separate_pass(G, precision, cls_global):
    """ilu_fuse_first folds z^0 = P r into the first forward sweep, each cell
    forming its lower neighbours' z^0 with the separate pass's arithmetic and
    rounding: steps and CLS coefficients are bit-identical, with one and three
    sweeps, FP16 factors in the mixed mode and the global normal equations."""
    c = I.shock_vortex_case(40, 20)
    mixed = precision == "mixed"
    kw = dict(precision=G.MIXED if mixed else G.FP64, basis_fp32=int(mixed), ilu_fp16=int(mixed),
              cls_global=cls_global)
    for sweeps in (1, 3):
        a = G.GksMesh(c.mesh, ilu_sweeps=sweeps, ilu_fuse_first=1, **kw)
        b = G.GksMesh(c.mesh, ilu_sweeps=sweeps, ilu_fuse_first=0, **kw)
        ca, ia = a.cls_reconstruct(dev(c.w0))
        cb, ib = b.cls_reconstruct(dev(c.w0))
        assert ia["iters"] == ib["iters"] and np.array_equal(host(ca), host(cb))
        wa, wb = dev(c.w0), dev(c.w0)
        for _ in range(3):
            ra, rb = a.step(wa), b.step(wb)
            assert ra["iters"] == rb["iters"]
        assert np.array_equal(host(wa), host(wb))


@pytest.mark.parametrize("precision", ["fp64", "mixed"])
def test_sweep_pairs_are_the_single_sweeps(G, precision):
    """ilu_sweep_pairs runs two consecutive sweeps of a relation in one launch,
    each cell forming its neighbours' first-sweep values with the single
    sweep's arithmetic and rounding: CLS coefficients and steps are
    bit-identical to one sweep per launch, for 2, 3 and 4 sweeps and unequal
    forward / backward counts (FP16 factors in the mixed mode)."""
    c = I.shock_vortex_case(40, 20)
    mixed = precision == "mixed"
    kw = dict(precision=G.MIXED if mixed else G.FP64, basis_fp32=int(mixed), ilu_fp16=int(mixed))
    for sweeps, bwd in ((2, -1), (3, -1), (4, 1), (1, 2), (2, 3)):
        a = G.GksMesh(c.mesh, ilu_sweeps=sweeps, ilu_sweeps_bwd=bwd, ilu_sweep_pairs=1, **kw)
        b = G.GksMesh(c.mesh, ilu_sweeps=sweeps, ilu_sweeps_bwd=bwd, ilu_sweep_pairs=0, **kw)
        ca, ia = a.cls_reconstruct(dev(c.w0))
        cb, ib = b.cls_reconstruct(dev(c.w0))
        assert ia["iters"] == ib["iters"] and np.array_equal(host(ca), host(cb)), (sweeps, bwd)
        wa, wb = dev(c.w0), dev(c.w0)
        for _ in range(3):
            ra, rb = a.step(wa), b.step(wb)
            assert ra["iters"] == rb["iters"]
        assert np.array_equal(host(wa), host(wb)), (sweeps, bwd)


def test_fused_gram_schmidt_products_reach_the_same_solution(G, O):
    """spmv_dots forms the first Gram-Schmidt products inside the operator
    kernel (FP32 basis): a different summation order, so the iterates differ by
    rounding, but both reach the FP64 tolerance and the oracle's coefficients,
    and three steps agree to 1e-10."""
    c = I.shock_vortex_case(40, 20)
    ref, _, _, _ = O.OracleMesh(c.mesh).cls_solve(c.w0)
    out = []
    for fused in (1, 0):
        m = G.GksMesh(c.mesh, precision=G.MIXED, basis_fp32=1, spmv_dots=fused)
        coef, info = m.cls_reconstruct(dev(c.w0))
        assert info["converged"] == 1 and max(info["relres"]) <= 1e-12
        got = host(coef)
        for v in range(4):
            assert rel_max(got[v], ref[v]) <= 1e-9
        w = dev(c.w0)
        for _ in range(3):
            assert m.step(w, 1e-3)["status"] == 0
        out.append(host(w))
    assert rel_max(out[0], out[1]) <= 1e-10


@pytest.mark.parametrize("slope0_mode", [0, 1])
def test_split_flux_kernel_is_the_single_role_kernel(G, slope0_mode):
    """flux_split gives the FP64 part of the mixed flux (values, interface state,
    collision time, zeroth-order terms) and its FP32 slope-carrying part to
    different warps of a persistent block.  The arithmetic is the same as one
    thread doing both; the compiler may contract multiply-adds differently in
    the two kernels, so the states agree to rounding (1e-13 of each variable's
    magnitude after three steps, far below any mistake in the tile hand-over)
    on Dirichlet, outflow, slip and no-slip boundaries, with enough faces that
    each block takes several tiles (both buffers reused)."""
    kw = dict(precision=G.MIXED, basis_fp32=1, ilu_fp16=1, slope0_mode=slope0_mode)
    for c in (I.shock_vortex_case(200, 100), I.cavity_case(24)):
        a = G.GksMesh(c.mesh, flux_split=1, **kw)
        b = G.GksMesh(c.mesh, flux_split=0, **kw)
        wa, wb = dev(c.w0), dev(c.w0)
        for _ in range(3):
            ra, rb = a.step(wa), b.step(wb)
            assert abs(ra["dt"] - rb["dt"]) <= 1e-13 * rb["dt"]
        d = rel_max(host(wa), host(wb), axis=1)
        print(c.name, "split vs single-role kernel, max relative difference per variable:", d)
        assert np.all(d <= 1e-13), d


def test_split_flux_kernel_on_a_batch_with_finished_cases(G):
    """Per-case time steps and cases that have reached their end time (dt = 0,
    no flux) in the split kernel: the single-role kernel's states to rounding."""
    cases = [I.shock_vortex_case(30, 15), I.cavity_case(12), I.advection_case(10)]
    w0 = np.concatenate([c.w0 for c in cases], axis=1)
    out = []
    for split in (1, 0):
        b = G.GksMesh.batch([c.mesh for c in cases], precision=G.MIXED, basis_fp32=1, flux_split=split)
        w = dev(w0)
        r = b.batch_run(w, t_final=np.array([1e-3, 1e9, 2e-3]), max_steps=6)
        out.append((host(w), r))
    assert out[0][1]["n_finished"] >= 1 and out[0][1]["n_failed"] == 0
    assert out[0][1]["steps"] == out[1][1]["steps"]
    assert np.all(np.abs(out[0][1]["t"] - out[1][1]["t"]) <= 1e-13 * out[1][1]["t"])
    d = rel_max(out[0][0], out[1][0], axis=1)
    print("batch: split vs single-role kernel, max relative difference per variable:", d)
    assert np.all(d <= 1e-13), d
