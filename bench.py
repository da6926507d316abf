#!/usr/bin/env python
"""Benchmark of one explicit step of the third-order gas-kinetic scheme with
CLS reconstruction (GMRES + ILU(0) on RCM order, BGK flux at face Gauss
points, conservative update) on the 1,000,000-triangle shock-vortex workload.

    python bench.py [--gpus N] [--steps K] [--warmup W] [--impl gks|reference]

Prints one JSON line (rank 0).  `value` is triangle-steps/s with the state
resident in HBM; `e2e` is the same metric through the C ABI with the state
copied host->device and device->host every step.  With N > 1 (launched by
torch.distributed.run) every rank advances its own independent replica of the
workload (weak scaling, no data-path collective).  `--impl reference` times the
CPU oracle on the host cores on a bounded sample of the same workload.
"""
from __future__ import annotations

import argparse
import hashlib
import json
import math
import os
import statistics
import subprocess
import sys
import tempfile
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

METRIC = "triangle-steps/s"
WARM = {"prev": 0, "extrap": 1, "extrap2": 2}     # gks_config.warm_extrap
HBM_FALLBACK_GBS = 6800.0
# non-tensor pipe rates per SM and clock: FP64 2 DFMA (4 flop), FP32 128 FFMA (256 flop)
FP64_FLOP_PER_CLK_SM = 4
FP32_FLOP_PER_CLK_SM = 256
NOMINAL_SM_MHZ = 2070.0
# how the CLS solve is launched (gks_config.no_graphs): one graph per solve with
# device-side GMRES control, per-part graphs under host control (ncu cannot
# profile the kernel nodes of graphs with conditional nodes), or plain launches
FLUX_SPLIT = {"on": 1, "off": 0}
GRAPHS = {"device": 0, "host": 2, "none": 1}
# event-timed kernel classes of the library's profiler, in its class order
PROF_NAMES = ["flux", "spmv", "ilu", "orth", "update", "resid", "corr", "ctl"]

WORKLOADS = {
    "shock_vortex_1m": dict(kind="shock_vortex", nx=1000, ny=500),
    "shock_vortex_small": dict(kind="shock_vortex", nx=200, ny=100),
    "shock_vortex_400k": dict(kind="shock_vortex", nx=632, ny=316),
    "advection_20": dict(kind="advection", n=20),
    "batch_512": dict(kind="batch", n=512),
    "cavity_256": dict(kind="cavity", n=256),
    "cavity_64": dict(kind="cavity", n=64),
}


def make_case(name: str, replica: int = 0):
    from paper_1802_00704_gb300 import inputs as I
    w = WORKLOADS[name]
    if w["kind"] == "shock_vortex":
        return I.shock_vortex_case(w["nx"], w["ny"], seed=1802 + replica)
    if w["kind"] == "cavity":
        return I.cavity_case(w["n"], seed=1802 + replica)
    return I.advection_case(w["n"], seed=1802 + replica)


# the source files of each face-flux kernel a counter record describes (the
# file that defines it and the headers with its device code)
FLUX_SOURCES = {
    "mixed_flux_df": ("gks_flux_df.cu", "gks_kinetic.cuh", "gks_face.cuh", "gks_lead_df.cuh", "gks_df.cuh",
                      "gks_erfcx_coef.h"),
    "mixed_flux_ws": ("gks_flux.cu", "gks_kinetic.cuh", "gks_face.cuh"),
    "mixed_flux": ("gks_flux.cu", "gks_kinetic.cuh", "gks_face.cuh"),
    "flux": ("gks_flux.cu", "gks_kinetic.cuh", "gks_face.cuh"),
}


def source_hash(kernel: str = "mixed_flux_df") -> str:
    """Hash of the sources of a face-flux kernel (those its counter record was taken on)."""
    h = hashlib.sha256()
    csrc = os.path.join(ROOT, "paper_1802_00704_gb300", "csrc")
    for f in FLUX_SOURCES[kernel]:
        with open(os.path.join(csrc, f), "rb") as fh:
            h.update(fh.read())
    return h.hexdigest()[:16]


def measured_peaks() -> dict:
    p = os.path.join(ROOT, "MEASURED_PEAKS.json")
    if os.path.exists(p):
        with open(p) as fh:
            return json.load(fh)
    return {}


def counter_record(kernel: str):
    """ncu counters of a face-flux kernel from the committed record
    (profiles/traffic.txt: kernel source_hash dram_bytes_per_launch
    gauss_points_per_launch fp64_flop_per_gp fp32_flop_per_gp), if they were
    taken on the current kernel sources; '-' marks a counter not taken."""
    p = os.path.join(ROOT, "profiles", "traffic.txt")
    if not os.path.exists(p):
        return None
    if kernel not in FLUX_SOURCES:
        return None
    cur = source_hash(kernel)
    for line in open(p):
        parts = line.split()
        if len(parts) >= 6 and not line.startswith("#") and parts[0] == kernel and parts[1] == cur:
            num = [None if x == "-" else float(x) for x in parts[2:6]]
            return {"dram_bytes": num[0], "gauss_points": num[1], "fp64_flop_per_gp": num[2],
                    "fp32_flop_per_gp": num[3]}
    return None


def probe_peaks(dev, reps: int = 5) -> dict:
    """Measured roofs on this GPU: FP64 and FP32 multiply-add chains (the
    library's FMA probe), a streaming read and a copy of 2 GiB (larger than L2);
    best of reps launches, CUDA events on the launching stream.  Beside them the
    rates derived from the pipes' per-SM throughput, the device's SM count and
    the nominal maximum SM clock."""
    import torch

    from paper_1802_00704_gb300 import gks
    props = torch.cuda.get_device_properties(dev)
    nsm = props.multi_processor_count
    stream = torch.cuda.current_stream(dev)
    sink = torch.zeros(16 * nsm, dtype=torch.float64, device=dev)

    def best(launch):
        out = None
        for _ in range(reps + 1):
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            e0.record(stream)
            work = launch()
            e1.record(stream)
            e1.synchronize()
            ms = e0.elapsed_time(e1)
            rate = work / (ms / 1e3)
            out = rate if out is None else max(out, rate)
        return out

    fp64 = best(lambda: gks.probe_fma(True, sink, blocks_per_sm=4, iters=512)) / 1e12
    fp32 = best(lambda: gks.probe_fma(False, sink, blocks_per_sm=8, iters=8192)) / 1e12
    n = (2 << 30) // 4
    a = torch.ones(n, dtype=torch.float32, device=dev)
    b = torch.empty_like(a)
    rd = best(lambda: gks.probe_read(a, sink)) / 1e9
    cp = best(lambda: gks.probe_copy(a, b)) / 1e9
    del a, b
    clk = NOMINAL_SM_MHZ * 1e6
    return {"fp64_tflops": fp64, "fp32_tflops": fp32, "read_gbs": rd, "copy_gbs": cp, "sm_count": nsm,
            "fp64_tflops_derived": FP64_FLOP_PER_CLK_SM * nsm * clk / 1e12,
            "fp32_tflops_derived": FP32_FLOP_PER_CLK_SM * nsm * clk / 1e12,
            "how": "gks_probe_fma (8 independent FMA chains per thread, 4 resp. 8 blocks of 256 threads per SM), "
                   "gks_probe_read / gks_probe_copy (16-byte streaming loads, 2 GiB); best of 5, CUDA events; "
                   f"derived: 4 (FP64) and 256 (FP32) flop/clk/SM x {nsm} SMs x {NOMINAL_SM_MHZ:.0f} MHz"}


def flux_kernel(args, mixed: bool):
    """(record key, kernel name) of the face-flux kernel a configuration launches."""
    if mixed and args.flux_lead == "pairs":
        return "mixed_flux_df", "k_face_flux_df"
    if mixed and args.flux_split != "off":
        return "mixed_flux_ws", "k_face_flux_ws"
    return ("mixed_flux", "k_face_flux") if mixed else ("flux", "k_face_flux")


def flux_roofline(key: str, name: str, launches: int, per_launch_ms: float, gp: int, peaks: dict) -> dict:
    """Roofline object of the face-flux kernel, which the arithmetic pipes bound:
    flop per Gauss point from the ncu record of the current sources (FMA = 2),
    times the Gauss points of one launch, over the event-timed launch duration,
    against the measured rate of the busier pipe (FP64 or FP32)."""
    rec = counter_record(key)
    roof = {"kernel": name, "launches": launches, "avg_ms": per_launch_ms, "bound": "alu", "unit": "TFLOP/s"}
    cand = []
    for pipe in ("fp64", "fp32"):
        fl = rec[f"{pipe}_flop_per_gp"] if rec else None
        roof[f"{pipe}_flop_per_gauss_point"] = fl
        if fl:
            ach = fl * gp / (per_launch_ms / 1e3) / 1e12
            cand.append((ach / peaks[f"{pipe}_tflops"], pipe, ach))
    if cand:
        frac, pipe, ach = max(cand)
        roof.update({"pipe": pipe, "achieved": ach, "peak": peaks[f"{pipe}_tflops"], "frac": frac,
                     "peak_source": f"measured: {pipe.upper()} multiply-add chain probe on this GPU in this run",
                     "peak_derived": peaks[f"{pipe}_tflops_derived"],
                     "frac_of_derived": ach / peaks[f"{pipe}_tflops_derived"],
                     "other_pipes": {p: round(f, 3) for f, p, _ in cand if p != pipe}})
    else:
        roof.update({"achieved": None, "peak": None, "frac": None,
                     "note": "no ncu flop counters for the current flux sources (profiles/traffic.txt)"})
    roof["traffic"] = rec["dram_bytes"] * gp / rec["gauss_points"] if rec and rec["dram_bytes"] else None
    return roof


class ClockSampler:
    """nvidia-smi samples of SM clock and throttle reasons during the timed region."""

    FIELDS = ("clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,clocks_event_reasons.hw_slowdown,"
              "clocks_event_reasons.hw_thermal_slowdown,clocks_event_reasons.sw_thermal_slowdown,"
              "clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_id: str):
        self.tmp = tempfile.NamedTemporaryFile("w+", suffix=".csv", delete=False)
        try:
            self.proc = subprocess.Popen(["nvidia-smi", "-i", gpu_id, f"--query-gpu={self.FIELDS}",
                                          "--format=csv,noheader,nounits", "-lms", "200"],
                                         stdout=self.tmp, stderr=subprocess.DEVNULL)
        except OSError:
            self.proc = None

    def stop(self) -> dict:
        if self.proc is None:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except subprocess.TimeoutExpired:
            self.proc.kill()
        self.tmp.flush()
        self.tmp.seek(0)
        sm, smax, power, reasons = [], [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for line in self.tmp.read().splitlines():
            parts = [q.strip() for q in line.split(",")]
            if len(parts) < 8:
                continue
            try:
                sm.append(float(parts[0]))
                smax.append(float(parts[1]))
                power.append(float(parts[2]))
            except ValueError:
                continue
            for nm, val in zip(names, parts[4:8]):
                if val.lower().startswith("active"):
                    reasons.add(nm)
        os.unlink(self.tmp.name)
        return {"sm_mhz": statistics.median(sm) if sm else None, "sm_max_mhz": max(smax) if smax else None,
                "power_w_median": statistics.median(power) if power else None, "samples": len(sm),
                "reasons": sorted(reasons)}


def tri_area(nodes, tris):
    p = nodes[tris]
    return 0.5 * abs((p[:, 1, 0] - p[:, 0, 0]) * (p[:, 2, 1] - p[:, 0, 1]) -
                     (p[:, 2, 0] - p[:, 0, 0]) * (p[:, 1, 1] - p[:, 0, 1]))


def gpu_id_of(dev) -> str:
    """nvidia-smi id of a torch device (its UUID when torch exposes it)."""
    import torch
    props = torch.cuda.get_device_properties(dev)
    gid = str(dev.index)
    if getattr(props, "uuid", None) is not None:
        gid = str(props.uuid)
        gid = gid if gid.startswith("GPU-") else "GPU-" + gid
    return gid


def dist_setup():
    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("gloo")
    return world, rank, local


def barrier(world):
    if world > 1:
        import torch.distributed as dist
        dist.barrier()


def allmax(world, x: float) -> float:
    if world == 1:
        return x
    import torch
    import torch.distributed as dist
    t = torch.tensor([x], dtype=torch.float64)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def cpu_info() -> dict:
    """Model, clock and thread count of the host CPU (Linux /proc, lscpu)."""
    out = {"threads": os.cpu_count()}
    try:
        txt = subprocess.run(["lscpu"], capture_output=True, text=True, timeout=10).stdout
        for line in txt.splitlines():
            k, _, v = line.partition(":")
            k, v = k.strip(), v.strip()
            if k in ("Model name", "Architecture", "CPU max MHz", "Socket(s)", "Core(s) per socket"):
                out[k.lower().replace(" ", "_").replace("(s)", "s")] = v
    except (OSError, subprocess.SubprocessError):
        pass
    return out


def oracle_sample(steps: int, warmup: int = 0, threads: int | None = None):
    """The CPU oracle on a bounded sample of the workload: the same shock-vortex
    problem on a 200 x 100 split-quad mesh (40,000 triangles).  Returns the
    baseline record, the final state and the oracle's time steps."""
    from oracle import oracle
    oracle.build()
    c = make_case("shock_vortex_small")
    om = oracle.OracleMesh(c.mesh)
    w = c.w0.copy()
    for _ in range(warmup):
        om.step(w)
    dts = []
    t0 = time.perf_counter()
    for _ in range(steps):
        info = om.step(w)
        if info.status != 0:
            raise RuntimeError(f"oracle step status {info.status}")
        dts.append(info.dt)
    el = time.perf_counter() - t0
    cores = threads or int(os.environ.get("OMP_NUM_THREADS", os.cpu_count() or 1))
    rec = {"value": c.mesh.n_tri * steps / el, "unit": METRIC, "cores": cores, "kind": "oracle",
           "sample": f"{steps} oracle steps of the 200x100 (40,000-triangle) shock-vortex mesh, "
                     f"FP64, OpenMP over faces, sequential GMRES+ILU(0)",
           "seconds": el}
    return rec, w, dts, c


def oracle_single_thread(steps: int) -> dict:
    """The oracle with one OpenMP thread on the same sample (a child process,
    since the thread count is fixed when OpenMP starts)."""
    code = ("import bench, json; r, _, _, _ = bench.oracle_sample(%d, threads=1); r.pop('seconds'); "
            "print(json.dumps(r))" % steps)
    env = dict(os.environ, OMP_NUM_THREADS="1")
    r = subprocess.run([sys.executable, "-c", code], capture_output=True, text=True, cwd=ROOT, env=env, timeout=900)
    if r.returncode != 0:
        return {"error": r.stderr.strip().splitlines()[-1] if r.stderr.strip() else "failed"}
    return json.loads(r.stdout.strip().splitlines()[-1])


def errors_vs_oracle(case, w_oracle, dts, dev, mixed_kw: dict) -> dict:
    """The GPU path (mixed and FP64) advanced by the oracle's time steps from
    the same initial state: relative L1 (sum |Omega| |q - q_o| / sum |Omega| |q_o|)
    and relative max (max |q - q_o| / max |q_o|) per conserved variable."""
    import numpy as np
    import torch

    from paper_1802_00704_gb300 import gks
    area = tri_area(case.mesh.nodes, case.mesh.tris)
    out = {}
    for name, kw in (("mixed", mixed_kw), ("fp64", {})):
        m = gks.GksMesh(case.mesh, **kw)
        w = torch.from_numpy(case.w0.copy()).to(dev)
        for dt in dts:
            if m.step(w, dt)["status"] != 0:
                raise RuntimeError("GPU step failed on the oracle sample")
        g = w.cpu().numpy()
        l1 = np.sum(area * np.abs(g - w_oracle), axis=1) / np.sum(area * np.abs(w_oracle), axis=1)
        mx = np.max(np.abs(g - w_oracle), axis=1) / np.max(np.abs(w_oracle), axis=1)
        out[name] = {"rel_l1": [float(x) for x in l1], "rel_max": [float(x) for x in mx]}
        del m
    out["sample"] = (f"{len(dts)} steps of the 200x100 (40,000-triangle) shock-vortex mesh with the oracle's "
                     "time steps; variables rho, rho u, rho v, E")
    return out


def class_bytes(cls: str, prof: dict, T: int, F: int, steps: int, sweeps: int, exact: bool, mixed: bool,
                basis32: bool, ilu16: bool = False, sweeps_bwd: int = -1, fuse_first: bool = True,
                pairs: bool = False, fused_dots: bool = False) -> float:
    """Algorithmic DRAM bytes moved by one kernel class over the timed region,
    from the solver's work counters (Arnoldi iterations n, sum of j + 1 over
    them, preconditioner applications).  Per cell: operator = diagonal block 15
    values + 3 off-diagonal blocks of 3 values + 3 int32 neighbours; ILU pivot
    inverse 25 values; a Krylov or work vector 20 values; a neighbour reads the
    first 2 of the 5 unknowns of each variable (8 values, counted once).  Sizes:
    sM operator/factor values, sZ preconditioner vectors (8 FP64 path, 4 mixed),
    sB Krylov basis (8, or 4 with the FP32-stored basis), sP the ILU factors (sM,
    or 2 with FP16 copies).  With the block-diagonal pass folded into the first
    forward sweep the neighbours' z^0 comes from their own factors and right-hand
    sides, already counted as those cells' reads; with backward sweep pairs
    likewise the neighbours' first-sweep values."""
    sM = 4 if mixed else 8
    sZ = 4 if mixed else 8
    sB = 4 if basis32 else 8
    sP = 2 if ilu16 else sM
    n, jsum = prof["arnoldi"], prof["arnoldi_jsum"]
    op = sM * (15 + 9) + 12
    if cls == "orth":
        # per iteration j: dots read V_0..V_j and w, the update reads them again and
        # writes w: (2 j + 5) vectors; FP64 mode runs the pair twice (CGS2); with the
        # products formed in the operator kernel only the update's (j + 3) remain
        vecs = (jsum + 2 * n) if fused_dots else (2 * jsum + 3 * n)
        return T * 20 * sB * vecs * (1 if mixed else 2)
    if cls == "spmv":                   # y = K z: z (own + neighbour values), operator, y (basis)
        # (+ V_0..V_j when the operator kernel also forms the Gram-Schmidt products)
        return T * ((op + 20 * sZ + 20 * sB) * n + (20 * sB * jsum if fused_dots else 0))
    if cls == "ilu":
        pc = prof["precond"]
        if exact:
            fwd = 20 * sB + 8 * sZ + sP * (25 + 9) + 12 + 20 * sZ
            bwd = 20 * sZ + 8 * sZ + sP * (25 + 9) + 12 + 20 * sZ
            return T * (fwd + bwd) * pc
        first = 20 * sB + sP * 25 + 20 * sZ
        fwd = 20 * sB + 8 * sZ + sP * (25 + 9) + 12 + 20 * sZ
        bwd = 20 * sZ + 8 * sZ + sP * (25 + 9) + 12 + 20 * sZ
        nbwd = sweeps if sweeps_bwd < 0 else sweeps_bwd
        # with sweep pairs a launch covers two sweeps and moves a single sweep's
        # bytes (the neighbours' first-sweep inputs are other cells' reads)
        nbl = (nbwd // 2 + nbwd % 2) if pairs else nbwd
        if fuse_first and sweeps > 0:
            return T * ((fwd - 8 * sZ) + (sweeps - 1) * fwd + nbl * bwd) * pc
        return T * (first + sweeps * fwd + nbl * bwd) * pc
    if cls == "update":                 # w in/out, 1/|Omega|, 3 face slots; each face flux once
        return (T * (8 * 8 + 8 + 12) + F * 4 * 8) * steps
    if cls == "resid":                  # FP64 b - K x: x (the neighbours' entries counted once), operator, b, r
        return T * (8 * (15 + 9) + 12 + 20 * 8 + 20 * 8 + 20 * sB) * prof["residuals"]
    if cls == "corr":                   # x += Z y: the cycle's Z vectors, x read and written (FP64)
        cycles = max(prof["residuals"] - steps, 0)
        return T * (20 * sZ * n + 20 * 8 * 2 * cycles)
    raise KeyError(cls)


def timed_leg(args, case, precision: str, world: int, dev, sample_clocks: bool):
    """W warm-up steps, then K timed steps of the step on the resident state."""
    import torch

    from paper_1802_00704_gb300 import gks
    exact = args.precond == "exact"
    mixed = precision == "mixed"
    m = gks.GksMesh(case.mesh, precond=gks.PC_ILU_EXACT if exact else gks.PC_ILU_SWEEP, ilu_sweeps=args.sweeps,
                    precision=gks.MIXED if mixed else gks.FP64, basis_fp32=int(mixed and args.basis == "fp32"),
                    limiter=int(args.limiter), warm_extrap=WARM[args.warm], no_graphs=GRAPHS[args.graphs],
                    ilu_fp16=int(mixed and args.ilu16 == "on"), ilu_fuse_first=int(args.ilu_fuse == "on"),
                    flux_split=FLUX_SPLIT[args.flux_split], gmres_m=args.gmres_m,
                    flux_lead=int(args.flux_lead == "pairs"), ilu_sweep_pairs=int(args.sweep_pairs == "on"),
                    spmv_dots=int(args.spmv_dots == "on"))
    w = torch.from_numpy(case.w0.copy()).to(dev)
    stream = torch.cuda.current_stream()
    tune = m.autotune(w, trial_steps=2) if args.tune else None
    for _ in range(args.warmup):
        m.run(w, max_steps=1)
    torch.cuda.synchronize()
    sampler = None
    if sample_clocks:
        sampler = ClockSampler(gpu_id_of(dev))
        time.sleep(0.3)
    barrier(world)
    torch.cuda.synchronize()
    ev0, ev1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    l0 = gks.launch_count()
    ev0.record(stream)
    info = m.run(w, max_steps=args.steps)
    ev1.record(stream)
    torch.cuda.synchronize()
    launches = gks.launch_count() - l0
    barrier(world)
    clocks = sampler.stop() if sampler else None
    ms = allmax(world, ev0.elapsed_time(ev1))
    # a second pass of K steps with CUDA events around each kernel class (the
    # events would perturb the timed pass) for the per-class times and work counts
    m.profile_begin(range(gks.PROF_CLASSES))
    m.run(w, max_steps=args.steps)
    torch.cuda.synchronize()
    prof = m.profile_end()
    return {"mesh": m, "w": w, "info": info, "prof": prof, "launches": launches, "clocks": clocks, "ms": ms,
            "stats": m.stats(), "tune": tune,
            "knobs": {"ilu_sweeps": m.cfg.ilu_sweeps, "ilu_sweeps_bwd": m.cfg.ilu_sweeps_bwd,
                      "ilu_fuse_first": m.cfg.ilu_fuse_first, "warm_extrap": m.cfg.warm_extrap,
                      "inner_rtol": m.cfg.inner_rtol, "gmres_m": m.cfg.gmres_m,
                      "ilu_sweep_pairs": m.cfg.ilu_sweep_pairs, "spmv_dots": m.cfg.spmv_dots,
                      "flux_shape": m.cfg.flux_shape}}


def run_gks(args, world, rank, local):
    import numpy as np
    import torch

    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)
    case = make_case(args.workload, replica=rank)
    T, F = case.mesh.n_tri, case.mesh.n_face
    exact = args.precond == "exact"
    mixed = args.precision == "mixed"

    main = timed_leg(args, case, args.precision, world, dev, sample_clocks=True)
    value = world * T * args.steps / (main["ms"] / 1e3)

    # end to end through the C ABI with host buffers (pinned), every step
    m = main["mesh"]
    w_host = torch.from_numpy(case.w0.copy()).pin_memory()
    w_dev = torch.empty((4, T), dtype=torch.float64, device=dev)
    barrier(world)
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    for _ in range(args.steps):
        w_dev.copy_(w_host, non_blocking=True)
        m.step(w_dev)
        w_host.copy_(w_dev, non_blocking=True)
    torch.cuda.synchronize()
    e2e_s = allmax(world, time.perf_counter() - t0)
    e2e_value = world * T * args.steps / e2e_s
    bytes_state = 4 * T * 8

    # per-class device time (CUDA events on the launching stream) against each class's roof
    prof, info = main["prof"], main["info"]
    names = PROF_NAMES
    peaks = probe_peaks(dev)
    hbm_peak = measured_peaks().get("hbm_gbs")
    hbm_src = "measured" if hbm_peak else "fallback"
    hbm_peak = hbm_peak or HBM_FALLBACK_GBS
    basis32 = mixed and args.basis == "fp32"
    classes = {}
    for q, nm in enumerate(names):
        ms_c = prof["ms"][q]
        ent = {"ms": round(ms_c, 3), "launch_groups": prof["n"][q]}
        if nm not in ("flux", "ctl") and ms_c > 0:
            by = class_bytes(nm, prof, T, F, args.steps, main["knobs"]["ilu_sweeps"], exact, mixed, basis32,
                             mixed and args.ilu16 == "on", main["knobs"]["ilu_sweeps_bwd"],
                             bool(main["knobs"]["ilu_fuse_first"]), bool(main["knobs"]["ilu_sweep_pairs"]),
                             bool(main["knobs"]["spmv_dots"]) and basis32)
            gbs = by / (ms_c / 1e3) / 1e9
            ent.update({"bytes": by, "gbs": round(gbs, 1), "frac": round(gbs / hbm_peak, 3)})
        classes[nm] = ent
    # the dominant kernel is the face-flux kernel (one launch per step): ALU-bound
    q = names.index("flux")
    per_launch_ms = prof["ms"][q] / max(prof["n"][q], 1)
    key, kname = flux_kernel(args, mixed)
    roof = flux_roofline(key, kname, prof["n"][q], per_launch_ms, 2 * F, peaks)
    roof["hbm_peak"] = {"gbs": hbm_peak, "source": hbm_src, "probe_read_gbs": round(peaks["read_gbs"], 1),
                        "probe_copy_gbs": round(peaks["copy_gbs"], 1)}
    roof["peaks"] = peaks
    roof["classes"] = classes
    roof["work"] = {"arnoldi_per_step": prof["arnoldi"] / args.steps,
                    "mean_j": (prof["arnoldi_jsum"] - prof["arnoldi"]) / max(prof["arnoldi"], 1),
                    "precond_per_step": prof["precond"] / args.steps,
                    "fp64_residuals_per_step": prof["residuals"] / args.steps}
    st = main["stats"]

    out = {
        "metric": METRIC, "value": value, "unit": METRIC, "n_gpus": world, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": main["ms"] / args.steps, "higher_is_better": True, "scaling": "weak",
        "vs_baseline": None, "dtype": "f32+f64 (mixed)" if mixed else "f64", "data": "synthetic",
        "config": {"workload": f"shock-vortex {case.mesh.nx}x{case.mesh.ny} split quads, {T} triangles, "
                               f"{F} faces, GMRES({main['knobs']['gmres_m']}) rtol 1e-12",
                   "n_tri": T, "n_face": F, "precision": args.precision,
                   "krylov_basis": "fp32" if basis32 else "fp64", "limiter": bool(args.limiter),
                   "solve_graphs": args.graphs, "ilu_factors": "fp16" if mixed and args.ilu16 == "on" else None,
                   "warm_start": args.warm, "autotuned": bool(args.tune), "knobs": main["knobs"],
                   "precond": ("ilu0_rcm_exact" if exact else f"ilu0_rcm_sweep{main['knobs']['ilu_sweeps']}"),
                   "l2": f"inputs larger than L2: {st['device_bytes'] / 2**30:.1f} GiB resident per replica",
                   "parallelism": "replicas" if world > 1 else "single GPU",
                   "gmres_iters_per_step": info["gmres_iters"] / max(info["steps"], 1),
                   "levels_lower": st["levels_lower"], "levels_upper": st["levels_upper"]},
        "roofline": roof,
        "e2e": {"value": e2e_value, "unit": METRIC, "h2d_bytes_per_step": bytes_state,
                "d2h_bytes_per_step": bytes_state},
        "gpu_launches": main["launches"],
        "clocks": main["clocks"],
    }
    if mixed and not args.no_compare:
        # the plain FP64 path on the same GPU, same steps, and the distance between the two states
        ref = timed_leg(args, case, "fp64", world, dev, sample_clocks=False)
        wm, wf = main["w"].cpu().numpy(), ref["w"].cpu().numpy()
        area = tri_area(case.mesh.nodes, case.mesh.tris)
        l1 = np.sum(area * np.abs(wm - wf), axis=1) / np.sum(area * np.abs(wf), axis=1)
        out["fp64"] = {"value": world * T * args.steps / (ref["ms"] / 1e3), "ms_per_step": ref["ms"] / args.steps,
                       "gmres_iters_per_step": ref["info"]["gmres_iters"] / max(ref["info"]["steps"], 1),
                       "class_ms": {nm: round(ref["prof"]["ms"][q], 3) for q, nm in enumerate(names)},
                       "arnoldi_per_step": ref["prof"]["arnoldi"] / args.steps, "knobs": ref["knobs"]}
        out["mixed_vs_fp64_rel_l1"] = [float(x) for x in l1]
        out["speedup_vs_fp64"] = value / out["fp64"]["value"]
    if rank == 0 and world == 1 and not args.no_cpu_baseline:
        cb, w_o, dts, small = oracle_sample(args.cpu_steps)
        cb.pop("seconds", None)
        cb["cpu"] = cpu_info()
        st1 = oracle_single_thread(1)
        cb["single_thread"] = {k: st1[k] for k in ("value", "cores", "error") if k in st1}
        cb["single_thread"]["sample"] = "1 oracle step of the same mesh, OMP_NUM_THREADS=1"
        out["cpu_baseline"] = cb
        if mixed:
            mkw = gks_mixed_kw(args)
            mkw.update(main["knobs"])
            out["error_vs_oracle"] = errors_vs_oracle(small, w_o, dts, dev, mkw)
    if rank == 0:
        print(json.dumps(out), flush=True)


def gks_mixed_kw(args) -> dict:
    """Configuration of the benchmarked mixed path (as timed_leg builds it)."""
    from paper_1802_00704_gb300 import gks
    return dict(precision=gks.MIXED, basis_fp32=int(args.basis == "fp32"), ilu_sweeps=args.sweeps,
                ilu_fp16=int(args.ilu16 == "on"), ilu_fuse_first=int(args.ilu_fuse == "on"),
                flux_split=FLUX_SPLIT[args.flux_split], warm_extrap=WARM[args.warm],
                flux_lead=int(args.flux_lead == "pairs"))


def oracle_batch_sample(cases, steps: int):
    """The CPU oracle (robust limiter) on the six smallest cases of the batch."""
    from oracle import oracle
    oracle.build()
    small = sorted(cases, key=lambda c: c.mesh.n_tri)[:6]
    t0, tri = time.perf_counter(), 0
    for c in small:
        om = oracle.OracleMesh(c.mesh, limiter=2)
        w = c.w0.copy()
        for _ in range(steps):
            if om.step(w).status != 0:
                raise RuntimeError("oracle step failed")
        tri += c.mesh.n_tri * steps
    el = time.perf_counter() - t0
    cores = int(os.environ.get("OMP_NUM_THREADS", os.cpu_count() or 1))
    return {"value": tri / el, "unit": METRIC, "cores": cores, "kind": "oracle",
            "sample": f"{steps} oracle steps (robust limiter) of each of the 6 smallest cases of the batch "
                      f"({sum(c.mesh.n_tri for c in small)} triangles), FP64"}


def run_batch(args, world, rank, local):
    """Config 5: 512 independent cases (log-uniform 1e3-2e5 triangles) in one
    handle, mixed precision, robust limiter, every kernel covering all cases."""
    import numpy as np
    import torch

    from paper_1802_00704_gb300 import gks
    from paper_1802_00704_gb300 import inputs as I
    cases = I.batch_cases(WORKLOADS[args.workload]["n"], workers=min(16, os.cpu_count() or 1))
    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)
    T = sum(c.mesh.n_tri for c in cases)
    F = sum(c.mesh.n_face for c in cases)
    w0 = np.ascontiguousarray(np.concatenate([c.w0 for c in cases], axis=1))
    mixed = args.precision == "mixed"

    def leg(prec_mixed: bool, clocks: bool):
        b = gks.GksMesh.batch([c.mesh for c in cases], precision=gks.MIXED if prec_mixed else gks.FP64,
                              limiter=2, gmres_m=12, warm_extrap=WARM[args.warm],
                              basis_fp32=int(prec_mixed and args.basis == "fp32"), no_graphs=GRAPHS[args.graphs],
                              ilu_fp16=int(prec_mixed and args.ilu16 == "on"),
                              ilu_fuse_first=int(args.ilu_fuse == "on"),
                              flux_split=FLUX_SPLIT[args.flux_split])
        w = torch.from_numpy(w0.copy()).to(dev)
        tune = b.autotune(w, trial_steps=1) if args.tune else None
        r = b.batch_run(w, max_steps=args.warmup)
        if r["n_failed"]:
            print(f"warning: {r['n_failed']} cases failed in the warm-up", file=sys.stderr)
        torch.cuda.synchronize()
        sampler = ClockSampler(gpu_id_of(dev)) if clocks else None
        if sampler:
            time.sleep(0.3)
        barrier(world)
        torch.cuda.synchronize()
        ev0, ev1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        l0 = gks.launch_count()
        ev0.record(torch.cuda.current_stream())
        r = b.batch_run(w, max_steps=args.steps)
        ev1.record(torch.cuda.current_stream())
        torch.cuda.synchronize()
        launches = gks.launch_count() - l0
        barrier(world)
        ck = sampler.stop() if sampler else None
        ms = allmax(world, ev0.elapsed_time(ev1))
        b.profile_begin(range(gks.PROF_CLASSES))
        b.batch_run(w, max_steps=args.steps)
        torch.cuda.synchronize()
        prof = b.profile_end()
        return b, w, r, prof, launches, ck, ms, tune

    b, w, r, prof, launches, clocks, ms, tune = leg(mixed, True)
    value = world * T * args.steps / (ms / 1e3)
    # end to end: state copied host -> device and back every step
    w_host = torch.from_numpy(w0.copy()).pin_memory()
    w_dev = torch.empty_like(w)
    barrier(world)
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    for _ in range(args.steps):
        w_dev.copy_(w_host, non_blocking=True)
        b.batch_run(w_dev, max_steps=1)
        w_host.copy_(w_dev, non_blocking=True)
    torch.cuda.synchronize()
    e2e_value = world * T * args.steps / allmax(world, time.perf_counter() - t0)
    knobs = {"ilu_sweeps": b.cfg.ilu_sweeps, "ilu_sweeps_bwd": b.cfg.ilu_sweeps_bwd,
             "ilu_fuse_first": b.cfg.ilu_fuse_first, "warm_extrap": b.cfg.warm_extrap,
             "inner_rtol": b.cfg.inner_rtol, "gmres_m": b.cfg.gmres_m, "ilu_sweep_pairs": b.cfg.ilu_sweep_pairs,
             "spmv_dots": b.cfg.spmv_dots}
    names = PROF_NAMES
    hbm_peak = measured_peaks().get("hbm_gbs") or HBM_FALLBACK_GBS
    classes = {}
    for q, nm in enumerate(names):
        ent = {"ms": round(prof["ms"][q], 3), "launch_groups": prof["n"][q]}
        if nm not in ("flux", "ctl") and prof["ms"][q] > 0:
            by = class_bytes(nm, prof, T, F, args.steps, knobs["ilu_sweeps"], False, mixed,
                             mixed and args.basis == "fp32", mixed and args.ilu16 == "on", knobs["ilu_sweeps_bwd"],
                             bool(knobs["ilu_fuse_first"]), bool(knobs["ilu_sweep_pairs"]),
                             bool(knobs["spmv_dots"]) and mixed and args.basis == "fp32")
            gbs = by / (prof["ms"][q] / 1e3) / 1e9
            ent.update({"bytes": by, "gbs": round(gbs, 1), "frac": round(gbs / hbm_peak, 3)})
        classes[nm] = ent
    per_launch_ms = prof["ms"][0] / max(prof["n"][0], 1)
    key, kname = flux_kernel(args, mixed)
    roof = flux_roofline(key, kname, prof["n"][0], per_launch_ms, 2 * F, probe_peaks(dev))
    roof["classes"] = classes
    roof["work"] = {"arnoldi_per_step": prof["arnoldi"] / args.steps,
                    "mean_j": (prof["arnoldi_jsum"] - prof["arnoldi"]) / max(prof["arnoldi"], 1)}
    wm = w.cpu().numpy()
    stat = r["status"]
    out = {
        "metric": METRIC, "value": value, "unit": METRIC, "n_gpus": world, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": ms / args.steps, "higher_is_better": True, "scaling": "weak",
        "vs_baseline": None, "dtype": "f32+f64 (mixed)" if mixed else "f64", "data": "synthetic",
        "config": {"workload": f"batch of {len(cases)} cases (log-uniform 1e3-2e5 triangles; advection / "
                               f"Riemann strips), {T} triangles, {F} faces, robust limiter, GMRES({knobs['gmres_m']}) rtol 1e-12",
                   "n_tri": T, "n_face": F, "n_cases": len(cases), "precision": args.precision,
                   "krylov_basis": "fp32" if mixed and args.basis == "fp32" else "fp64",
                   "autotuned": bool(args.tune), "knobs": knobs, "failed_cases": int(np.sum(stat != 0)),
                   "l2": "inputs larger than L2", "parallelism": "replicas" if world > 1 else "single GPU"},
        "roofline": roof,
        "e2e": {"value": e2e_value, "unit": METRIC, "h2d_bytes_per_step": 4 * T * 8, "d2h_bytes_per_step": 4 * T * 8},
        "gpu_launches": launches,
        "clocks": clocks,
    }
    del b
    if mixed and not args.no_compare:
        bf, wf, rf, proff, _, _, msf, _ = leg(False, False)
        wfh = wf.cpu().numpy()
        area = np.concatenate([tri_area(c.mesh.nodes, c.mesh.tris) for c in cases])
        l1 = np.sum(area * np.abs(wm - wfh), axis=1) / np.sum(area * np.abs(wfh), axis=1)
        out["fp64"] = {"value": world * T * args.steps / (msf / 1e3), "ms_per_step": msf / args.steps,
                       "class_ms": {nm: round(proff["ms"][q], 3) for q, nm in enumerate(names)}}
        out["mixed_vs_fp64_rel_l1"] = [float(x) for x in l1]
        out["speedup_vs_fp64"] = value / out["fp64"]["value"]
        del bf
    if rank == 0 and world == 1 and not args.no_cpu_baseline:
        out["cpu_baseline"] = oracle_batch_sample(cases, args.cpu_steps)
    if rank == 0:
        print(json.dumps(out), flush=True)


def run_cavity(args, world, rank, local):
    """Config 3: the viscous lid-driven cavity (isothermal no-slip walls, lid
    Mach 0.15, Re 1000, Pr 0.72) on 256 x 256 split quads (131,072 triangles),
    mixed and FP64, for a bounded number of steps (reaching the steady residual
    1e-8 takes millions of explicit steps): triangle-steps/s of each, the
    steady-residual history of the run control's rule (max over variables of
    sqrt(sum |Omega| (w^{n+1} - w^n)^2) / dt, relative to the first step), and
    the distance between the two paths' states."""
    import numpy as np
    import torch

    from paper_1802_00704_gb300 import gks
    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)
    case = make_case(args.workload, replica=rank)
    T, F = case.mesh.n_tri, case.mesh.n_face
    pr = case.meta["prandtl"]
    area = torch.from_numpy(tri_area(case.mesh.nodes, case.mesh.tris)).to(dev)

    def leg(mixed: bool, clocks: bool, flux_lead=None):
        kw = gks_mixed_kw(args) if mixed else {}
        if flux_lead is not None:
            kw["flux_lead"] = flux_lead
        m = gks.GksMesh(case.mesh, mu=case.mu, prandtl=pr, **kw)
        w = torch.from_numpy(case.w0.copy()).to(dev)
        tune = m.autotune(w, trial_steps=2) if args.tune else None
        w.copy_(torch.from_numpy(case.w0))
        m.reset_warm_start()
        # residual history from the initial state (every step, host-side rule)
        hist, r0 = [], None
        for q in range(args.history):
            w_old = w.clone()
            info = m.run(w, max_steps=1)
            r = max(float(torch.sqrt(torch.sum(area * (w[v] - w_old[v]) ** 2))) / info["last_dt"]
                    for v in range(4))
            r0 = r if r0 is None else r0
            hist.append(r / r0)
        for _ in range(args.warmup):
            m.run(w, max_steps=1)
        torch.cuda.synchronize()
        sampler = ClockSampler(gpu_id_of(dev)) if clocks else None
        if sampler:
            time.sleep(0.3)
        barrier(world)
        torch.cuda.synchronize()
        ev0, ev1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        l0 = gks.launch_count()
        ev0.record(torch.cuda.current_stream())
        info = m.run(w, max_steps=args.steps)
        ev1.record(torch.cuda.current_stream())
        torch.cuda.synchronize()
        launches = gks.launch_count() - l0
        barrier(world)
        ck = sampler.stop() if sampler else None
        ms = allmax(world, ev0.elapsed_time(ev1))
        return {"m": m, "w": w, "ms": ms, "info": info, "hist": hist, "launches": launches, "clocks": ck,
                "knobs": {"ilu_sweeps": m.cfg.ilu_sweeps, "warm_extrap": m.cfg.warm_extrap,
                          "inner_rtol": m.cfg.inner_rtol, "gmres_m": m.cfg.gmres_m}}

    mixed = args.precision == "mixed"
    a = leg(mixed, True)
    value = world * T * args.steps / (a["ms"] / 1e3)
    out = {"metric": METRIC, "value": value, "unit": METRIC, "n_gpus": world, "steps": args.steps,
           "warmup": args.warmup, "ms_per_step": a["ms"] / args.steps, "higher_is_better": True, "scaling": "weak",
           "vs_baseline": None, "dtype": "f32+f64 (mixed)" if mixed else "f64", "data": "synthetic",
           "config": {"workload": f"lid-driven cavity {case.mesh.nx}x{case.mesh.ny} split quads, {T} triangles, "
                                  f"Re {case.meta['re']:.0f}, lid Mach 0.15, Pr {pr}, isothermal no-slip walls",
                      "n_tri": T, "n_face": F, "precision": args.precision, "knobs": a["knobs"],
                      "l2": "inputs smaller than L2 (the Krylov basis is not)",
                      "parallelism": "replicas" if world > 1 else "single GPU"},
           "steady_residual": {"rule": "max_v sqrt(sum |Omega| dw_v^2) / dt relative to the first step",
                               "history_every_step": [round(x, 6) for x in a["hist"]],
                               "after_timed_steps_steps": int(a["info"]["steps"]) + args.history + args.warmup},
           "gpu_launches": a["launches"], "clocks": a["clocks"]}
    if mixed and not args.no_compare:
        b = leg(False, False)
        wm, wf = a["w"].cpu().numpy(), b["w"].cpu().numpy()
        ar = tri_area(case.mesh.nodes, case.mesh.tris)
        l1 = np.sum(ar * np.abs(wm - wf), axis=1) / np.sum(ar * np.abs(wf), axis=1)
        out["fp64"] = {"value": world * T * args.steps / (b["ms"] / 1e3), "ms_per_step": b["ms"] / args.steps}
        out["mixed_vs_fp64_rel_l1"] = [float(x) for x in l1]
        out["speedup_vs_fp64"] = value / out["fp64"]["value"]
        out["steady_residual"]["history_every_step_fp64"] = [round(x, 6) for x in b["hist"]]
        # the mixed solver with the FP64 path's flux kernel (flux_lead = 2): the
        # viscous stress no longer carried in FP32
        c2 = leg(True, False, flux_lead=2)
        l1c = np.sum(ar * np.abs(c2["w"].cpu().numpy() - wf), axis=1) / np.sum(ar * np.abs(wf), axis=1)
        out["mixed_fp64_flux"] = {"value": world * T * args.steps / (c2["ms"] / 1e3),
                                  "ms_per_step": c2["ms"] / args.steps, "knobs": c2["knobs"],
                                  "rel_l1_vs_fp64": [float(x) for x in l1c]}
    if rank == 0:
        print(json.dumps(out), flush=True)


def run_reference(args, world, rank):
    if rank != 0:
        return
    cb, _, _, _ = oracle_sample(args.steps, warmup=args.warmup)
    secs = cb.pop("seconds")
    cb["cpu"] = cpu_info()
    out = {"impl": "reference", "metric": METRIC, "value": cb["value"], "unit": METRIC, "n_gpus": world,
           "steps": args.steps, "warmup": args.warmup, "ms_per_step": 1e3 * secs / args.steps,
           "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
           "config": {"workload": "shock-vortex, CPU oracle on a 200x100 (40,000-triangle) sample of the "
                                  "1000x500 workload", "n_tri": 40000},
           "cpu_baseline": cb,
           "e2e": {"value": cb["value"], "unit": METRIC, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(out), flush=True)


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=20)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="gks", choices=["gks", "reference"])
    ap.add_argument("--workload", default="shock_vortex_1m", choices=sorted(WORKLOADS))
    ap.add_argument("--precond", default="sweep", choices=["sweep", "exact"])
    ap.add_argument("--precision", default="mixed", choices=["mixed", "fp64"])
    ap.add_argument("--no-compare", action="store_true", help="skip the FP64 comparison leg")
    ap.add_argument("--sweeps", type=int, default=2)
    ap.add_argument("--basis", default="fp32", choices=["fp32", "fp64"],
                    help="Krylov basis of the mixed path's inner cycles: FP32 (FP32 Gram-Schmidt arithmetic, "
                         "FP64 sums across threads) or FP64")
    ap.add_argument("--limiter", action="store_true", help="shock detector + DWBAP limiter on")
    ap.add_argument("--ilu16", default="on", choices=["on", "off"],
                    help="mixed path: FP16 copies of the ILU(0) factors for the FP32 preconditioner")
    ap.add_argument("--flux-split", default="on", choices=sorted(FLUX_SPLIT),
                    help="mixed path: FP64 and FP32 parts of the flux in different warps")
    ap.add_argument("--gmres-m", type=int, default=30, help="GMRES restart length (the tuner may pick a shorter one)")
    ap.add_argument("--flux-lead", default="pairs", choices=["pairs", "fp64"],
                    help="mixed path: the flux's FP64-accuracy part in double-FP32 pairs (default) or in FP64")
    ap.add_argument("--spmv-dots", default="on", choices=["on", "off"],
                    help="FP32 basis: the operator kernel also forms the Gram-Schmidt products")
    ap.add_argument("--sweep-pairs", default="on", choices=["on", "off"],
                    help="two ILU sweeps of a relation per launch (same results)")
    ap.add_argument("--ilu-fuse", default="on", choices=["on", "off"],
                    help="fold the block-diagonal ILU pass into the first forward sweep")
    ap.add_argument("--graphs", default="device", choices=sorted(GRAPHS),
                    help="CLS solve launch: device-controlled graph (default), per-part graphs, plain launches")
    ap.add_argument("--no-tune", dest="tune", action="store_false",
                    help="skip the autotuner (ilu_sweeps, warm start, inner tolerance) before the warm-up")
    ap.add_argument("--warm", default="extrap", choices=sorted(WARM),
                    help="CLS initial guess: previous solution, or its linear / quadratic extrapolation")
    ap.add_argument("--cpu-steps", type=int, default=3)
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--history", type=int, default=50,
                    help="cavity workloads: steps of steady-residual history before the warm-up")
    args = ap.parse_args()
    if args.warmup < 3 and args.impl == "gks":
        print("warning: fewer than 3 warm-up steps", file=sys.stderr)
    world, rank, local = dist_setup()
    if args.impl == "reference":
        run_reference(args, world, rank)
    elif WORKLOADS[args.workload]["kind"] == "batch":
        run_batch(args, world, rank, local)
    elif WORKLOADS[args.workload]["kind"] == "cavity":
        run_cavity(args, world, rank, local)
    else:
        run_gks(args, world, rank, local)
    if world > 1:
        import torch.distributed as dist
        dist.destroy_process_group()


if __name__ == "__main__":
    main()
