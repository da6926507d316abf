"""Host logic of the measurement harness (bench.py), no GPU: the algorithmic
byte model of the solver's kernel classes (the per-cell figures the roofline
fractions divide by), the profiler class order shared with the library, the
option maps, and the committed traffic record's format."""
import os
import re

import pytest

import bench
from paper_1802_00704_gb300 import gks


def _prof(n=6, jsum=12, precond=6, residuals=3):
    return {"arnoldi": n, "arnoldi_jsum": jsum, "precond": precond, "residuals": residuals}


def test_profiler_classes_match_the_library():
    assert len(bench.PROF_NAMES) == gks.PROF_CLASSES
    order = [gks.PROF_FLUX, gks.PROF_SPMV, gks.PROF_ILU, gks.PROF_ORTH, gks.PROF_UPDATE, gks.PROF_RESID,
             gks.PROF_CORR, gks.PROF_CTL]
    assert [bench.PROF_NAMES[q] for q in order] == ["flux", "spmv", "ilu", "orth", "update", "resid", "corr", "ctl"]


def test_ilu_bytes_per_application():
    """Per cell and application (FP32 basis and vectors, FP16 factors, 2 + 2
    sweeps): separate block-diagonal pass 210 B, each forward or backward sweep
    272 B; with the pass folded into the first forward sweep that sweep moves
    240 B and the pass is gone (1,056 against 1,298 B: 19 % fewer)."""
    T, pc = 1000, 5
    p = _prof(precond=pc)
    args = dict(T=T, F=0, steps=1, sweeps=2, exact=False, mixed=True, basis32=True, ilu16=True, sweeps_bwd=-1)
    assert bench.class_bytes("ilu", p, fuse_first=False, **args) == T * 1298 * pc
    assert bench.class_bytes("ilu", p, fuse_first=True, **args) == T * 1056 * pc
    # one backward sweep instead of two
    args1 = dict(args, sweeps_bwd=1)
    assert bench.class_bytes("ilu", p, fuse_first=True, **args1) == T * (1056 - 272) * pc
    # no forward sweep: nothing to fold, the block-diagonal pass stays
    args0 = dict(args, sweeps=0, sweeps_bwd=0)
    assert bench.class_bytes("ilu", p, fuse_first=True, **args0) == T * 210 * pc
    # backward sweep pairs: two backward sweeps in one launch, moving one sweep's bytes
    assert bench.class_bytes("ilu", p, fuse_first=True, pairs=True, **args) == T * (240 + 272 + 272) * pc
    args3 = dict(args, sweeps=3, sweeps_bwd=3)
    assert bench.class_bytes("ilu", p, fuse_first=True, pairs=True, **args3) == T * (240 + 2 * 272 + 2 * 272) * pc


def test_fp64_and_exact_ilu_bytes():
    T, pc = 10, 1
    p = _prof(precond=pc)
    # FP64 path: 8-byte values everywhere; level-scheduled exact ILU reads each factor once per relation
    exact = bench.class_bytes("ilu", p, T=T, F=0, steps=1, sweeps=2, exact=True, mixed=False, basis32=False)
    fwd = 20 * 8 + 8 * 8 + 8 * 34 + 12 + 20 * 8
    bwd = 20 * 8 + 8 * 8 + 8 * 34 + 12 + 20 * 8
    assert exact == T * (fwd + bwd) * pc


def test_gram_schmidt_operator_and_residual_bytes():
    T = 100
    p = _prof(n=6, jsum=12, residuals=3)
    # mixed, FP32 basis: (2 jsum + 3 n) vectors of 20 values, once
    assert bench.class_bytes("orth", p, T=T, F=0, steps=1, sweeps=2, exact=False, mixed=True,
                             basis32=True) == T * 20 * 4 * (2 * 12 + 3 * 6)
    # FP64: 8-byte basis and the classical Gram-Schmidt pass twice
    assert bench.class_bytes("orth", p, T=T, F=0, steps=1, sweeps=2, exact=False, mixed=False,
                             basis32=False) == T * 20 * 8 * (2 * 12 + 3 * 6) * 2
    # the first Gram-Schmidt products in the operator kernel: the orth class keeps the update
    # ((j + 3) vectors), the operator class adds the basis vectors V_0..V_j
    assert bench.class_bytes("orth", p, T=T, F=0, steps=1, sweeps=2, exact=False, mixed=True, basis32=True,
                             fused_dots=True) == T * 20 * 4 * (12 + 2 * 6)
    assert bench.class_bytes("spmv", p, T=T, F=0, steps=1, sweeps=2, exact=False, mixed=True, basis32=True,
                             fused_dots=True) == T * ((4 * 24 + 12 + 20 * 4 + 20 * 4) * 6 + 20 * 4 * 12)
    # operator: blocks (24 values) + neighbour indices + source + result per iteration
    assert bench.class_bytes("spmv", p, T=T, F=0, steps=1, sweeps=2, exact=False, mixed=True,
                             basis32=True) == T * (4 * 24 + 12 + 20 * 4 + 20 * 4) * 6
    # refinement residual: FP64 (or FP32-pair) operator, x (the neighbours' entries counted once, as
    # for the other kernels: ncu reads 524.6 MB per 1M-cell launch = 8 * 24 + 12 + 160 + 160), b, the
    # basis slot
    assert bench.class_bytes("resid", p, T=T, F=0, steps=1, sweeps=2, exact=False, mixed=True,
                             basis32=True) == T * (8 * 24 + 12 + 160 + 160 + 80) * 3


def test_update_and_correction_bytes():
    T, F, steps = 50, 80, 4
    p = _prof(n=6, residuals=3 * steps)
    assert bench.class_bytes("update", p, T=T, F=F, steps=steps, sweeps=2, exact=False, mixed=True,
                             basis32=True) == (T * 84 + F * 32) * steps
    # Z vectors once per Arnoldi iteration, x read and written once per cycle (residuals beyond one per step)
    assert bench.class_bytes("corr", p, T=T, F=F, steps=steps, sweeps=2, exact=False, mixed=True,
                             basis32=True) == T * (20 * 4 * 6 + 320 * (3 * steps - steps))
    with pytest.raises(KeyError):
        bench.class_bytes("flux", p, T=T, F=F, steps=steps, sweeps=2, exact=False, mixed=True, basis32=True)


def test_option_maps_match_the_config():
    assert bench.WARM == {"prev": 0, "extrap": 1, "extrap2": 2}
    assert bench.FLUX_SPLIT == {"on": 1, "off": 0}
    assert bench.GRAPHS == {"device": 0, "host": 2, "none": 1}
    assert bench.METRIC == "triangle-steps/s"


def test_counter_record_format():
    """profiles/traffic.txt: kernel, a 16-hex-digit hash of the flux sources,
    DRAM bytes per launch, the Gauss points of that launch and the FP64 / FP32
    flops per Gauss point ('-' if not taken); a line is used only while the
    hash matches the sources (else the roofline's achieved rate and traffic are
    null), and bench.py's hash is deterministic."""
    p = os.path.join(bench.ROOT, "profiles", "traffic.txt")
    kernels = set()
    for line in open(p):
        if line.startswith("#") or not line.strip():
            continue
        k, h, by, gp, f64, f32 = line.split()[:6]
        assert re.fullmatch(r"[0-9a-f]{16}", h)
        assert float(by) > 0 and float(gp) > 0
        assert all(x == "-" or float(x) > 0 for x in (f64, f32))
        kernels.add(k)
    assert {"mixed_flux_ws", "mixed_flux", "flux"} <= kernels
    assert bench.source_hash() == bench.source_hash() and re.fullmatch(r"[0-9a-f]{16}", bench.source_hash())
    assert bench.counter_record("no_such_kernel") is None


def _peaks():
    return {"fp64_tflops": 1.2, "fp32_tflops": 74.0, "fp64_tflops_derived": 1.26, "fp32_tflops_derived": 80.5}


def test_flux_roofline_uses_the_counters_of_the_timed_kernel(monkeypatch):
    """The flux roofline takes its flops per Gauss point from the record of the
    kernel it names (never a constant of another kernel), divides by the event
    time of one launch, and reports the busier pipe against its measured rate."""
    seen = []

    def rec(key):
        seen.append(key)
        return {"dram_bytes": 2.0e8, "gauss_points": 1.0e6, "fp64_flop_per_gp": 600.0, "fp32_flop_per_gp": 8000.0}

    monkeypatch.setattr(bench, "counter_record", rec)
    gp, ms = 3_000_000, 2.0
    r = bench.flux_roofline("mixed_flux_ws", "k_face_flux_ws", 10, ms, gp, _peaks())
    assert seen == ["mixed_flux_ws"] and r["kernel"] == "k_face_flux_ws"
    a64 = 600.0 * gp / (ms / 1e3) / 1e12
    a32 = 8000.0 * gp / (ms / 1e3) / 1e12
    assert r["pipe"] == ("fp64" if a64 / 1.2 > a32 / 74.0 else "fp32")
    assert abs(r["achieved"] - (a64 if r["pipe"] == "fp64" else a32)) < 1e-12
    assert abs(r["frac"] - r["achieved"] / r["peak"]) < 1e-12
    assert abs(r["traffic"] - 2.0e8 * 3) < 1e-3
    # stale counters (hash mismatch): no achieved rate, no traffic
    monkeypatch.setattr(bench, "counter_record", lambda key: None)
    r = bench.flux_roofline("mixed_flux_ws", "k_face_flux_ws", 10, ms, gp, _peaks())
    assert r["achieved"] is None and r["frac"] is None and r["traffic"] is None


def test_flux_kernel_follows_the_configuration():
    """The roofline names the kernel the configuration launches and reads that
    kernel's counters: pairs -> k_face_flux_df, FP64 lead split ->
    k_face_flux_ws, FP64 lead single-role and the FP64 path -> k_face_flux."""
    from types import SimpleNamespace as NS
    assert bench.flux_kernel(NS(flux_lead="pairs", flux_split="on"), True) == ("mixed_flux_df", "k_face_flux_df")
    assert bench.flux_kernel(NS(flux_lead="fp64", flux_split="on"), True) == ("mixed_flux_ws", "k_face_flux_ws")
    assert bench.flux_kernel(NS(flux_lead="fp64", flux_split="off"), True) == ("mixed_flux", "k_face_flux")
    assert bench.flux_kernel(NS(flux_lead="pairs", flux_split="on"), False) == ("flux", "k_face_flux")


def test_counter_records_name_known_kernels_and_the_default_one_is_current():
    """Every record of profiles/traffic.txt names a flux kernel whose sources
    bench.py knows, each kernel's hash covers only its own files, and the
    default mixed kernel's record was taken on its current sources (else the
    benchmark's roofline would have no achieved rate)."""
    p = os.path.join(bench.ROOT, "profiles", "traffic.txt")
    for line in open(p):
        if line.startswith("#") or not line.strip():
            continue
        assert line.split()[0] in bench.FLUX_SOURCES
    assert bench.source_hash("mixed_flux_df") != bench.source_hash("flux")
    rec = bench.counter_record("mixed_flux_df")
    assert rec is not None and rec["fp32_flop_per_gp"] > 0 and rec["dram_bytes"] > 0


def test_reference_arm_prints_its_line():
    """bench.py --impl reference times the oracle on the host cores (the only
    reference this tier has) and prints the contract's line: impl, the metric of
    the GPU arm, a cpu_baseline describing the run and an e2e with no copies."""
    import json
    import subprocess
    import sys
    r = subprocess.run([sys.executable, os.path.join(bench.ROOT, "bench.py"), "--impl", "reference", "--steps", "1",
                        "--warmup", "0"], capture_output=True, text=True, timeout=600, cwd=bench.ROOT)
    assert r.returncode == 0, r.stderr[-2000:]
    line = json.loads([l for l in r.stdout.splitlines() if l.startswith("{")][-1])
    assert line["impl"] == "reference" and line["metric"] == bench.METRIC and line["value"] > 0
    assert line["higher_is_better"] is True and line["cpu_baseline"]["kind"] == "oracle"
    assert line["cpu_baseline"]["value"] == line["value"] and line["cpu_baseline"]["cores"] >= 1
    assert line["e2e"] == {"value": line["value"], "unit": line["unit"], "h2d_bytes_per_step": 0,
                           "d2h_bytes_per_step": 0}
