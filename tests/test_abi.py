"""The C-ABI library builds, loads and exports every entry point that
include/gks.h declares (no compute call: this runs without a GPU)."""
import ctypes as C
import os
import re

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.fixture(scope="module")
def lib():
    from paper_1802_00704_gb300 import build, gks
    build.build()
    return gks.load()


def _declared():
    txt = open(os.path.join(ROOT, "include", "gks.h")).read()
    return re.findall(r"GKS_EXPORT\s+[\w\s\*]+?\b(gks_\w+)\s*\(", txt)


def test_header_declares_entry_points():
    names = _declared()
    assert set(names) >= {"gks_mesh_create", "gks_cls_reconstruct", "gks_flux", "gks_step", "gks_run"}


def test_library_exports_every_declared_symbol(lib):
    from paper_1802_00704_gb300 import gks
    for name in _declared():
        assert hasattr(lib, name), name
    assert set(_declared()) == set(gks.EXPORTED)


def test_config_defaults(lib):
    from paper_1802_00704_gb300 import gks
    c = gks.config()
    assert c.gamma == 1.4 and c.cfl == 0.3 and c.cls_w == 0.3 and c.gmres_m == 30
    assert c.gmres_rtol == 1e-12 and c.precision == gks.FP64 and c.limiter == 0 and c.basis_fp32 == 0
    assert c.warm_extrap == 0 and c.second_order == 0 and c.no_graphs == 0
    assert c.cls_M == 1 and c.cls_global == 0 and c.slope0_mode == 0 and c.ilu_fp16 == 0
    assert c.limit_char == 0 and c.inner_rtol == 1e-6 and c.ilu_sweeps_bwd == -1 and c.ilu_fuse_first == 1
    assert c.flux_split == 1
    assert c.prandtl == 1.0
    assert c.flux_lead == 1 and c.ilu_sweep_pairs == 1 and c.spmv_dots == 1
    assert c.flux_shape == 0 and c.reserved == 0 and c.precond == gks.PC_ILU_SWEEP


def _c_layout(struct, fields):
    """sizeof and offsetof of a struct of include/gks.h, from a C program
    compiled with gcc against the header (the layout the library sees)."""
    import subprocess
    import tempfile
    body = "\n".join(f'    printf("%zu\\n", offsetof({struct}, {f}));' for f in fields)
    src = (f'#include <stddef.h>\n#include <stdio.h>\n#include "gks.h"\n'
           f'int main(void) {{\n    printf("%zu\\n", sizeof({struct}));\n{body}\n    return 0;\n}}\n')
    with tempfile.TemporaryDirectory() as tmp:
        cpath, exe = os.path.join(tmp, "layout.c"), os.path.join(tmp, "layout")
        open(cpath, "w").write(src)
        subprocess.run(["gcc", "-I", os.path.join(ROOT, "include"), cpath, "-o", exe], check=True)
        out = subprocess.run([exe], check=True, capture_output=True, text=True).stdout.split()
    return int(out[0]), [int(x) for x in out[1:]]


@pytest.mark.parametrize("struct,mirror", [("gks_config", "Config"), ("gks_tune_result", "TuneResult"),
                                           ("gks_run_info", "RunInfo"), ("gks_profile", "Profile"),
                                           ("gks_mesh_stats", "MeshStats")])
def test_ctypes_mirrors_match_the_header(struct, mirror):
    """The binding's ctypes structures have the size and field offsets of the
    C structures of include/gks.h."""
    pytest.importorskip("subprocess")
    from paper_1802_00704_gb300 import gks
    cls = getattr(gks, mirror)
    names = [f for f, _ in cls._fields_]
    size, offs = _c_layout(struct, names)
    assert C.sizeof(cls) == size
    assert [getattr(cls, f).offset for f in names] == offs


def test_binding_refuses_cpu_tensors(lib):
    import torch
    from paper_1802_00704_gb300 import gks
    with pytest.raises(TypeError):
        gks._dev(torch.zeros(4, 3, dtype=torch.float64))


@pytest.mark.parametrize("field,value", [
    ("ilu_sweeps_bwd", -2), ("ilu_sweeps_bwd", 9), ("ilu_fuse_first", 2), ("flux_split", 2), ("flux_split", -1),
    ("ilu_fp16", 1),            # FP16 factors need the mixed precision
    ("cls_M", 0),               # values-only equations need the second-order variant
    ("slope0_mode", 2), ("no_graphs", 3), ("warm_extrap", 3), ("inner_rtol", 0.0),
    ("flux_shape", 3), ("flux_shape", -1), ("reserved", 1),
])
def test_invalid_config_is_refused_before_any_device_call(lib, field, value):
    """gks_mesh_create checks the configuration first: an invalid field gives
    GKS_EINVAL with a message, and no CUDA call is made (this runs without a
    GPU)."""
    from paper_1802_00704_gb300 import gks
    from paper_1802_00704_gb300 import inputs as I
    case = I.advection_case(3)
    with pytest.raises(gks.GksError) as e:
        gks.GksMesh(case.mesh, **{field: value})
    assert e.value.status == gks.GKS_EINVAL and "invalid gks_config" in str(e.value)


@pytest.mark.parametrize("precond", [-1, 4])
def test_unknown_preconditioner_is_refused(lib, precond):
    """The four preconditioners (sync-free exact ILU, sweeps, block Jacobi, level
    launches) are 0..3; anything else is GKS_EINVAL before any device call."""
    from paper_1802_00704_gb300 import gks
    from paper_1802_00704_gb300 import inputs as I
    case = I.advection_case(3)
    with pytest.raises(gks.GksError) as e:
        gks.GksMesh(case.mesh, precond=precond)
    assert e.value.status == gks.GKS_EINVAL and "precond" in str(e.value)
