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
    # the ctypes mirror has the size of the C struct: 4 doubles, 2 ints, 1 double, 10 ints, 2 doubles
    assert C.sizeof(gks.Config) == 4 * 8 + 2 * 4 + 8 + 10 * 4 + 2 * 8 + 7 * 4 + 4   # + padding
    assert gks.Config.inner_rtol.offset == 88 and gks.Config.prandtl.offset == 96
    assert gks.Config.slope0_mode.offset == 104 and gks.Config.ilu_fp16.offset == 108
    assert gks.Config.cls_global.offset == 112 and gks.Config.cls_M.offset == 116
    assert gks.Config.ilu_sweeps_bwd.offset == 120 and gks.Config.ilu_fuse_first.offset == 124
    assert gks.Config.flux_split.offset == 128


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
