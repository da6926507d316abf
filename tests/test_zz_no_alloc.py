"""The allocation-free time-step entry point (gks_cfl_dt_noalloc) gives the
same step as gks_cfl_dt, on two calls in a row that share its static scratch.
It exists for callers that cannot allocate device memory at that moment
(time loops that reserve all memory up front, device memory owned by another
allocator).  This file is collected last on purpose."""
import numpy as np
import pytest

from paper_1802_00704_gb300 import inputs as I
from tests.gpu_util import dev, needs_gpu, torch

pytestmark = [pytest.mark.gpu, needs_gpu]


def test_noalloc_cfl_dt_matches_allocating_entry_point():
    from paper_1802_00704_gb300 import build, gks
    build.build()
    c = I.shock_vortex_case(120, 60)            # 14,400 cells: many reduction blocks and a ragged tail
    m = gks.GksMesh(c.mesh)
    w_a = dev(c.w0)
    w_b = dev(c.w0 * np.array([[1.0], [0.7], [1.3], [1.05]]))   # a second, different state
    dt_dev = torch.full((1,), float("nan"), dtype=torch.float64, device="cuda")
    for w in (w_a, w_b):                        # two calls in a row through the same scratch
        ref = m.cfl_dt(w)
        m.cfl_dt_noalloc(w, dt_dev)
        got = float(dt_dev.cpu().item())
        assert abs(got - ref) <= 1e-14 * ref, (got, ref)
