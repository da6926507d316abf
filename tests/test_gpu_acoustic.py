"""The second-order variant (k_i = 1 for every cell) and the acoustic pressure
pulse of Sec. IV on the GPU: parity of the second-order variant with the oracle
(1e-10 relative max after one step, 1e-8 after 20), and the third- against the
second-order scheme on the pulse, measured against the exact linear-acoustics
solution (cell averages of the Hankel integral) on 40^2, 80^2 and 160^2
split-quad meshes.  The convergence test uses the amplitude 1e-4 instead of the
paper's 0.01: the Euler solution departs from linear acoustics by O(eps^2),
which at 0.01 is a floor (about 3.5e-7 in L1) that the third-order scheme
reaches at 160^2."""
import math

import numpy as np
import pytest

from paper_1802_00704_gb300 import inputs as I
from tests.acoustic_exact import pulse_pressure_cell_average
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


@pytest.mark.parametrize("name", ["pulse20", "shock_vortex40x20"])
def test_second_order_variant_matches_oracle(O, G, name):
    c = I.acoustic_pulse_case(20) if name == "pulse20" else I.shock_vortex_case(40, 20)
    om = O.OracleMesh(c.mesh, second_order=1)
    gm = G.GksMesh(c.mesh, second_order=1)
    assert gm.stats()["n_k1"] == c.mesh.n_tri
    wo, wg = c.w0.copy(), dev(c.w0)
    for n in range(20):
        info = om.step(wo)
        assert info.status == 0
        gm.step(wg, info.dt)
        if n == 0:
            assert np.all(rel_max(host(wg) - c.w0, wo - c.w0, axis=1) <= 1e-9)
            assert np.all(rel_max(host(wg), wo, axis=1) <= 1e-10)
    assert np.all(rel_max(host(wg), wo, axis=1) <= 1e-8)


def _pulse_error(G, n, second, precision, tend=0.05, eps=1e-4):
    c = I.acoustic_pulse_case(n, eps=eps)
    m = G.GksMesh(c.mesh, second_order=second, precision=G.MIXED if precision == "mixed" else G.FP64)
    w = dev(c.w0)
    info = m.run(w, t_final=tend, max_steps=100000)
    assert abs(info["t"] - tend) <= 1e-14
    wh = host(w)
    p = 0.4 * (wh[3] - 0.5 * (wh[1] ** 2 + wh[2] ** 2) / wh[0])
    nodes, tris = c.mesh.nodes, c.mesh.tris
    q = nodes[tris]
    a = 0.5 * np.abs((q[:, 1, 0] - q[:, 0, 0]) * (q[:, 2, 1] - q[:, 0, 1]) -
                     (q[:, 2, 0] - q[:, 0, 0]) * (q[:, 1, 1] - q[:, 0, 1]))
    ex = pulse_pressure_cell_average(nodes, tris, tend, eps=eps)
    return np.sum(a * np.abs(p - ex)) / a.sum()


@pytest.mark.parametrize("precision", ["fp64", "mixed"])
def test_acoustic_pulse_third_vs_second_order(G, precision):
    e3 = [_pulse_error(G, n, 0, precision) for n in (40, 80, 160)]
    e2 = [_pulse_error(G, n, 1, precision) for n in (40, 80, 160)]
    r3 = [math.log2(e3[k] / e3[k + 1]) for k in range(2)]
    r2 = [math.log2(e2[k] / e2[k + 1]) for k in range(2)]
    print(f"pulse {precision}: third {e3} orders {r3}; second {e2} orders {r2}")
    assert all(a < b for a, b in zip(e3, e2))
    assert r3[1] > 2.5 and r3[1] > r2[1] + 0.3
