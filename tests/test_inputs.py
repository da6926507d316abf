"""Input generator: split-quad meshes, periodic pairing, boundary tags, determinism."""
import os

import numpy as np
import pytest

from paper_1802_00704_gb300 import inputs as I


def test_splitmix64_reference_values():
    # first outputs of SplitMix64 from state 0 (published reference sequence, tests/golden)
    gold = os.path.join(os.path.dirname(__file__), "golden", "splitmix64_seed0.txt")
    ref = [int(l, 16) for l in open(gold) if l.strip() and not l.startswith("#")]
    z = I.splitmix64(0, len(ref))
    assert [int(v) for v in z] == ref


@pytest.mark.parametrize("n", [3, 4, 20])
def test_periodic_counts_and_matching(n):
    c = I.advection_case(n)
    m = c.mesh
    assert m.n_tri == 2 * n * n
    assert m.n_face == 3 * n * n
    cnt = np.bincount(np.concatenate([m.faces[:, 2], m.faces[m.faces[:, 3] >= 0, 3]]), minlength=m.n_tri)
    assert np.all(cnt == 3)
    per = m.faces[:, 4] == I.TAG_PERIODIC
    assert per.sum() == 2 * n
    for f in np.nonzero(per)[0]:
        n0, n1, l, r, _ = m.faces[f]
        edge = {tuple(np.round(m.nodes[q], 12)) for q in (n0, n1)}
        rnodes = {tuple(np.round(p + m.face_shift[f], 12)) for p in m.nodes[m.tris[r]]}
        lnodes = {tuple(np.round(p, 12)) for p in m.nodes[m.tris[l]]}
        assert edge <= rnodes and edge <= lnodes


def test_strip_and_walls():
    s = I.sod_case()
    tags = np.bincount(s.mesh.faces[:, 4], minlength=6)
    assert s.mesh.n_tri == 6400 and s.mesh.n_face == 9608
    assert tags[I.TAG_DIRICHLET] == 16 and tags[I.TAG_PERIODIC] == 400
    cv = I.cavity_case(8)
    assert np.bincount(cv.mesh.faces[:, 4], minlength=6)[I.TAG_NOSLIP] == 32


def test_ccw_and_area():
    c = I.shock_vortex_case(20, 10)
    p = c.mesh.nodes[c.mesh.tris]
    a2 = (p[:, 1, 0] - p[:, 0, 0]) * (p[:, 2, 1] - p[:, 0, 1]) - (p[:, 2, 0] - p[:, 0, 0]) * (p[:, 1, 1] - p[:, 0, 1])
    assert np.all(a2 > 0)
    assert abs(0.5 * a2.sum() - 2.0) < 1e-12


def test_deterministic():
    a = I.advection_case(10, seed=5)
    b = I.advection_case(10, seed=5)
    c = I.advection_case(10, seed=6)
    assert np.array_equal(a.mesh.nodes, b.mesh.nodes) and np.array_equal(a.w0, b.w0)
    assert not np.array_equal(a.mesh.nodes, c.mesh.nodes)


def test_cell_average_exact_for_quadratics():
    c = I.advection_case(6)
    got = I.cell_average(c.mesh, lambda x, y: (1.0 + x * y + 0.5 * x * x)[None])[0]
    p = c.mesh.nodes[c.mesh.tris]
    mid = 0.5 * (p + np.roll(p, -1, axis=1))
    ref = np.mean(1.0 + mid[..., 0] * mid[..., 1] + 0.5 * mid[..., 0] ** 2, axis=1)
    assert np.allclose(got, ref, rtol=0, atol=1e-13)
