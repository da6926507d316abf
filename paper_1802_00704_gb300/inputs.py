"""Seeded synthetic inputs for the third-order gas-kinetic scheme on triangles.

This module builds the inputs that both the CUDA library and the CPU oracle
consume: jittered split-quad triangulations (nodes, triangles, faces with
left/right cells, boundary tags and periodic shifts), per-face boundary data
and initial cell averages of the conservative variables.  It contains none of
the scheme's arithmetic (no geometry of the reconstruction, no flux, no
solver): only mesh topology, random numbers and quadrature of the analytic
initial conditions of the paper's test cases (Sec. IV: Eqs. (41)-(42)
density-perturbation advection, Eq. (44) Sod, Eqs. (49)-(52) shock-vortex,
Sec. IV.G lid-driven cavity).

Random numbers come from a counter-based SplitMix64 (Steele, Lea & Flood,
"Fast splittable pseudorandom number generators", OOPSLA 2014): output k of
stream `seed` is mix64(seed + (k+1) * 0x9E3779B97F4A7C15).

Face array layout (int32, 5 per face): n0, n1, cell_l, cell_r, tag.
  n0, n1   node indices of the face, in cell_l's frame;
  cell_r   -1 on a non-periodic boundary face;
  tag      TAG_* below.
face_shift (float64, 2 per face): translation that carries cell_r's
coordinates next to cell_l across a periodic face (zero otherwise).
bc_state (float64, 4 per face): conservative state (rho, rho u, rho v, E)
for Dirichlet faces; (u_wall, v_wall, T_wall, 0) for no-slip walls; unused
otherwise.
"""
from __future__ import annotations

import math
from dataclasses import dataclass, field

import numpy as np

TAG_INTERIOR = 0
TAG_PERIODIC = 1
TAG_DIRICHLET = 2
TAG_OUTFLOW = 3
TAG_SLIP = 4
TAG_NOSLIP = 5

_GOLDEN = np.uint64(0x9E3779B97F4A7C15)
_M1 = np.uint64(0xBF58476D1CE4E5B9)
_M2 = np.uint64(0x94D049BB133111EB)


def splitmix64(seed: int, n: int, offset: int = 0) -> np.ndarray:
    """Outputs offset .. offset+n-1 of the SplitMix64 stream `seed` (uint64)."""
    with np.errstate(over="ignore"):
        k = np.arange(offset + 1, offset + n + 1, dtype=np.uint64)
        z = np.uint64(seed & 0xFFFFFFFFFFFFFFFF) + k * _GOLDEN
        z = (z ^ (z >> np.uint64(30))) * _M1
        z = (z ^ (z >> np.uint64(27))) * _M2
        z = z ^ (z >> np.uint64(31))
    return z


def uniform01(seed: int, n: int, offset: int = 0) -> np.ndarray:
    """Uniform doubles in [0, 1) from the top 53 bits of SplitMix64."""
    return (splitmix64(seed, n, offset) >> np.uint64(11)).astype(np.float64) * (2.0 ** -53)


@dataclass
class Mesh:
    nodes: np.ndarray          # (n_nodes, 2) float64
    tris: np.ndarray           # (n_tri, 3) int32, counter-clockwise
    faces: np.ndarray          # (n_face, 5) int32
    face_shift: np.ndarray     # (n_face, 2) float64
    bc_state: np.ndarray       # (n_face, 4) float64
    nx: int = 0
    ny: int = 0
    lx: float = 1.0
    ly: float = 1.0
    meta: dict = field(default_factory=dict)

    @property
    def n_tri(self) -> int:
        return int(self.tris.shape[0])

    @property
    def n_face(self) -> int:
        return int(self.faces.shape[0])


_SIDES = ("left", "right", "bottom", "top")


def split_quad_mesh(nx: int, ny: int, lx: float, ly: float, *, seed: int,
                    periodic_x: bool = False, periodic_y: bool = False,
                    bc: dict | None = None, jitter: float = 0.2,
                    x0: float = 0.0, y0: float = 0.0) -> Mesh:
    """nx x ny quads on [x0, x0+lx] x [y0, y0+ly]; interior nodes jittered by
    U(-jitter, jitter) times the quad side (per axis); each quad split on a
    diagonal chosen by a fair coin.  Boundary nodes are not jittered, so the
    two sides of a periodic direction match exactly.  Nodes on opposite
    periodic sides are kept as distinct nodes: every triangle owns unwrapped
    coordinates, and the periodic faces carry the shift instead.

    bc maps a side name ('left', 'right', 'bottom', 'top') to (tag, state4)
    for non-periodic sides.
    """
    if nx < 3 or ny < 3:
        raise ValueError("split_quad_mesh needs nx, ny >= 3")
    bc = dict(bc or {})
    hx, hy = lx / nx, ly / ny
    ii, jj = np.meshgrid(np.arange(nx + 1), np.arange(ny + 1), indexing="xy")
    ii = ii.ravel()
    jj = jj.ravel()
    n_nodes = (nx + 1) * (ny + 1)
    x = x0 + ii * hx
    y = y0 + jj * hy
    r = uniform01(seed, 2 * n_nodes)
    interior = (ii > 0) & (ii < nx) & (jj > 0) & (jj < ny)
    x = np.where(interior, x + (2.0 * r[0::2] - 1.0) * jitter * hx, x)
    y = np.where(interior, y + (2.0 * r[1::2] - 1.0) * jitter * hy, y)
    nodes = np.stack([x, y], axis=1)

    qi, qj = np.meshgrid(np.arange(nx), np.arange(ny), indexing="xy")
    qi = qi.ravel()
    qj = qj.ravel()
    n00 = qj * (nx + 1) + qi
    n10 = n00 + 1
    n01 = n00 + (nx + 1)
    n11 = n01 + 1
    diag = uniform01(seed, nx * ny, offset=2 * n_nodes) < 0.5
    t_a = np.where(diag[:, None], np.stack([n00, n10, n11], 1), np.stack([n00, n10, n01], 1))
    t_b = np.where(diag[:, None], np.stack([n00, n11, n01], 1), np.stack([n10, n11, n01], 1))
    tris = np.empty((2 * nx * ny, 3), dtype=np.int64)
    tris[0::2] = t_a
    tris[1::2] = t_b

    # Wrapped node ids identify nodes on opposite periodic sides.
    wi = np.where(periodic_x & (ii == nx), 0, ii) if periodic_x else ii
    wj = np.where(periodic_y & (jj == ny), 0, jj) if periodic_y else jj
    wid = wj * (nx + 1) + wi

    n_tri = tris.shape[0]
    ea = np.concatenate([tris[:, 0], tris[:, 1], tris[:, 2]])
    eb = np.concatenate([tris[:, 1], tris[:, 2], tris[:, 0]])
    et = np.concatenate([np.arange(n_tri)] * 3)
    wa, wb = wid[ea], wid[eb]
    key = np.minimum(wa, wb).astype(np.int64) * n_nodes + np.maximum(wa, wb)
    order = np.argsort(key, kind="stable")
    key_s = key[order]
    uniq, start, count = np.unique(key_s, return_index=True, return_counts=True)
    if np.any(count > 2):
        raise RuntimeError("non-manifold edge in split-quad mesh")

    faces = np.zeros((uniq.shape[0], 5), dtype=np.int64)
    shift = np.zeros((uniq.shape[0], 2))
    state = np.zeros((uniq.shape[0], 4))

    def on_side(a, b, side):
        if side == "left":
            return (ii[a] == 0) & (ii[b] == 0)
        if side == "right":
            return (ii[a] == nx) & (ii[b] == nx)
        if side == "bottom":
            return (jj[a] == 0) & (jj[b] == 0)
        return (jj[a] == ny) & (jj[b] == ny)

    # Two-sided faces.
    two = count == 2
    e0 = order[start[two]]
    e1 = order[start[two] + 1]
    raw0 = np.minimum(ea[e0], eb[e0]) * n_nodes + np.maximum(ea[e0], eb[e0])
    raw1 = np.minimum(ea[e1], eb[e1]) * n_nodes + np.maximum(ea[e1], eb[e1])
    periodic = raw0 != raw1
    # Interior: cell_l = lower triangle index.  Periodic: cell_l is the cell on
    # the right (x = x0+lx) or top (y = y0+ly) side, so the shift is +lx / +ly.
    e0_far = np.zeros(e0.shape, dtype=bool)
    e1_far = np.zeros(e1.shape, dtype=bool)
    sh = np.zeros((e0.shape[0], 2))
    if periodic_x:
        f0 = on_side(ea[e0], eb[e0], "right")
        f1 = on_side(ea[e1], eb[e1], "right")
        sh[periodic & (f0 | f1), 0] = lx
        e0_far |= f0
        e1_far |= f1
    if periodic_y:
        f0 = on_side(ea[e0], eb[e0], "top")
        f1 = on_side(ea[e1], eb[e1], "top")
        sh[periodic & (f0 | f1), 1] = ly
        e0_far |= f0
        e1_far |= f1
    swap = np.where(periodic, e1_far & ~e0_far, et[e1] < et[e0])
    el = np.where(swap, e1, e0)
    er = np.where(swap, e0, e1)
    idx_two = np.nonzero(two)[0]
    faces[idx_two, 0] = ea[el]
    faces[idx_two, 1] = eb[el]
    faces[idx_two, 2] = et[el]
    faces[idx_two, 3] = et[er]
    faces[idx_two, 4] = np.where(periodic, TAG_PERIODIC, TAG_INTERIOR)
    shift[idx_two] = sh

    # One-sided faces: physical boundary.
    one = count == 1
    idx_one = np.nonzero(one)[0]
    eo = order[start[one]]
    faces[idx_one, 0] = ea[eo]
    faces[idx_one, 1] = eb[eo]
    faces[idx_one, 2] = et[eo]
    faces[idx_one, 3] = -1
    tagged = np.zeros(idx_one.shape[0], dtype=bool)
    for side in _SIDES:
        m = on_side(ea[eo], eb[eo], side)
        if not np.any(m):
            continue
        if side not in bc:
            raise ValueError(f"side '{side}' is a boundary but has no bc entry")
        tag, st = bc[side]
        faces[idx_one[m], 4] = tag
        state[idx_one[m]] = np.asarray(st, dtype=np.float64)
        tagged |= m
    if not np.all(tagged):
        raise RuntimeError("untagged boundary face")

    return Mesh(nodes=nodes, tris=tris.astype(np.int32), faces=faces.astype(np.int32),
                face_shift=shift, bc_state=state, nx=nx, ny=ny, lx=lx, ly=ly,
                meta={"x0": x0, "y0": y0, "seed": seed})


# ---------------------------------------------------------------------------
# Initial conditions: cell averages by collapsed (Duffy) Gauss quadrature.

def _duffy_rule(n: int = 8):
    g, w = np.polynomial.legendre.leggauss(n)
    s = 0.5 * (g + 1.0)
    ws = 0.5 * w
    su, sv = np.meshgrid(s, s, indexing="ij")
    wu, wv = np.meshgrid(ws, ws, indexing="ij")
    # x = p0 + a (p1 - p0) + a b (p2 - p1); Jacobian 2|T| a.
    return su.ravel(), sv.ravel(), (2.0 * wu * wv * su).ravel()


def cell_average(mesh: Mesh, fn, n: int = 8) -> np.ndarray:
    """Cell averages of fn(x, y) -> (k, npts) over each triangle; returns (k, T)."""
    a, b, w = _duffy_rule(n)
    p = mesh.nodes[mesh.tris]                       # (T, 3, 2)
    p0, p1, p2 = p[:, 0], p[:, 1], p[:, 2]
    xq = p0[:, None, :] + a[None, :, None] * (p1 - p0)[:, None, :] \
        + (a * b)[None, :, None] * (p2 - p1)[:, None, :]
    vals = np.asarray(fn(xq[..., 0], xq[..., 1]))   # (k, T, nq)
    return np.einsum("ktq,q->kt", vals, w)


def prim_to_cons(rho, u, v, p, gamma):
    return np.stack([rho, rho * u, rho * v, p / (gamma - 1.0) + 0.5 * rho * (u * u + v * v)])


@dataclass
class Case:
    name: str
    mesh: Mesh
    w0: np.ndarray             # (4, T) conservative cell averages, SoA
    gamma: float = 1.4
    mu: float = 0.0
    t_final: float = 0.0
    steps: int = 0
    meta: dict = field(default_factory=dict)


def advection_case(n: int, *, seed: int = 1802, k: int = 1, amp: float = 0.2,
                   length: float = 2.0, gamma: float = 1.4) -> Case:
    """Diagonal density wave rho = 1 + amp sin(k pi (x + y)), u = v = 1, p = 1 on
    a doubly periodic [0, length]^2 (the 2-D restatement of Eqs. (41)-(42))."""
    mesh = split_quad_mesh(n, n, length, length, seed=seed, periodic_x=True, periodic_y=True)

    def fn(x, y):
        rho = 1.0 + amp * np.sin(k * math.pi * (x + y))
        return prim_to_cons(rho, np.ones_like(rho), np.ones_like(rho), np.ones_like(rho), gamma)

    return Case("advection", mesh, cell_average(mesh, fn), gamma=gamma,
                meta={"k": k, "amp": amp, "length": length})


def advection_exact_density(case: Case, t: float) -> np.ndarray:
    k, amp = case.meta["k"], case.meta["amp"]
    return cell_average(case.mesh, lambda x, y: (1.0 + amp * np.sin(k * math.pi * (x + y - 2.0 * t)))[None])[0]


def riemann_strip_case(nx: int, ny: int, *, left, right, x_split: float = 0.5,
                       seed: int = 1802, gamma: float = 1.4, name: str = "sod") -> Case:
    """Strip [0,1] x [0, ny/nx]: periodic in y, Dirichlet (initial states) at x = 0, 1.
    left/right are primitive (rho, u, v, p)."""
    ly = ny / nx
    wl = prim_to_cons(*[np.float64(q) for q in left], gamma)
    wr = prim_to_cons(*[np.float64(q) for q in right], gamma)
    mesh = split_quad_mesh(nx, ny, 1.0, ly, seed=seed, periodic_y=True,
                           bc={"left": (TAG_DIRICHLET, wl), "right": (TAG_DIRICHLET, wr)})

    def fn(x, y):
        m = x < x_split
        return np.where(m[None], wl[:, None, None], wr[:, None, None]) * np.ones_like(x)[None]

    return Case(name, mesh, cell_average(mesh, fn), gamma=gamma,
                meta={"left": tuple(left), "right": tuple(right), "x_split": x_split})


def sod_case(nx: int = 400, ny: int = 8, seed: int = 1802) -> Case:
    """Sod initial data, Eq. (44)."""
    return riemann_strip_case(nx, ny, left=(1.0, 0.0, 0.0, 1.0), right=(0.125, 0.0, 0.0, 0.1), seed=seed)


def _vortex_profile(eps, a, b, gamma, n=20001):
    """Tangential velocity of the compact vortex and the temperature that keeps it
    in radial equilibrium along an isentrope (T = p / rho, T_inf = 1)."""
    r = np.linspace(0.0, b, n)
    ut = np.where(r <= a, eps * r / a, eps * a / (a * a - b * b) * (r - b * b / np.maximum(r, 1e-300)))
    ut[0] = 0.0
    integrand = np.where(r > 0, ut * ut / np.maximum(r, 1e-300), 0.0)
    # T(r) = 1 - (gamma-1)/gamma * int_r^b ut^2/r' dr'
    seg = 0.5 * (integrand[1:] + integrand[:-1]) * np.diff(r)
    tail = np.concatenate([np.cumsum(seg[::-1])[::-1], [0.0]])
    temp = 1.0 - (gamma - 1.0) / gamma * tail
    return r, ut, temp


def shock_vortex_case(nx: int = 1000, ny: int = 500, *, seed: int = 1802, gamma: float = 1.4,
                      mach: float = 1.1, eps: float = 0.3, a: float = 0.075, b: float = 0.175) -> Case:
    """Stationary Mach-1.1 normal shock at x = 0.5 (left state Eq. (49)) with a
    compact vortex centred at (0.25, 0.5) on [0,2] x [0,1].  Supersonic inflow
    (Dirichlet) on the left, extrapolation outflow on the right, slip walls top
    and bottom."""
    u1 = mach * math.sqrt(gamma)
    rho_ratio = (gamma + 1.0) * mach ** 2 / ((gamma - 1.0) * mach ** 2 + 2.0)
    p_ratio = 1.0 + 2.0 * gamma / (gamma + 1.0) * (mach ** 2 - 1.0)
    rho2, p2, u2 = rho_ratio, p_ratio, u1 / rho_ratio
    wl = prim_to_cons(np.float64(1.0), np.float64(u1), np.float64(0.0), np.float64(1.0), gamma)
    wr = prim_to_cons(np.float64(rho2), np.float64(u2), np.float64(0.0), np.float64(p2), gamma)
    mesh = split_quad_mesh(nx, ny, 2.0, 1.0, seed=seed,
                           bc={"left": (TAG_DIRICHLET, wl), "right": (TAG_OUTFLOW, wr),
                               "bottom": (TAG_SLIP, np.zeros(4)), "top": (TAG_SLIP, np.zeros(4))})
    rt, ut_t, temp_t = _vortex_profile(eps, a, b, gamma)

    def fn(x, y):
        dx, dy = x - 0.25, y - 0.5
        r = np.sqrt(dx * dx + dy * dy)
        ut = np.interp(r, rt, ut_t, right=0.0)
        temp = np.interp(r, rt, temp_t, right=1.0)
        rinv = np.where(r > 0, 1.0 / np.maximum(r, 1e-300), 0.0)
        rho_v = temp ** (1.0 / (gamma - 1.0))
        left = x < 0.5
        rho = np.where(left, rho_v, rho2)
        u = np.where(left, u1 - ut * dy * rinv, u2)
        v = np.where(left, ut * dx * rinv, 0.0)
        p = np.where(left, rho_v * temp, p2)
        return prim_to_cons(rho, u, v, p, gamma)

    return Case("shock_vortex", mesh, cell_average(mesh, fn), gamma=gamma, t_final=0.6,
                meta={"mach": mach, "eps": eps, "a": a, "b": b})


def cavity_case(n: int = 256, *, seed: int = 1802, gamma: float = 1.4, lid_mach: float = 0.15,
                reynolds: float = 1000.0, prandtl: float = 0.72) -> Case:
    """Lid-driven cavity on the unit square: isothermal no-slip walls at T = 1,
    top wall moving at lid_mach * sqrt(gamma) (Sec. IV.G); the Prandtl number the
    workload asks for is carried in meta["prandtl"]."""
    u_lid = lid_mach * math.sqrt(gamma)
    mu = u_lid / reynolds
    wall = np.array([0.0, 0.0, 1.0, 0.0])
    lid = np.array([u_lid, 0.0, 1.0, 0.0])
    mesh = split_quad_mesh(n, n, 1.0, 1.0, seed=seed,
                           bc={"left": (TAG_NOSLIP, wall), "right": (TAG_NOSLIP, wall),
                               "bottom": (TAG_NOSLIP, wall), "top": (TAG_NOSLIP, lid)})
    t = mesh.n_tri
    w0 = prim_to_cons(np.ones(t), np.zeros(t), np.zeros(t), np.ones(t), gamma)
    return Case("cavity", mesh, w0, gamma=gamma, mu=mu, meta={"u_lid": u_lid, "re": reynolds, "prandtl": prandtl})


def acoustic_pulse_case(n: int, *, seed: int = 1802, eps: float = 0.01, half_width: float = 0.04,
                        gamma: float = 1.4) -> Case:
    """Acoustic pressure pulse of Sec. IV (Eq. (45)): unit square (periodic; the
    pulse stays far from the sides for t <= 0.2), rho = 1, u = v = 0,
    p = 1 + eps exp(-alpha eta^2), eta = |x - (0.5, 0.5)|, alpha = ln 2 / half_width^2."""
    alpha = math.log(2.0) / half_width ** 2
    mesh = split_quad_mesh(n, n, 1.0, 1.0, seed=seed, periodic_x=True, periodic_y=True)

    def fn(x, y):
        p = 1.0 + eps * np.exp(-alpha * ((x - 0.5) ** 2 + (y - 0.5) ** 2))
        return prim_to_cons(np.ones_like(x), np.zeros_like(x), np.zeros_like(x), p, gamma)

    return Case("acoustic_pulse", mesh, cell_average(mesh, fn), gamma=gamma,
                meta={"eps": eps, "alpha": alpha, "x0": 0.5, "y0": 0.5})


def batch_case(c: int, n_cases: int = 512, *, seed: int = 704, t_min: float = 1e3, t_max: float = 2e5,
               mesh_seed: int = 1802) -> Case:
    """Case c of the batch: log-uniform triangle count; even index periodic
    advection (wavenumber 1-4, amplitude 0.05-0.2), odd index Riemann strip
    (density and pressure ratios 2-10)."""
    r = uniform01(seed, 4 * n_cases).reshape(n_cases, 4)
    t_target = math.exp(math.log(t_min) + r[c, 0] * (math.log(t_max) - math.log(t_min)))
    if c % 2 == 0:
        n = max(3, int(round(math.sqrt(t_target / 2.0))))
        k = 1 + int(r[c, 1] * 4.0) % 4
        amp = 0.05 + 0.15 * r[c, 2]
        return advection_case(n, seed=mesh_seed + c, k=k, amp=amp)
    nx = max(3, int(round(t_target / 16.0)))
    rr = 2.0 + 8.0 * r[c, 1]
    rp = 2.0 + 8.0 * r[c, 2]
    return riemann_strip_case(nx, 8, left=(rr, 0.0, 0.0, rp), right=(1.0, 0.0, 0.0, 1.0), seed=mesh_seed + c,
                              name="riemann")


def batch_cases(n_cases: int = 512, *, seed: int = 704, t_min: float = 1e3, t_max: float = 2e5,
                mesh_seed: int = 1802, workers: int = 1) -> list[Case]:
    """All cases of the batch (see batch_case), generated by `workers` spawned
    processes when workers > 1 (the result does not depend on it)."""
    kw = dict(n_cases=n_cases, seed=seed, t_min=t_min, t_max=t_max, mesh_seed=mesh_seed)
    if workers <= 1:
        return [batch_case(c, **kw) for c in range(n_cases)]
    import functools
    import multiprocessing as mp
    from concurrent.futures import ProcessPoolExecutor
    with ProcessPoolExecutor(workers, mp_context=mp.get_context("spawn")) as ex:
        return list(ex.map(functools.partial(batch_case, **kw), range(n_cases), chunksize=4))
