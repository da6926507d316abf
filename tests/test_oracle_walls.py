"""Pins of the oracle's boundary ghost states and of the CFL rule against
mathematics outside the oracle.

The paper does not print its boundary conditions.  The isothermal no-slip wall
is read as the mirror image of the primitive fields: the pressure even, the
velocity odd about the wall velocity and the temperature T = p / rho odd about
the wall temperature.  A field with exactly that symmetry continues across the
wall unchanged, so its ghost must equal the interior state; the kinetic flux of
such data is then the Navier-Stokes flux of the continued field (viscous shear
stress, Fourier conduction), which the pins below check against their closed
forms.  Each pin fails if the reflected temperature, a momentum parity or the
wall-velocity frame is wrong."""
import math

import numpy as np
import pytest

GAMMA = 1.4
TAG_SLIP, TAG_NOSLIP = 4, 5


def _rows_from_fields(p, un, ut, T, gamma=GAMMA):
    """Face-frame conservative rows (6, 4) at (n, t) = (0, 0) of the primitive
    fields given as sympy expressions in n, t."""
    sp = pytest.importorskip("sympy")
    n, t = sp.symbols("n t")
    rho = p / T
    cons = [rho, rho * un, rho * ut, p / (gamma - 1) + rho * (un ** 2 + ut ** 2) / 2]
    derivs = [(), (n,), (t,), (n, n), (n, t), (t, t)]
    out = np.zeros((6, 4))
    for r, d in enumerate(derivs):
        for v, q in enumerate(cons):
            e = sp.diff(q, *d) if d else q
            out[r, v] = float(e.subs({n: 0, t: 0}))
    return out


def _wall_bc(theta, u_wt, T_w):
    """Boundary data (wall velocity x, y, wall temperature, unused) of a wall
    whose outward normal is (cos theta, sin theta), moving along its tangent."""
    nx, ny = math.cos(theta), math.sin(theta)
    return np.array([-ny * u_wt, nx * u_wt, T_w, 0.0]), nx, ny


def test_noslip_ghost_of_symmetric_fields_is_the_field_itself(oracle_mod):
    """Pressure even in n, velocity and temperature odd about their wall
    values: the reflected fields coincide with the interior fields, so the
    ghost rows equal the interior rows (all 24 entries, first and second
    derivatives included)."""
    sp = pytest.importorskip("sympy")
    n, t = sp.symbols("n t")
    u_wt, T_w = 0.37, 1.2
    p = 0.9 + 0.2 * t + 0.15 * n ** 2 - 0.1 * t ** 2
    un = 0.3 * n + 0.2 * n * t                       # odd about 0 (a tangentially moving wall)
    ut = u_wt + 0.5 * n - 0.4 * n * t                # odd about the wall velocity
    T = T_w - 0.3 * n + 0.25 * n * t                 # odd about the wall temperature
    wl = _rows_from_fields(p, un, ut, T)
    for theta in (0.0, 0.8, 2.9):
        bc, nx, ny = _wall_bc(theta, u_wt, T_w)
        wr = oracle_mod.ghost_rows(TAG_NOSLIP, bc, nx, ny, wl)
        assert np.allclose(wr, wl, rtol=0, atol=1e-13), (theta, wr - wl)


def test_noslip_ghost_reflects_values_about_the_wall_state(oracle_mod):
    """An interior state away from the wall values: the ghost has the same
    pressure, the velocity 2 u_w - u and the temperature 2 T_w - T."""
    bc, nx, ny = _wall_bc(0.4, 0.2, 1.1)
    rho, un, ut, p = 1.3, 0.1, -0.25, 0.8
    wl = np.zeros((6, 4))
    wl[0] = [rho, rho * un, rho * ut, p / (GAMMA - 1) + 0.5 * rho * (un * un + ut * ut)]
    wr = oracle_mod.ghost_rows(TAG_NOSLIP, bc, nx, ny, wl)
    Tg = 2 * 1.1 - p / rho
    rg = p / Tg
    ung, utg = -un, 2 * 0.2 - ut
    ref = [rg, rg * ung, rg * utg, p / (GAMMA - 1) + 0.5 * rg * (ung * ung + utg * utg)]
    assert np.allclose(wr[0], ref, rtol=1e-14)
    assert np.all(wr[1:] == 0.0)


def _uniform_rows(rho, un, ut, p):
    w = np.zeros((6, 4))
    w[0] = [rho, rho * un, rho * ut, p / (GAMMA - 1) + 0.5 * rho * (un * un + ut * ut)]
    return w


@pytest.mark.parametrize("prandtl", [1.0, 0.72])
def test_noslip_wall_state_has_no_mass_energy_or_shear_flux(oracle_mod, prandtl):
    """Gas at the wall velocity and temperature, no gradients: the only flux
    through the wall is the pressure in the normal momentum."""
    mu, dt = 2e-3, 1e-2
    for u_wt, T_w, p in ((0.0, 1.0, 1.0), (0.3, 1.25, 0.7)):
        bc, nx, ny = _wall_bc(1.1, u_wt, T_w)
        wl = _uniform_rows(p / T_w, 0.0, u_wt, p)
        wr = oracle_mod.ghost_rows(TAG_NOSLIP, bc, nx, ny, wl)
        f, _, st = oracle_mod.point_flux(wl, wr, dt, mu=mu, prandtl=prandtl)
        assert st == 0
        assert abs(f[0]) < 1e-13 * p * dt and abs(f[2]) < 1e-13 * p * dt and abs(f[3]) < 1e-13 * p * dt, f
        assert abs(f[1] - p * dt) < 1e-13 * p * dt


def test_noslip_linear_shear_gives_the_viscous_stress(oracle_mod):
    """u_t = u_w - s n (n the outward normal, uniform density and temperature at
    the wall values): the tangential momentum through the wall is the
    Navier-Stokes stress -mu du_t/dn times dt = mu s dt (plane Couette flow is
    a steady solution, so the time integral carries no higher-order term), and
    no mass crosses the wall."""
    mu, s, u_w = 1e-3, 0.5, 0.2
    bc, nx, ny = _wall_bc(0.0, u_w, 1.0)
    wl = _uniform_rows(1.0, 0.0, u_w, 1.0)
    wl[1, 2] = -s                                     # d(rho u_t)/dn
    wl[1, 3] = -s * u_w                               # d(rho |u|^2 / 2)/dn
    wl[3, 3] = s * s                                  # d2(rho |u|^2 / 2)/dn2
    wr = oracle_mod.ghost_rows(TAG_NOSLIP, bc, nx, ny, wl)
    assert np.allclose(wr, wl, atol=1e-15)
    for dt in (1e-3, 1e-2):
        f, _, st = oracle_mod.point_flux(wl, wr, dt, mu=mu)
        assert st == 0
        assert abs(f[2] / (mu * s * dt) - 1.0) < 1e-10, f
        assert abs(f[0]) < 1e-12 * mu * s * dt


@pytest.mark.parametrize("prandtl", [1.0, 0.72])
def test_noslip_linear_temperature_gives_fourier_conduction(oracle_mod, prandtl):
    """At rest against a fixed wall at T_w, uniform pressure, T = T_w + a n:
    the ghost continues the profile and the energy flux through the wall is
    Fourier conduction -c_p (mu / Pr) a dt, c_p = gamma / (gamma - 1)."""
    sp = pytest.importorskip("sympy")
    n, t = sp.symbols("n t")
    mu, dt, a, T_w = 1e-4, 1e-2, 0.1, 1.0
    wl = _rows_from_fields(sp.Float(1.0) + 0 * n, 0 * n, 0 * n, T_w + a * n)
    bc, nx, ny = _wall_bc(0.0, 0.0, T_w)
    wr = oracle_mod.ghost_rows(TAG_NOSLIP, bc, nx, ny, wl)
    assert np.allclose(wr, wl, atol=1e-14)
    f, _, st = oracle_mod.point_flux(wl, wr, dt, mu=mu, prandtl=prandtl)
    cp = GAMMA / (GAMMA - 1.0)
    ref = -cp * mu / prandtl * a * dt
    assert st == 0
    assert abs(f[3] - ref) < 1e-8 * abs(ref), (f, ref)
    assert abs(f[0]) < 1e-15 and abs(f[2]) < 1e-15


def test_slip_ghost_is_the_mirror_image(oracle_mod):
    """Slip wall: the conservative fields mirrored, normal momentum odd."""
    rng = np.random.default_rng(5)
    wl = _uniform_rows(1.1, 0.3, 0.2, 0.8)
    wl[1:] = 0.05 * rng.standard_normal((5, 4))
    wr = oracle_mod.ghost_rows(TAG_SLIP, np.zeros(4), 0.6, 0.8, wl)
    nord = np.array([0, 1, 0, 2, 1, 0])
    sv = np.array([1.0, -1.0, 1.0, 1.0])
    assert np.array_equal(wr, wl * sv[None, :] * ((-1.0) ** nord)[:, None])


def test_cfl_uses_the_inradius_of_right_triangles(oracle_mod):
    """Unjittered split quads are right triangles with legs hx, hy: inradius
    (hx + hy - sqrt(hx^2 + hy^2)) / 2, and the step of a uniform state is
    cfl * r / (|U| + c + 2 mu / (rho r))."""
    from paper_1802_00704_gb300 import inputs as I
    hx, hy = 0.25, 0.1
    m = I.split_quad_mesh(4, 5, 4 * hx, 5 * hy, seed=3, periodic_x=True, periodic_y=True, jitter=0.0)
    mu = 0.01
    om = oracle_mod.OracleMesh(m, mu=mu)
    r = om.cell_geometry()["inrad"]
    r_ref = 0.5 * (hx + hy - math.hypot(hx, hy))
    assert np.allclose(r, r_ref, rtol=1e-14)
    rho, u, v, p = 1.2, 0.3, -0.4, 0.9
    w = np.ascontiguousarray(np.stack([np.full(m.n_tri, x) for x in
                                       (rho, rho * u, rho * v, p / (GAMMA - 1) + 0.5 * rho * (u * u + v * v))]))
    dt = om.cfl_dt(w)
    ref = 0.3 * r_ref / (math.hypot(u, v) + math.sqrt(GAMMA * p / rho) + 2 * mu / (rho * r_ref))
    assert abs(dt - ref) < 1e-14 * ref
