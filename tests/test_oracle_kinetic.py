"""Pins of the oracle's kinetic part (Sec. II) against mathematics that does not
go through the oracle's own formulas: quadrature of the Maxwellian, analytic
logarithmic derivatives of g, the Euler equations, closed-form time integrals
and the exact Euler flux of a smooth solution."""
import math

import numpy as np
import pytest
import sympy as sp

GAMMA = 1.4
K = 2.0 / (GAMMA - 1.0) - 2.0


# --------------------------------------------------------------------------- moments

def _quad_moment(U, lam, half, a):
    """<u^a> by composite Gauss-Legendre on U -+ 14/sqrt(lam), split at 0."""
    s = 14.0 / math.sqrt(lam)
    lo, hi = U - s, U + s
    if half > 0:
        lo = max(lo, 0.0)
    if half < 0:
        hi = min(hi, 0.0)
    if hi <= lo:
        return 0.0
    x, w = np.polynomial.legendre.leggauss(60)
    edges = np.linspace(lo, hi, 41)
    tot = 0.0
    for e0, e1 in zip(edges[:-1], edges[1:]):
        u = 0.5 * (e0 + e1) + 0.5 * (e1 - e0) * x
        f = u ** a * math.sqrt(lam / math.pi) * np.exp(-lam * (u - U) ** 2)
        tot += 0.5 * (e1 - e0) * np.dot(w, f)
    return tot


@pytest.mark.parametrize("U,lam", [(0.3, 0.7), (-1.2, 2.5), (2.0, 0.4), (0.0, 1.0)])
def test_moments_vs_quadrature(oracle_mod, U, lam):
    for half in (0, 1, -1):
        for a in range(0, 10):
            ref = _quad_moment(U, lam, half, a)
            got = oracle_mod.moment(U, 0.0, lam, K, half, a, 0, 0)
            scale = max(1.0, abs(ref))
            assert abs(got - ref) <= 1e-13 * scale * (1 + a), (half, a, got, ref)
            if half == 0:
                s = oracle_mod.moment(U, 0.0, lam, K, 1, a, 0, 0) + oracle_mod.moment(U, 0.0, lam, K, -1, a, 0, 0)
                assert abs(s - got) <= 1e-13 * scale * (1 + a)


def test_internal_moments_gamma_ratio(oracle_mod):
    # <zeta^q> = Gamma(K/2 + q) / (Gamma(K/2) lam^q) for zeta = xi.xi, K = 3.
    lam = 0.83
    for q in range(4):
        ref = math.gamma(K / 2 + q) / (math.gamma(K / 2) * lam ** q)
        got = oracle_mod.moment(0.1, 0.2, lam, K, 0, 0, 0, q)
        assert abs(got - ref) < 1e-14 * ref


# --------------------------------------------------------------------------- slopes

x_, y_ = sp.symbols("x y", real=True)


def _field(kind):
    if kind == "general":
        rho = 1 + sp.Rational(3, 10) * sp.sin(sp.Rational(13, 10) * x_ + sp.Rational(2, 5) * y_)
        U = sp.Rational(1, 2) + sp.Rational(1, 5) * sp.cos(sp.Rational(7, 10) * x_ - sp.Rational(9, 10) * y_)
        V = -sp.Rational(3, 10) + sp.Rational(1, 10) * sp.sin(sp.Rational(1, 2) * x_ + sp.Rational(11, 10) * y_)
        p = 1 + sp.Rational(1, 4) * sp.cos(sp.Rational(4, 5) * x_ + sp.Rational(3, 10) * y_)
    else:  # density wave advected by a uniform flow at uniform pressure
        rho = 1 + sp.Rational(1, 5) * sp.sin(2 * x_ + sp.Rational(3, 4) * y_)
        U, V, p = sp.Rational(4, 5), -sp.Rational(3, 10), sp.Integer(1)
    return rho, U, V, p


def _cons(rho, U, V, p):
    return [rho, rho * U, rho * V, p / (GAMMA - 1) + rho * (U ** 2 + V ** 2) / 2]


def _rows(W, pt):
    rows = [W, [sp.diff(q, x_) for q in W], [sp.diff(q, y_) for q in W],
            [sp.diff(q, x_, 2) for q in W], [sp.diff(q, x_, y_) for q in W], [sp.diff(q, y_, 2) for q in W]]
    return np.array([[float(q.subs(pt)) for q in r] for r in rows])


def _lng_coeffs(rho, U, V, p):
    """ln g = c0 + c1 u + c2 v + c3 (u^2+v^2+zeta)/2 as sympy expressions."""
    lam = rho / (2 * p)
    c3 = -2 * lam
    c1 = 2 * lam * U
    c2 = 2 * lam * V
    c0 = sp.log(rho) + (K + 2) / 2 * sp.log(lam) - lam * (U ** 2 + V ** 2)
    return [c0, c1, c2, c3]


@pytest.mark.parametrize("kind", ["general", "advection"])
def test_space_slopes_are_log_derivatives(oracle_mod, kind):
    rho, U, V, p = _field(kind)
    W = _cons(rho, U, V, p)
    pt = {x_: 0.3, y_: 0.7}
    rows = _rows(W, pt)
    sl = oracle_mod.state_slopes(rows, GAMMA)
    c = _lng_coeffs(rho, U, V, p)
    ev = lambda e: np.array([float(q.subs(pt)) for q in e])
    a1 = ev([sp.diff(q, x_) for q in c])
    a2 = ev([sp.diff(q, y_) for q in c])
    a11 = ev([sp.diff(q, x_, 2) for q in c])
    a12 = ev([sp.diff(q, x_, y_) for q in c])
    a22 = ev([sp.diff(q, y_, 2) for q in c])
    for got, ref in [(sl[0], a1), (sl[1], a2), (sl[3], a11), (sl[4], a12), (sl[5], a22)]:
        assert np.allclose(got, ref, rtol=1e-11, atol=1e-11), (got, ref)


def test_time_slope_matches_euler(oracle_mod):
    """rho <psi A> = dW/dt = -(dF/dx + dG/dy) for the Euler fluxes F, G."""
    rho, U, V, p = _field("general")
    W = _cons(rho, U, V, p)
    E = W[3]
    F = [rho * U, rho * U * U + p, rho * U * V, (E + p) * U]
    G = [rho * V, rho * U * V, rho * V * V + p, (E + p) * V]
    pt = {x_: -0.4, y_: 0.25}
    dWdt = np.array([float((-sp.diff(f, x_) - sp.diff(g, y_)).subs(pt)) for f, g in zip(F, G)])
    rows = _rows(W, pt)
    sl = oracle_mod.state_slopes(rows, GAMMA)
    A = sl[2]
    r0, u0, v0 = rows[0, 0], rows[0, 1] / rows[0, 0], rows[0, 2] / rows[0, 0]
    lam = r0 / (2 * (GAMMA - 1) * (rows[0, 3] - 0.5 * r0 * (u0 * u0 + v0 * v0)))
    # <psi psi^T> from quadrature-verified moments
    m = lambda a, b, z: oracle_mod.moment(u0, v0, lam, K, 0, a, b, z)
    psi = [[(1, 0, 0, 0)], [(1, 1, 0, 0)], [(1, 0, 1, 0)], [(0.5, 2, 0, 0), (0.5, 0, 2, 0), (0.5, 0, 0, 1)]]
    M = np.array([[sum(ca * cb * m(a1 + a2, b1 + b2, z1 + z2) for ca, a1, b1, z1 in psi[i] for cb, a2, b2, z2 in psi[j])
                   for j in range(4)] for i in range(4)])
    assert np.allclose(r0 * M @ A, dWdt, rtol=1e-11, atol=1e-11)


def test_time_slopes_for_pure_advection(oracle_mod):
    """For rho(x - U t) at uniform U, V, p the exact g is transported, so
    A = -(U a1 + V a2), A1 = -(U a11 + V a12), A2 = -(U a12 + V a22) and
    At = U^2 a11 + 2 U V a12 + V^2 a22 (Eq. (12) read on the exact solution)."""
    rho, U, V, p = _field("advection")
    W = _cons(rho, U, V, p)
    rows = _rows(W, {x_: 0.2, y_: -0.1})
    sl = oracle_mod.state_slopes(rows, GAMMA)
    u, v = float(U), float(V)
    a1, a2, A, a11, a12, a22, A1, A2, At = sl
    assert np.allclose(A, -(u * a1 + v * a2), atol=1e-12)
    assert np.allclose(A1, -(u * a11 + v * a12), atol=1e-12)
    assert np.allclose(A2, -(u * a12 + v * a22), atol=1e-12)
    assert np.allclose(At, u * u * a11 + 2 * u * v * a12 + v * v * a22, atol=1e-12)


# --------------------------------------------------------------------------- time integrals

def _closed_forms(dt, tau, exact):
    e = math.exp(-dt / tau)
    T0 = tau * (1 - e)
    T1 = tau * T0 - tau * dt * e
    T2 = 2 * tau * T1 - tau * dt * dt * e
    c = [dt - T0, T1 + tau * T0 - tau * dt, dt * dt / 2 - tau * dt + tau * T0, -(T2 + 2 * tau * T1),
         dt ** 3 / 3 - tau * dt * dt, -tau * dt * dt / 2 - tau * T1, T0, -T1, T2]
    if exact:
        k = 2 * tau * tau * (dt - T0)
        c[3] += k
        c[4] += k
        c[5] += k
    return np.array(c)


@pytest.mark.parametrize("ratio", [0.3, 1.0, 5.0, 100.0])
@pytest.mark.parametrize("exact", [0, 1])
def test_time_integrals_closed_form(oracle_mod, ratio, exact):
    dt = 0.013
    tau = dt / ratio
    got = oracle_mod.time_integrals(dt, tau, exact)
    ref = _closed_forms(dt, tau, exact)
    scale = np.array([dt, dt * dt, dt * dt, dt ** 3, dt ** 3, dt ** 3, dt, dt * dt, dt ** 3])
    assert np.all(np.abs(got - ref) <= 1e-13 * scale), (got - ref) / scale


def test_time_integrals_small_tau_limit(oracle_mod):
    dt = 0.02
    c = oracle_mod.time_integrals(dt, 1e-15 * dt, 0)
    # As tau -> 0 the kernel of Eq. (8) concentrates at t' = t, where x' = 0:
    # only the time-Taylor terms of g survive (c1 -> 1, c3 -> t, c5 -> t^2).
    assert abs(c[0] - dt) < 1e-12 * dt
    assert abs(c[1]) < 1e-12 * dt * dt
    assert abs(c[2] - dt * dt / 2) < 1e-12 * dt * dt
    assert abs(c[3]) < 1e-12 * dt ** 3
    assert abs(c[4] - dt ** 3 / 3) < 1e-12 * dt ** 3
    assert abs(c[5]) < 1e-12 * dt ** 3
    assert abs(c[6]) < 1e-12 * dt and abs(c[7]) < 1e-12 * dt * dt


# --------------------------------------------------------------------------- Gauss-point flux

def _prim_rows(rho, U, V, p):
    w = np.zeros((6, 4))
    w[0] = [rho, rho * U, rho * V, p / (GAMMA - 1) + 0.5 * rho * (U * U + V * V)]
    return w


def test_constant_state_flux_is_euler_flux(oracle_mod):
    for rho, U, V, p in [(1.3, 0.7, -0.4, 0.9), (0.2, -2.0, 0.5, 0.05), (1.0, 0.0, 0.0, 1.0)]:
        w = _prim_rows(rho, U, V, p)
        dt = 0.013
        f, aux, st = oracle_mod.point_flux(w, w, dt)
        E = w[0, 3]
        ref = dt * np.array([rho * U, rho * U * U + p, rho * U * V, (E + p) * U])
        assert st == 0
        assert np.allclose(f, ref, rtol=1e-13, atol=1e-15 * dt)


def test_slip_wall_mirror_has_no_mass_or_energy_flux(oracle_mod):
    rng = np.random.default_rng(3)
    wl = _prim_rows(1.1, 0.3, 0.2, 0.8)
    wl[1:] = 0.05 * rng.standard_normal((5, 4))
    sign_n = np.array([0, 1, 0, 2, 1, 0])
    s = np.array([1.0, -1.0, 1.0, 1.0])
    wr = wl * s[None, :] * ((-1.0) ** sign_n)[:, None]
    f, _, st = oracle_mod.point_flux(wl, wr, 0.01)
    assert st == 0
    assert abs(f[0]) < 1e-15 and abs(f[2]) < 1e-15 and abs(f[3]) < 1e-15
    assert f[1] > 0


def _euler_flux(W):
    rho, mx, my, E = W
    u, v = mx / rho, my / rho
    p = (GAMMA - 1) * (E - 0.5 * rho * (u * u + v * v))
    return np.array([mx, mx * u + p, mx * v, (E + p) * u])


def test_flux_is_third_order_in_time_for_advection(oracle_mod):
    """With tau -> 0 (viscous form, mu = 1e-12) the time-integrated flux of a
    smooth transported density wave matches the exact Euler flux integral with
    an O(dt^4) error (third-order scheme)."""
    u, v, p, k, th, ph = 0.8, -0.3, 1.0, 2.0, 0.4, 0.7
    c, s_ = math.cos(th), math.sin(th)

    def cons(t):
        rho = 1 + 0.2 * math.sin(k * ((-u * t) * c + (-v * t) * s_) + ph)
        return np.array([rho, rho * u, rho * v, p / (GAMMA - 1) + 0.5 * rho * (u * u + v * v)])

    a1, a2 = 0.2 * k * math.cos(ph), -0.2 * k * k * math.sin(ph)
    drho = [1 + 0.2 * math.sin(ph), a1 * c, a1 * s_, a2 * c * c, a2 * c * s_, a2 * s_ * s_]
    rows = np.array([[dr, dr * u, dr * v, 0.5 * dr * (u * u + v * v)] for dr in drho])
    rows[0, 3] += p / (GAMMA - 1)
    gx, gw = np.polynomial.legendre.leggauss(20)
    errs = []
    for dt in [0.08, 0.04, 0.02]:
        ref = sum(0.5 * dt * wq * _euler_flux(cons(0.5 * dt * (xq + 1))) for xq, wq in zip(gx, gw))
        f, _, st = oracle_mod.point_flux(rows, rows, dt, mu=1e-12)
        assert st == 0
        errs.append(np.abs(f - ref).max())
    assert errs[0] / errs[1] > 12 and errs[1] / errs[2] > 12, errs


def test_flux_time_taylor_general_flow(oracle_mod):
    """General smooth state, tau -> 0: the equilibrium part of Eq. (15) is then
    the second-order time Taylor expansion of g at the point, so the
    time-integrated flux must equal F dt + F_t dt^2/2 + F_tt dt^3/6 of the Euler
    equations (time derivatives by Cauchy-Kowalewski) up to rounding."""
    rho, U, V, p = _field("general")
    W = _cons(rho, U, V, p)

    def fluxes(Wv):
        r, mx, my, e = Wv
        uu, vv = mx / r, my / r
        pp = (GAMMA - 1) * (e - (mx * uu + my * vv) / 2)
        return [mx, mx * uu + pp, mx * vv, (e + pp) * uu], [my, mx * vv, my * vv + pp, (e + pp) * vv]

    ws = sp.symbols("w0:4")
    Fs, Gs = fluxes(ws)
    JF = sp.Matrix(Fs).jacobian(ws)
    JG = sp.Matrix(Gs).jacobian(ws)
    sub = dict(zip(ws, W))
    Fx, Gx = sp.Matrix(Fs).subs(sub), sp.Matrix(Gs).subs(sub)
    Wt = -(Fx.diff(x_) + Gx.diff(y_))
    Ft = JF.subs(sub) * Wt
    Gt = JG.subs(sub) * Wt
    Wtt = -(Ft.diff(x_) + Gt.diff(y_))
    HF = [sp.Matrix([JF[i, :]]).jacobian(ws) for i in range(4)]
    Ftt = sp.Matrix([(Wt.T * HF[i].subs(sub) * Wt)[0] for i in range(4)]) + JF.subs(sub) * Wtt
    pt = {x_: 0.1, y_: -0.2}
    F0 = np.array([float(q.subs(pt)) for q in Fx])
    F1 = np.array([float(q.subs(pt)) for q in Ft])
    F2 = np.array([float(q.subs(pt)) for q in Ftt])
    rows = _rows(W, pt)
    errs = []
    for dt in [0.04, 0.02, 0.01]:
        ref = F0 * dt + F1 * dt ** 2 / 2 + F2 * dt ** 3 / 6
        f, _, st = oracle_mod.point_flux(rows, rows, dt, mu=1e-12)
        assert st == 0
        errs.append(np.abs(f - ref).max() / np.abs(ref).max())
    assert max(errs) < 1e-12, errs


def _conduction_rows(g=0.1, T0=1.0, p=1.0, U=0.0, V=0.0, gamma=GAMMA):
    """Face-frame rows of a state with uniform pressure and velocity and a
    temperature T = p / rho growing linearly along the face normal (T0 + g n)."""
    rho0, drho, d2rho = p / T0, -p * g / T0 ** 2, 2.0 * p * g * g / T0 ** 3
    w = np.zeros((6, 4))
    for r, d in ((0, rho0), (1, drho), (3, d2rho)):
        w[r] = [d, d * U, d * V, 0.5 * d * (U * U + V * V)]
    w[0, 3] += p / (gamma - 1.0)
    return w


@pytest.mark.parametrize("prandtl", [1.0, 0.72, 2.0 / 3.0])
def test_heat_flux_is_fourier_conduction(oracle_mod, prandtl):
    """At rest, uniform pressure, linear temperature: the flux is pressure in the
    normal momentum and Fourier conduction -c_p (mu / Pr) dT/dn in the energy
    (c_p = gamma / (gamma - 1), the conductivity of the BGK-NS limit rescaled by
    the Prandtl correction), whatever tangential velocity the gas has."""
    g, mu, dt = 0.1, 1e-4, 1e-2
    cp = GAMMA / (GAMMA - 1.0)
    for V in (0.0, 0.3):
        w = _conduction_rows(g=g, V=V)
        f, _, st = oracle_mod.point_flux(w, w, dt, mu=mu, prandtl=prandtl)
        assert st == 0
        assert abs(f[0]) < 1e-15 and abs(f[1] - dt) < 1e-14
        assert abs(f[3] - (-cp * mu / prandtl * g * dt)) < 1e-10 * cp * mu * g * dt
        assert abs(f[2]) < 1e-14


def test_prandtl_rescales_only_the_heat_flux(oracle_mod):
    """With normal flow the energy flux also carries U (E + p): the Prandtl
    correction changes the energy flux by (1/Pr - 1) times the conduction part
    only, and leaves mass and momentum fluxes untouched."""
    g, mu, dt, U = 0.1, 1e-4, 1e-3, 0.4
    cp = GAMMA / (GAMMA - 1.0)
    w = _conduction_rows(g=g, U=U)
    f1, _, _ = oracle_mod.point_flux(w, w, dt, mu=mu, prandtl=1.0)
    f2, _, _ = oracle_mod.point_flux(w, w, dt, mu=mu, prandtl=0.72)
    assert np.all(np.abs(f2[:3] - f1[:3]) <= 1e-15 * np.abs(f1[:3]).max())
    heat = -cp * mu * g * dt
    assert abs((f2[3] - f1[3]) - (1.0 / 0.72 - 1.0) * heat) < 0.02 * abs((1.0 / 0.72 - 1.0) * heat)


# --------------------------------------------------- interface derivatives (slope0_mode)


def _two_fields():
    rho, U, V, p = _field("general")
    rho2 = 0.6 + sp.Rational(1, 5) * sp.cos(sp.Rational(9, 10) * x_ - sp.Rational(3, 5) * y_)
    U2 = sp.Rational(-1, 5) + sp.Rational(3, 10) * sp.sin(sp.Rational(6, 5) * x_ + sp.Rational(1, 2) * y_)
    V2 = sp.Rational(2, 5) + sp.Rational(1, 5) * sp.cos(sp.Rational(3, 10) * x_ + y_)
    p2 = sp.Rational(7, 10) + sp.Rational(1, 10) * sp.sin(x_ - sp.Rational(2, 5) * y_)
    pt = {x_: 0.4, y_: -0.2}
    return _rows(_cons(rho, U, V, p), pt), _rows(_cons(rho2, U2, V2, p2), pt)


def _taylor(rows, x, y):
    """Value row of the state whose reconstruction has the given rows, at (x, y)."""
    out = np.zeros((6, 4))
    out[0] = rows[0] + x * rows[1] + y * rows[2] + 0.5 * x * x * rows[3] + x * y * rows[4] + 0.5 * y * y * rows[5]
    return out


def test_kinetic_interface_derivatives_are_derivatives_of_w0(oracle_mod):
    """slope0_mode = 1: the derivative rows of W0 are the derivatives of the value
    rho_l <psi>_{u>0,l} + rho_r <psi>_{u<0,r} when the left and right states vary
    as their reconstructions do: checked against Richardson-extrapolated central
    differences of that value (computed from shifted states with zero derivative
    rows, so only the zeroth-order half-space moments enter)."""
    wl, wr = _two_fields()
    got = oracle_mod.interface_w0(wl, wr, GAMMA, mode=1)

    def F(x, y):
        return oracle_mod.interface_w0(_taylor(wl, x, y), _taylor(wr, x, y), GAMMA, mode=0)[0]

    def rich(d, e):
        return (4.0 * d(e / 2) - d(e)) / 3.0

    e = 2e-3
    d_n = rich(lambda h: (F(h, 0) - F(-h, 0)) / (2 * h), e)
    d_t = rich(lambda h: (F(0, h) - F(0, -h)) / (2 * h), e)
    d_nn = rich(lambda h: (F(h, 0) - 2 * F(0, 0) + F(-h, 0)) / (h * h), e)
    d_tt = rich(lambda h: (F(0, h) - 2 * F(0, 0) + F(0, -h)) / (h * h), e)
    d_nt = rich(lambda h: (F(h, h) - F(h, -h) - F(-h, h) + F(-h, -h)) / (4 * h * h), e)
    fd = np.array([F(0, 0), d_n, d_t, d_nn, d_nt, d_tt])
    for r in range(6):
        scale = np.max(np.abs(fd[r]))
        assert np.max(np.abs(got[r] - fd[r])) <= 1e-8 * scale, (r, got[r], fd[r])
    # and they differ from the mean of the left and right rows (mode 0)
    mean = oracle_mod.interface_w0(wl, wr, GAMMA, mode=0)
    assert np.max(np.abs(got[1:] - mean[1:])) > 1e-3 * np.max(np.abs(mean[1:]))


def test_kinetic_interface_derivatives_reduce_to_the_state_for_continuous_data(oracle_mod):
    """For equal left and right states the two half spaces add up to the full
    space: both modes give W0 = W with the state's own derivative rows, and the
    same flux."""
    wl, _ = _two_fields()
    for mode in (0, 1):
        w0 = oracle_mod.interface_w0(wl, wl, GAMMA, mode=mode)
        assert np.allclose(w0, wl, rtol=1e-13, atol=1e-13 * np.max(np.abs(wl)))
    f0, _, s0 = oracle_mod.point_flux(wl, wl, 0.01)
    f1, _, s1 = oracle_mod.point_flux(wl, wl, 0.01, slope0_mode=1)
    assert s0 == s1 == 0
    assert np.allclose(f1, f0, rtol=1e-12, atol=1e-14)
