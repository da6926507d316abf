"""Double-FP32 arithmetic of the mixed flux (pairs of FP32 numbers on the FP32
pipe) against CUDA's FP64 results, and the flux kernel that uses it against
the FP64-lead mixed kernels and the oracle.

Bounds: the sums and products of Joldes, Muller & Popescu (2017) are within
4 u^2 = 2^-46 (u = 2^-24) of the exact result of their (pair-rounded)
arguments, quotients within 16 u^2; exp, expm1 are asked for 2^-45 relative
(the truncation of their series is below 2^-50, the rest is the rounding of
about 20 pair operations), erfcx for 2^-43 (14 Horner steps in pairs) against CUDA's FP64 functions (torch on
the GPU, within about 1 ulp = 2^-52), wherever the result is at least 2^-100:
below that the low word is an FP32 subnormal and the pair keeps an absolute
accuracy of 2^-149 instead (the flux only adds such values to O(1) terms)."""
import math

import numpy as np
import pytest

from paper_1802_00704_gb300 import inputs as I
from tests.gpu_util import dev, host, needs_gpu, rel_max, torch

pytestmark = [pytest.mark.gpu, needs_gpu]

BOUND = 2.0 ** -45


@pytest.fixture(scope="module")
def G():
    from paper_1802_00704_gb300 import build, gks
    build.build()
    return gks


@pytest.fixture(scope="module")
def O():
    from oracle import oracle
    oracle.build()
    return oracle


def _pair_value(t):
    """hi + lo of the split pair, exactly, in FP64 (hi + lo has <= 48 bits)."""
    return t[:, 0] + t[:, 1]


def test_split_is_the_nearest_pair(G):
    """hi = x rounded to FP32 and lo = x - hi rounded to FP32, bit for bit as
    numpy's IEEE conversions give them, over exponents -98..127, both signs,
    and halfway cases of the hi rounding (ties to even).  Below 2^-98 lo can be
    an FP32 subnormal and may differ from the single rounding by one subnormal
    step (2^-149): it is rounded to 24 bits before the scaling."""
    rng = np.random.default_rng(11)
    x = rng.uniform(1.0, 2.0, 40000) * np.exp2(rng.integers(-98, 127, 40000)) * rng.choice([-1.0, 1.0], 40000)
    # exact ties of the FP32 rounding: 24 leading bits then a single 1 bit
    base = np.float32(rng.uniform(1.0, 2.0, 2000)).astype(np.float64)
    ties = base + np.exp2(np.floor(np.log2(base)) - 24)
    x = np.concatenate([x, ties, -ties, [1.0, -1.0, 3.0e38]])
    got = host(G.probe_df("split", dev(x)))
    hi = x.astype(np.float32)
    lo = (x - hi.astype(np.float64)).astype(np.float32)
    bad = np.nonzero((got[:, 0] != hi.astype(np.float64)) | (got[:, 1] != lo.astype(np.float64)))[0]
    assert bad.size == 0, (x[bad[:5]], got[bad[:5]], hi[bad[:5]], lo[bad[:5]])
    tiny = rng.uniform(1.0, 2.0, 4000) * np.exp2(rng.integers(-126, -98, 4000)) * rng.choice([-1.0, 1.0], 4000)
    got = host(G.probe_df("split", dev(tiny)))
    hi = tiny.astype(np.float32)
    lo = (tiny - hi.astype(np.float64)).astype(np.float32)
    assert np.array_equal(got[:, 0], hi.astype(np.float64))
    assert np.max(np.abs(got[:, 1] - lo.astype(np.float64))) <= 2.0 ** -149


def test_pair_arithmetic_within_bound(G):
    rng = np.random.default_rng(12)
    n = 50000
    a = rng.uniform(0.5, 2.0, n) * np.exp2(rng.integers(-30, 30, n)) * rng.choice([-1.0, 1.0], n)
    b = rng.uniform(0.5, 2.0, n) * np.exp2(rng.integers(-30, 30, n)) * rng.choice([-1.0, 1.0], n)
    pa = _pair_value(host(G.probe_df("split", dev(a))))
    pb = _pair_value(host(G.probe_df("split", dev(b))))
    # products within 4 u^2 (DWTimesDW3); quotients within 16 u^2 (a one-step
    # remainder correction: the bound proved for such division is 15 u^2 + O(u^3))
    for op, ref, bound in (("mul", pa * pb, 2.0 ** -46), ("div", pa / pb, 2.0 ** -44), ("recip", 1.0 / pa, 2.0 ** -44)):
        got = host(G.probe_df(op, dev(a), dev(b)))[:, 0]
        assert np.max(np.abs(got / ref - 1.0)) <= bound, (op, np.max(np.abs(got / ref - 1.0)))
    got = host(G.probe_df("sqrt", dev(np.abs(a))))[:, 0]
    assert np.max(np.abs(got / np.sqrt(np.abs(pa)) - 1.0)) <= 2.0 ** -46
    # sums: relative to the result (the accurate pair sum keeps cancellation exact up to 3 u^2)
    got = host(G.probe_df("add", dev(a), dev(b)))[:, 0]
    ref = pa + pb
    ok = ref != 0
    assert np.max(np.abs(got[ok] - ref[ok]) / np.abs(ref[ok])) <= 2.0 ** -46


def test_exp_expm1_erfcx_against_cuda_fp64(G):
    rng = np.random.default_rng(13)
    x = np.concatenate([rng.uniform(-87.0, 88.0, 60000), rng.uniform(-1.0, 1.0, 20000),
                        np.linspace(-0.35, 0.35, 1001)])
    xs = _pair_value(host(G.probe_df("split", dev(x))))        # the arguments as the pairs hold them
    xt = dev(xs)
    got = host(G.probe_df("exp", dev(x)))[:, 0]
    ref = host(torch.exp(xt))
    big = ref >= 2.0 ** -100
    assert np.max(np.abs(got[big] / ref[big] - 1.0)) <= BOUND
    assert np.max(np.abs(got[~big] - ref[~big])) <= 2.0 ** -140
    y = x[np.abs(x) <= 30.0]
    ys = _pair_value(host(G.probe_df("split", dev(y))))
    got = host(G.probe_df("expm1", dev(y)))[:, 0]
    ref = host(torch.expm1(dev(ys)))
    nz = ref != 0
    assert np.max(np.abs(got[nz] / ref[nz] - 1.0)) <= BOUND
    # exp below the FP32 normal range is flushed to zero
    assert np.all(host(G.probe_df("exp", dev(np.array([-87.5, -100.0, -1e4]))))[:, 0] == 0.0)
    z = np.concatenate([rng.uniform(0.0, 10.0, 60000), np.linspace(0.0, 1e-3, 101), [0.0, 10.0]])
    zs = _pair_value(host(G.probe_df("split", dev(z))))
    got = host(G.probe_df("erfcx", dev(z)))[:, 0]
    ref = host(torch.special.erfcx(dev(zs)))
    # the polynomial itself is within 2e-17; the 14 Horner steps in pairs add up
    # to about 14 x 7 u^2 of rounding (measured 4.6e-14)
    assert np.max(np.abs(got / ref - 1.0)) <= 2.0 ** -43


def _random_rows(rng, n, deriv=0.1):
    from tests.test_gpu_parity import _random_states
    w = _random_states(rng, n)
    w[:, 1:] *= deriv
    return w


@pytest.mark.parametrize("prandtl,kin", [(1.0, 0), (0.72, 0), (1.0, 1)])
def test_pair_lead_matches_fp64_lead(G, prandtl, kin):
    """The mixed point flux with its FP64-accuracy part in double-FP32
    (flux_lead = 1) against the same flux with that part in FP64 (flux_lead = 0).
    With zero derivative rows the flux is that part alone (every slope-carrying
    term vanishes): the two agree to 1e-13.  With derivatives they agree to the
    FP32 part's rounding, which the compiler contracts differently in the two
    kernels (1e-8 of the flux scale)."""
    rng = np.random.default_rng(21)
    n = 4000
    wl, wr = _random_rows(rng, n), _random_rows(rng, n)
    w0l, w0r = wl.copy(), wr.copy()
    w0l[:, 1:] = 0.0
    w0r[:, 1:] = 0.0
    for dt, mu in ((0.004, 0.0), (0.004, 2e-3), (1e-5, 1e-2)):
        kw = dict(precision=G.MIXED, mu=mu, prandtl=prandtl, slope0_mode=kin)
        for (ql, qr), tol in (((w0l, w0r), 1e-13), ((wl, wr), 1e-8)):
            a = host(G.point_flux(dev(ql), dev(qr), dt, flux_lead=1, **kw))
            b = host(G.point_flux(dev(ql), dev(qr), dt, flux_lead=0, **kw))
            scale = np.max(np.abs(b), axis=0)
            err = np.max(np.abs(a - b), axis=0) / scale
            assert np.all(err <= tol), (dt, mu, tol, err)


def test_pair_lead_supersonic_and_tiny_states(G, O):
    """Half-space moments far in the tails (|z| up to 10 and beyond, where
    exp(-z^2) underflows) and a tangential momentum of size 1e-25: with no
    gradients the flux is the zeroth-order part alone, so the pair flux matches
    the oracle to the pairs' precision, the tiny component relative to itself."""
    def rows(rho, U, V, p):
        w = np.zeros((6, 4))
        w[0] = [rho, rho * U, rho * V, p / 0.4 + 0.5 * rho * (U * U + V * V)]
        return w
    Us = (-12.0, -6.0, -3.0, 0.0, 3.0, 6.0, 12.0)
    wl = np.stack([rows(1.1, U, 1e-25, 0.6) for U in Us])
    wr = np.stack([rows(0.9, U, 2e-25, 0.5) for U in Us])
    dt = 0.002
    got = host(G.point_flux(dev(wl), dev(wr), dt, precision=G.MIXED))
    ref = np.stack([O.point_flux(wl[q], wr[q], dt)[0] for q in range(len(Us))])
    for q in range(len(Us)):
        big = [0, 1, 3]
        sc = np.max(np.abs(ref[q, big]))
        assert np.max(np.abs(got[q, big] - ref[q, big])) <= 1e-12 * sc, (q, got[q], ref[q])
        assert abs(got[q, 2] - ref[q, 2]) <= 1e-11 * abs(ref[q, 2]), (q, got[q, 2], ref[q, 2])


@pytest.mark.parametrize("name", ["advection20", "shock_vortex40x20", "walled13x9"])
def test_pair_flux_kernel_matches_fp64_lead_kernels(G, name):
    """Face fluxes of the double-FP32 kernel against the FP64-lead kernels
    (warp-specialised and single-role) on the same coefficients: every face
    within 1e-8 of the flux scale (the slope-carrying part is FP32 in all three,
    contracted differently by the compiler)."""
    from tests.test_gpu_parity import CASES
    c = CASES[name]()
    w = dev(c.w0)
    out = {}
    for lead, split in ((1, 1), (0, 1), (0, 0)):
        m = G.GksMesh(c.mesh, precision=G.MIXED, flux_lead=lead, flux_split=split)
        coef, info = m.cls_reconstruct(w)
        dt = 0.5 * m.cfl_dt(w)
        out[(lead, split)] = host(m.flux(w, coef, dt)[0])
    ref = out[(0, 1)]
    scale = np.max(np.abs(ref), axis=1, keepdims=True)
    for k in ((1, 1), (0, 0)):
        assert np.all(np.abs(out[k] - ref) <= 1e-8 * scale), (k, np.max(np.abs(out[k] - ref) / scale))
