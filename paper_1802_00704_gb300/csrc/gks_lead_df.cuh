// The parts of the mixed-precision face flux that need more than FP32, in
// double-FP32 arithmetic (gks_df.cuh) on the FP32 pipe: the Gauss-point values
// of the reconstruction, the interface equilibrium W0 of the half-space moments
// (Sec. II.B, after Eq. (15)), its primitive state, the collision time
// (Eqs. (39)-(40)), the time integrals of c1 and c7 (Eq. (13)) and the
// zeroth-order flux terms C1 rho0 <u psi>_0 + C7 (rho_l <u psi>_{u>0} +
// rho_r <u psi>_{u<0}).  The slope-carrying terms stay in FP32
// (kin::gp_body_mixed), formed from the FP32 roundings of these values.
#pragma once

#include "gks_df.cuh"

namespace gks {
namespace lead {

using dfm::df;

struct LeadConst {
    df gm1;        // gamma - 1
    df igm1;       // 1 / (gamma - 1)
    df K;          // internal degrees of freedom, 2 / (gamma - 1) - 2
    df kp1;        // K + 1
    df mu;         // viscosity (0: the inviscid collision time)
    df c001;       // 0.01, the inviscid collision time's base factor
    df hisp;       // 1 / (2 sqrt(pi))
};

struct State {
    df rho, U, V, p, h;    // h = p / rho = 1 / (2 lambda), Eq. (3)
};

// Primitive state of (rho, rho U, rho V, E); false unless rho > 0 and p > 0.
__device__ __forceinline__ bool prim(const df *w, const LeadConst &c, State &s)
{
    s.rho = w[0];
    const df ir = dfm::recip(w[0]);
    s.U = dfm::mul(w[1], ir);
    s.V = dfm::mul(w[2], ir);
    const df ke = dfm::scale2(dfm::add(dfm::mul(w[1], s.U), dfm::mul(w[2], s.V)), 0.5f);
    s.p = dfm::mul(dfm::sub(w[3], ke), c.gm1);
    s.h = dfm::mul(s.p, ir);
    return s.rho.hi > 0.0f && s.p.hi > 0.0f;
}

// Half-space moments <u^k>, k = 0..3, of the 1-D Maxwellian sqrt(lambda/pi)
// exp(-lambda (u - U)^2) over u > 0 (sign = +1) or u < 0 (sign = -1):
// <1> = erfc(z) / 2 with z = -sign sqrt(lambda) U, erfc(|z|) = exp(-z^2)
// erfcx(|z|); <u> = U <1> + sign exp(-z^2) / (2 sqrt(pi lambda));
// <u^{k+2}> = U <u^{k+1}> + (k + 1) h <u^k>.
__device__ __forceinline__ void half_moments(const State &s, float sign, const LeadConst &c, df *m)
{
    const df h2 = dfm::scale2(s.h, 2.0f);              // 1 / lambda
    const df rs = dfm::sqrt(h2);                        // 1 / sqrt(lambda)
    df z = dfm::div(s.U, rs);
    if (sign > 0.0f) z = dfm::neg(z);
    const df ex = dfm::exp(dfm::neg(dfm::mul(z, z)));
    df y = dfm::dabs(z);
    if (y.hi > 10.0f) y = {10.0f, 0.0f};                // exp(-z^2) is below 2^-126 there
    const df half_erfc = dfm::scale2(dfm::mul(ex, dfm::erfcx(y)), 0.5f);
    m[0] = z.hi >= 0.0f ? half_erfc : dfm::add(dfm::neg(half_erfc), 1.0f);
    const df g = dfm::mul(dfm::mul(ex, rs), c.hisp);    // exp(-z^2) / (2 sqrt(pi lambda))
    m[1] = dfm::add(dfm::mul(s.U, m[0]), sign > 0.0f ? g : dfm::neg(g));
    m[2] = dfm::add(dfm::mul(s.U, m[1]), dfm::mul(s.h, m[0]));
    m[3] = dfm::add(dfm::mul(s.U, m[2]), dfm::mul(h2, m[1]));
}

struct Lead {
    df f[4];       // zeroth-order flux terms
    df w0[4];      // interface state
    df tau;        // collision time
    df c0c6;       // HEAT: C1 + C7 integrals (the zeroth-order <psi f> is (C0 + C6) w0)
    df zu, zv;     // HEAT: interface velocity
};

// vl, vr: face-frame values (rho, rho U, rho V, E); false if a state is not physical
__device__ __forceinline__ bool gp_lead(const df *vl, const df *vr, df dt, const LeadConst &c, Lead &o)
{
    State L, R, Z;
    if (!(prim(vl, c, L) & prim(vr, c, R))) return false;
    df ml[4], mr[4];
    // one copy of the (large) half-moment code for both sides: the flux kernel
    // is long enough for instruction fetch to stall it
#pragma unroll 1
    for (int side = 0; side < 2; ++side) {
        df m[4];
        half_moments(side ? R : L, side ? -1.0f : 1.0f, c, m);
        if (side) {
#pragma unroll
            for (int q = 0; q < 4; ++q) mr[q] = m[q];
        } else {
#pragma unroll
            for (int q = 0; q < 4; ++q) ml[q] = m[q];
        }
    }
    // W0 = rho_l <psi>_{u>0} + rho_r <psi>_{u<0}; <e> = (<u^2> + <1>(V^2 + (K + 1) h)) / 2
    const df lm0 = dfm::mul(L.rho, ml[0]), rm0 = dfm::mul(R.rho, mr[0]);
    const df lm1 = dfm::mul(L.rho, ml[1]), rm1 = dfm::mul(R.rho, mr[1]);
    const df lm2 = dfm::mul(L.rho, ml[2]), rm2 = dfm::mul(R.rho, mr[2]);
    const df al = dfm::add(dfm::mul(L.V, L.V), dfm::mul(L.h, c.kp1));
    const df ar = dfm::add(dfm::mul(R.V, R.V), dfm::mul(R.h, c.kp1));
    df *w0 = o.w0;
    w0[0] = dfm::add(lm0, rm0);
    w0[1] = dfm::add(lm1, rm1);
    w0[2] = dfm::add(dfm::mul(lm0, L.V), dfm::mul(rm0, R.V));
    w0[3] = dfm::scale2(dfm::add(dfm::add(lm2, dfm::mul(lm0, al)), dfm::add(rm2, dfm::mul(rm0, ar))), 0.5f);
    if (!prim(w0, c, Z)) return false;
    // collision time, Eqs. (39)-(40), the pressure-jump term times dt
    const df jump = dfm::div(dfm::dabs(dfm::sub(L.p, R.p)), dfm::dabs(dfm::add(L.p, R.p)));
    o.tau = c.mu.hi > 0.0f ? dfm::add(dfm::div(c.mu, Z.p), dfm::mul(dt, jump)) : dfm::mul(dt, dfm::add(jump, c.c001));
    // integrals over [0, dt] of c1 and c7: C6 = tau (1 - e^{-x}), C0 = dt - C6, x = dt / tau
    const df x = dfm::div(dt, o.tau);
    const df t0 = dfm::neg(dfm::expm1(dfm::neg(x)));
    const df C6 = dfm::mul(o.tau, t0);
    const df C0 = dfm::mul(o.tau, dfm::sub(x, t0));
    // C0 rho0 <u psi>_0: <u^2> = U^2 + h, <u^3> = U (U^2 + 3 h), <u (v^2 + xi^2)> = U (V^2 + (K + 1) h)
    const df s0 = dfm::mul(C0, Z.rho);
    const df m2z = dfm::add(dfm::mul(Z.U, Z.U), Z.h);
    const df m3z = dfm::mul(Z.U, dfm::add(m2z, dfm::scale2(Z.h, 2.0f)));
    const df az = dfm::add(dfm::mul(Z.V, Z.V), dfm::mul(Z.h, c.kp1));
    const df su = dfm::mul(s0, Z.U);
    // C7 (rho_l <u psi>_{u>0} + rho_r <u psi>_{u<0})
    const df lm3 = dfm::mul(L.rho, ml[3]), rm3 = dfm::mul(R.rho, mr[3]);
    o.f[0] = dfm::add(su, dfm::mul(C6, w0[1]));
    o.f[1] = dfm::add(dfm::mul(s0, m2z), dfm::mul(C6, dfm::add(lm2, rm2)));
    o.f[2] = dfm::add(dfm::mul(su, Z.V), dfm::mul(C6, dfm::add(dfm::mul(lm1, L.V), dfm::mul(rm1, R.V))));
    const df e0 = dfm::add(m3z, dfm::mul(Z.U, az));
    const df ek = dfm::add(dfm::add(lm3, dfm::mul(lm1, al)), dfm::add(rm3, dfm::mul(rm1, ar)));
    o.f[3] = dfm::scale2(dfm::add(dfm::mul(s0, e0), dfm::mul(C6, ek)), 0.5f);
    o.c0c6 = dfm::add(C0, C6);
    o.zu = Z.U;
    o.zv = Z.V;
    return true;
}

// Heat flux relative to the velocity (U, V) from the flux moments F = <u psi f>
// and D = <psi f>: <(1/2)(u - U)|c|^2 f> expanded in the moments (the same
// expansion as kin::heat_flux), in pairs.
__device__ __forceinline__ df heat_flux(const df *F, const df *D, df U, df V)
{
    using namespace dfm;
    const df q2 = add(mul(U, U), mul(V, V));
    df q = sub(F[3], add(mul(U, F[1]), mul(V, F[2])));
    q = add(q, mul(add(scale2(q2, 0.5f), mul(U, U)), F[0]));
    q = sub(q, mul(U, D[3]));
    q = add(q, mul(mul(U, V), D[2]));
    return sub(q, mul(scale2(mul(U, q2), 0.5f), D[0]));
}

}  // namespace lead
}  // namespace gks
