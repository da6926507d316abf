// Double-FP32 ("double-word") arithmetic: a value is an unevaluated sum
// hi + lo of two FP32 numbers with |lo| <= ulp(hi) / 2, about 48 significant
// bits.  GB300 runs FP64 at 1/64 of the FP32 rate, so the parts of the mixed
// face flux that need more than FP32 (the interface state, the collision time
// and the zeroth-order flux terms) run in this arithmetic on the FP32 pipe.
//
// Building blocks: Knuth's TwoSum, Dekker's FastTwoSum and the exact product
// by a fused multiply-add; sums and products of pairs follow the algorithms of
// M. Joldes, J.-M. Muller and V. Popescu, "Tight and rigorous error bounds for
// basic building blocks of double-word arithmetic", ACM TOMS 44 (2017):
// AccurateDWPlusDW (relative error < 3u^2, u = 2^-24), DWPlusFP, DWTimesDW3
// (< 4u^2) and DWTimesFP3 (< 2u^2).  Division and square root take one FP32
// step and correct it with the remainder formed exactly (Dekker 1971).  Every
// operation is written with the _rn intrinsics so that the compiler neither
// contracts nor reorders the error-free transforms.
//
// exp: Cody-Waite reduction by ln 2 (three-part constant), a further 2^-4
// scaling, the Taylor series of expm1 (leading terms in pairs, the tail in
// FP32) and four squarings in expm1 form, (1 + e)^2 - 1 = e (2 + e).
// erfcx(y) = exp(y^2) erfc(y), 0 <= y <= 10: the polynomial in Weideman's
// variable Z = (L - y) / (L + y) of gks_erfcx_coef.h (written by
// gen_erfcx_coef.py), evaluated by Horner's rule (leading 14 coefficients in
// pairs, the tail in FP32).
#pragma once

#include <cuda_runtime.h>

#include "gks_erfcx_coef.h"

namespace gks {
namespace dfm {

struct df {
    float hi, lo;
};

// the pair nearest to a double (host and device; on the device this uses the
// FP64 pipe: for constants and the conversion kernel only)
__host__ __device__ inline df from_double(double x)
{
    const float h = (float)x;
    return {h, (float)(x - (double)h)};
}

__device__ __forceinline__ double to_double(df x) { return (double)x.hi + (double)x.lo; }

__device__ __forceinline__ df two_sum(float a, float b)
{
    const float s = __fadd_rn(a, b);
    const float bb = __fsub_rn(s, a);
    const float e = __fadd_rn(__fsub_rn(a, __fsub_rn(s, bb)), __fsub_rn(b, bb));
    return {s, e};
}

// requires |a| >= |b| (or a = 0)
__device__ __forceinline__ df fast_two_sum(float a, float b)
{
    const float s = __fadd_rn(a, b);
    return {s, __fsub_rn(b, __fsub_rn(s, a))};
}

__device__ __forceinline__ df two_prod(float a, float b)
{
    const float p = __fmul_rn(a, b);
    return {p, __fmaf_rn(a, b, -p)};
}

__device__ __forceinline__ df neg(df x) { return {-x.hi, -x.lo}; }
__device__ __forceinline__ df dabs(df x) { return x.hi < 0.0f ? neg(x) : x; }

// AccurateDWPlusDW
__device__ __forceinline__ df add(df x, df y)
{
    const df s = two_sum(x.hi, y.hi);
    const df t = two_sum(x.lo, y.lo);
    const df v = fast_two_sum(s.hi, __fadd_rn(s.lo, t.hi));
    return fast_two_sum(v.hi, __fadd_rn(t.lo, v.lo));
}

__device__ __forceinline__ df sub(df x, df y) { return add(x, neg(y)); }

// DWPlusFP
__device__ __forceinline__ df add(df x, float y)
{
    const df s = two_sum(x.hi, y);
    return fast_two_sum(s.hi, __fadd_rn(x.lo, s.lo));
}

// DWTimesDW3
__device__ __forceinline__ df mul(df x, df y)
{
    const df c = two_prod(x.hi, y.hi);
    const float tl0 = __fmul_rn(x.lo, y.lo);
    const float tl1 = __fmaf_rn(x.hi, y.lo, tl0);
    const float cl2 = __fmaf_rn(x.lo, y.hi, tl1);
    return fast_two_sum(c.hi, __fadd_rn(c.lo, cl2));
}

// DWTimesFP3
__device__ __forceinline__ df mul(df x, float y)
{
    const df c = two_prod(x.hi, y);
    return fast_two_sum(c.hi, __fmaf_rn(x.lo, y, c.lo));
}

// exact scaling by a power of two p (no overflow or underflow)
__device__ __forceinline__ df scale2(df x, float p) { return {__fmul_rn(x.hi, p), __fmul_rn(x.lo, p)}; }

// x / y: q1 = x.hi / y.hi (reciprocal times numerator), the remainder
// x - q1 y formed exactly up to its own rounding, q2 = remainder / y.hi.
__device__ __forceinline__ df div(df x, df y)
{
    const float r = __frcp_rn(y.hi);
    const float q1 = __fmul_rn(x.hi, r);
    const df p = two_prod(q1, y.hi);
    float e = __fsub_rn(x.hi, p.hi);            // exact: p.hi is within a few ulp of x.hi
    e = __fsub_rn(e, p.lo);
    e = __fadd_rn(e, x.lo);
    e = __fmaf_rn(-q1, y.lo, e);
    return fast_two_sum(q1, __fmul_rn(e, r));
}

__device__ __forceinline__ df recip(df y)
{
    const float r = __frcp_rn(y.hi);
    const df p = two_prod(r, y.hi);
    float e = __fsub_rn(1.0f, p.hi);
    e = __fsub_rn(e, p.lo);
    e = __fmaf_rn(-r, y.lo, e);
    return fast_two_sum(r, __fmul_rn(e, r));
}

// sqrt(x), x > 0
__device__ __forceinline__ df sqrt(df x)
{
    const float s = __fsqrt_rn(x.hi);
    const df p = two_prod(s, s);
    float e = __fsub_rn(x.hi, p.hi);            // exact
    e = __fsub_rn(e, p.lo);
    e = __fadd_rn(e, x.lo);
    return fast_two_sum(s, __fmul_rn(e, __fmul_rn(0.5f, __frcp_rn(s))));
}

// The pair nearest to a double by integer operations (no FP64 instruction):
// hi = x rounded to FP32 (to nearest, ties to even), lo = x - hi rounded to
// FP32 (x - hi has at most 29 significant bits: an exact integer times a power
// of two).  Magnitudes outside the FP32 normal range [2^-126, 2^128) (zero,
// tiny, huge, non-finite) take the FP64 conversion.
__device__ __forceinline__ df split_double(double x)
{
    const unsigned long long b = (unsigned long long)__double_as_longlong(x);
    const int e = (int)((b >> 52) & 0x7ffu) - 1023;
    if (e < -126 || e > 127) return from_double(x);
    const unsigned long long m = b & 0xfffffffffffffull;
    const unsigned r = (unsigned)(m & 0x1fffffffull);             // the 29 bits below hi's mantissa
    const unsigned mh = (unsigned)(m >> 29);
    const bool up = r > 0x10000000u || (r == 0x10000000u && (mh & 1u));
    const unsigned sgn = (unsigned)(b >> 32) & 0x80000000u;
    const unsigned hb = ((((unsigned)(e + 127)) << 23) + mh + (up ? 1u : 0u)) | sgn;
    const int rem = (int)r - (up ? 0x20000000 : 0);                 // x - hi = rem 2^(e - 52) (sign aside)
    float lo = __int2float_rn(rem);
    if (e >= -74) {
        lo = __fmul_rn(lo, __int_as_float((e - 52 + 127) << 23));
    } else {
        lo = __fmul_rn(lo, __int_as_float((e - 52 + 64 + 127) << 23));
        lo = __fmul_rn(lo, __int_as_float((127 - 64) << 23));
    }
    return {__int_as_float((int)hb), sgn ? -lo : lo};
}

// Sum of products w + sum_k u_k phi_k: the pairs' high products exact by FMA,
// the cross terms in FP32, every term added to one running FP32 sum by TwoSum
// and the errors collected in a second word; normalised once at the end (by
// TwoSum: the sum may cancel down to the size of the collected errors).
struct Acc {
    float s, c;
};

__device__ __forceinline__ Acc acc_start(df w) { return {w.hi, w.lo}; }

__device__ __forceinline__ void acc_prod(Acc &a, df u, df phi)
{
    const float p = __fmul_rn(u.hi, phi.hi);
    float pe = __fmaf_rn(u.hi, phi.hi, -p);
    pe = __fmaf_rn(u.hi, phi.lo, pe);
    pe = __fmaf_rn(u.lo, phi.hi, pe);
    const df t = two_sum(a.s, p);
    a.s = t.hi;
    a.c = __fadd_rn(a.c, __fadd_rn(t.lo, pe));
}

__device__ __forceinline__ df acc_end(const Acc &a) { return two_sum(a.s, a.c); }

// ---- exp

// Cody-Waite split of ln 2: kLn2A has 15 significant bits, so k kLn2A is exact
// for |k| < 2^9; kLn2A + kLn2B + kLn2C = ln 2 to 1.3e-21.
constexpr float kLn2A = 0.693145751953125f, kLn2B = 1.428606765330187e-06f, kLn2C = 5.497923148104107e-14f;
constexpr float kLog2e = 1.4426950408889634f;
constexpr float kSixthHi = 0.1666666716337204f, kSixthLo = -4.967053879312289e-09f;
constexpr float kInv24Hi = 0.0416666679084301f, kInv24Lo = -1.241763469828072e-09f;

// e with exp(r) = 1 + e, |r| <= 0.35
__device__ __forceinline__ df expm1_small(df r)
{
    const df s = scale2(r, 0.0625f);            // |s| <= 0.022
    const float sh = s.hi;
    // s^5/120 + s^6/720 + s^7/5040 relative to s^4: t = 1/120 + s/720 + s^2/5040 (FP32)
    const float t = __fmaf_rn(__fmaf_rn(sh, 1.0f / 5040.0f, 1.0f / 720.0f), sh, 1.0f / 120.0f);
    // e(s) = s (1 + s (1/2 + s (1/6 + s (1/24 + s t))))
    df q = add(df{kInv24Hi, kInv24Lo}, __fmul_rn(sh, t));
    q = add(mul(q, s), df{kSixthHi, kSixthLo});
    q = add(mul(q, s), 0.5f);
    q = add(mul(q, s), 1.0f);
    df e = mul(q, s);
#pragma unroll 1
    for (int k = 0; k < 4; ++k) e = mul(e, add(e, 2.0f));     // (1 + e)^2 - 1
    return e;
}

// exp(x) for x <= 88; results below 2^-126 are flushed to zero
__device__ __forceinline__ df exp(df x)
{
    if (x.hi < -87.0f) return {0.0f, 0.0f};
    const float k = rintf(__fmul_rn(x.hi, kLog2e));
    df r = two_sum(__fmaf_rn(-k, kLn2A, x.hi), x.lo);
    r = add(r, two_prod(-k, kLn2B));
    r = add(r, __fmul_rn(-k, kLn2C));
    const df e = expm1_small(r);
    const df one_e = add(e, 1.0f);
    const float p = __int_as_float(((int)k + 127) << 23);      // 2^k, k in [-126, 127]
    return scale2(one_e, p);
}

// exp(x) - 1 for |x| <= 0.35 directly (no cancellation), else exp(x) - 1
__device__ __forceinline__ df expm1(df x)
{
    if (fabsf(x.hi) <= 0.34f) return expm1_small(x);
    return add(exp(x), -1.0f);
}

// ---- erfcx(y) = exp(y^2) erfc(y), 0 <= y <= 10
__device__ __forceinline__ df erfcx(df y)
{
    const df Z = div(add(neg(y), kErfcxL), add(y, kErfcxL));
    const df s = add(mul(add(Z, df{-kErfcxZminHi, -kErfcxZminLo}), df{kErfcxScaleHi, kErfcxScaleLo}), -1.0f);
    constexpr int kHead = 14;                  // coefficients 0..13 in pairs
    float t = kErfcxHi[kErfcxDeg];
#pragma unroll
    for (int k = kErfcxDeg - 1; k >= kHead; --k) t = __fmaf_rn(t, s.hi, kErfcxHi[k]);
    df p = {t, 0.0f};
    // a rolled loop: the code of the flux kernel that calls this twice is
    // large enough for instruction fetch to stall it
#pragma unroll 1
    for (int k = kHead - 1; k >= 0; --k) p = add(mul(p, s), df{kErfcxHi[k], kErfcxLo[k]});
    return p;
}

}  // namespace dfm
}  // namespace gks
