#!/usr/bin/env python
"""Writes gks_erfcx_coef.h: the coefficients of the double-FP32 scaled
complementary error function erfcx(y) = exp(y^2) erfc(y), 0 <= y <= 10, used by
the mixed-precision face flux for the half-space Maxwellian moments.

Method: erfcx is smooth in Weideman's variable Z = (L - y) / (L + y) (J. A. C.
Weideman, "Computation of the complex error function", SIAM J. Numer. Anal. 31
(1994) 1497-1518, which expands the complex error function in powers of this
variable); here erfcx(y(Z)) is interpolated at Chebyshev points of the image of
[0, 10] in Z and the interpolant is rewritten as a polynomial in the scaled
variable s = (2 Z - Zmin - 1) / (1 - Zmin) in [-1, 1].  mpmath evaluates erfc
at 60 digits.  Each coefficient is stored as an FP32 pair (hi, lo),
hi + lo = the coefficient to 2^-48 relative.  The script prints the largest
relative error of the polynomial (exact arithmetic) on 4001 points.

    python gen_erfcx_coef.py > gks_erfcx_coef.h
"""
import sys

import mpmath as mp
import numpy as np

mp.mp.dps = 60
L = mp.mpf(4)
YMAX = mp.mpf(10)
DEG = 20


def erfcx(y):
    return mp.exp(y * y) * mp.erfc(y)


def main():
    zmin = (L - YMAX) / (L + YMAX)
    zmax = mp.mpf(1)
    n = DEG + 1
    xs = [mp.cos(mp.pi * (k + mp.mpf(1) / 2) / n) for k in range(n)]
    zs = [zmin + (zmax - zmin) * (x + 1) / 2 for x in xs]
    fs = [erfcx(L * (1 - z) / (1 + z)) for z in zs]
    cheb = [2 * mp.fsum(fs[j] * mp.cos(mp.pi * i * (j + mp.mpf(1) / 2) / n) for j in range(n)) / n for i in range(n)]
    cheb[0] /= 2
    mono = [mp.mpf(0)] * n
    for i in range(n):
        for k, pk in enumerate(mp.taylor(lambda t: mp.chebyt(i, t), 0, i)):
            mono[k] += cheb[i] * pk
    err = mp.mpf(0)
    for y in np.linspace(0.0, float(YMAX), 4001):
        y = mp.mpf(y)
        z = (L - y) / (L + y)
        s = (2 * z - zmin - zmax) / (zmax - zmin)
        v = mp.fsum(mono[k] * s ** k for k in range(n))
        err = max(err, abs(v / erfcx(y) - 1))
    pairs = []
    for a in mono:
        hi = float(np.float32(float(a)))
        lo = float(np.float32(float(a - mp.mpf(hi))))
        pairs.append((hi, lo))
    out = sys.stdout
    out.write("// Generated by gen_erfcx_coef.py: erfcx(y) = exp(y^2) erfc(y) on 0 <= y <= 10 as a\n")
    out.write(f"// polynomial of degree {DEG} in s = (2 Z - Zmin - 1) / (1 - Zmin), Z = (L - y) / (L + y),\n")
    out.write(f"// L = {float(L)}, Zmin = (L - 10) / (L + 10); coefficient k as an FP32 pair (hi, lo).\n")
    out.write(f"// Largest relative error of the polynomial on 4001 points: {float(err):.2e}.\n")
    out.write("#pragma once\n\nnamespace gks {\nnamespace dfm {\n\n")
    out.write(f"constexpr float kErfcxL = {float(L):.1f}f;\n")
    out.write(f"constexpr int kErfcxDeg = {DEG};\n")
    zm = float(zmin)
    zh = float(np.float32(zm))
    out.write(f"constexpr float kErfcxZminHi = {zh!r}f, kErfcxZminLo = {float(np.float32(float(zmin - mp.mpf(zh))))!r}f;\n")
    inv = 2 / (zmax - zmin)
    ih = float(np.float32(float(inv)))
    out.write(f"constexpr float kErfcxScaleHi = {ih!r}f, kErfcxScaleLo = {float(np.float32(float(inv - mp.mpf(ih))))!r}f;\n")
    out.write("__device__ constexpr float kErfcxHi[kErfcxDeg + 1] = {\n")
    out.write(",\n".join(f"    {h!r}f" for h, _ in pairs))
    out.write("};\n__device__ constexpr float kErfcxLo[kErfcxDeg + 1] = {\n")
    out.write(",\n".join(f"    {lo!r}f" for _, lo in pairs))
    out.write("};\n\n}  // namespace dfm\n}  // namespace gks\n")


if __name__ == "__main__":
    main()
