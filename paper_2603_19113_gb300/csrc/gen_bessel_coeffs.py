"""Generate the modulus/phase fits of H0^(1) used by the device code.

For x >= xa write H0^(1)(x) = M(x) exp(i theta(x)) and
    f(x) = M(x) sqrt(pi x / 2),     g(x) = theta(x) - (x - pi/4),
both smooth functions of t = xa / x in (0, 1] tending to f = 1, g = 0 as
x -> infinity (Hankel's asymptotic form, DLMF 10.17.1 / 10.18).  Each is fitted
by a Chebyshev series in u = 2 t - 1 on [-1, 1] from high-precision values of
J0 and Y0 (mpmath), and written out as monomial coefficients in u, highest
degree first, for Horner evaluation.

Run:  python gen_bessel_coeffs.py > bessel_coeffs.h
"""
import sys

import mpmath as mp
import numpy as np
import numpy.polynomial.chebyshev as C

mp.mp.dps = 40

# (name, xa, degree, precision)
FITS = [
    ("F32_X64", 64.0, 2, "float"),
    ("F32_X8", 8.0, 4, "float"),
    ("F32_X3", 3.0, 6, "float"),
    ("F64_X4", 4.0, 20, "double"),
    ("F64_X16", 16.0, 10, "double"),
    ("F64_X64", 64.0, 6, "double"),
]


def fg(x):
    x = mp.mpf(x)
    h = mp.besselj(0, x) + 1j * mp.bessely(0, x)
    f = abs(h) * mp.sqrt(mp.pi * x / 2)
    g = mp.arg(h) - (x - mp.pi / 4)
    g = g - 2 * mp.pi * mp.nint(g / (2 * mp.pi))
    return float(f), float(g)


def fit(xa, deg, nodes=160):
    k = np.arange(nodes)
    u = np.cos(np.pi * (k + 0.5) / nodes)
    t = (u + 1.0) / 2.0
    vals = [fg(xa / tt) for tt in t]
    F = np.array([v[0] for v in vals])
    G = np.array([v[1] for v in vals])
    cf = C.cheb2poly(C.chebfit(u, F, deg))
    cg = C.cheb2poly(C.chebfit(u, G, deg))
    # check on an independent grid
    tt = np.linspace(1e-6, 1.0, 257)
    ref = [fg(xa / s) for s in tt]
    uu = 2 * tt - 1
    ef = max(abs(np.polyval(cf[::-1], uu) / np.array([r[0] for r in ref]) - 1))
    eg = max(abs(np.polyval(cg[::-1], uu) - np.array([r[1] for r in ref])))
    return cf[::-1], cg[::-1], ef, eg


def main(out=sys.stdout):
    out.write("// Generated by gen_bessel_coeffs.py: modulus/phase fits of H0^(1).\n")
    out.write("// f(x) = |H0(x)| sqrt(pi x / 2), g(x) = arg H0(x) - (x - pi/4), for x >= XA,\n")
    out.write("// polynomials in u = 2 XA / x - 1, highest degree first (Horner).\n")
    out.write("#pragma once\n\n")
    for name, xa, deg, prec in FITS:
        cf, cg, ef, eg = fit(xa, deg)
        suf = "f" if prec == "float" else ""
        out.write(f"// {name}: x >= {xa}, degree {deg}; max rel. error of f {ef:.2e}, "
                  f"max abs. error of g {eg:.2e}\n")
        out.write(f"#define MBS_{name}_XA {xa!r}{suf}\n")
        out.write(f"#define MBS_{name}_DEG {deg}\n")
        for lab, cc in (("F", cf), ("G", cg)):
            body = ", ".join(f"{c:.17e}{suf}" for c in cc)
            out.write(f"#define MBS_{name}_{lab} {{{body}}}\n")
        out.write("\n")


if __name__ == "__main__":
    main()
