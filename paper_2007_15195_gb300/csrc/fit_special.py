"""Fit the FP32 normal CDF and quantile used by the mixed-precision Genz kernel.

Writes special_f32.cuh (coefficient tables) next to this script.  The forms
are published ones; the coefficients are fitted here, from the mathematics,
against scipy's double-precision erfcx / erfinv / ndtri:

  Phi of the lower tail (the form of the Numerical Recipes routine "erfcc",
  a Chebyshev-fitted exponent around a rational factor):
      Phi(-z) = t * 2^(-z^2 log2(e)/2 + P(t)),   t = 1 / (1 + z / (2 sqrt 2)),  z >= 0,
      P a polynomial in t on t in [1/(1 + 38/(2 sqrt 2)), 1] (z in [0, 38]).

  Phi^{-1} of the lower tail through erfinv (M. Giles, "Approximating the
  erfinv function", GPU Computing Gems Jade Edition, 2011):
      Phi^{-1}(r) = -sqrt(2) y f(w),  y = 1 - 2r,  w = -ln(4 r (1 - r)),
      f(w) = erfinv(y) / y, a polynomial in w on [0, 8] (r > 8.4e-5, the
      branch almost every lane takes), in sqrt(w) on [8, 36] and on [36, 130]
      and [130, 700] (the last two reached for r < 5e-17, mostly from
      log-space inputs).

The quantile pieces are emitted multiplied by sqrt(2), so that
Phi^{-1}(p) = (p - q) f_s(w) with f_s = sqrt(2) f and q = 1 - p on either
side of 1/2; the first piece also gets the map from L = log2(r (1 - r)) (so
w = -ln 2 (L + 2)) folded into its variable, u = a' L + b'.

Each piece is a polynomial in a variable mapped to [-1, 1], fitted in the
Chebyshev basis by Lawson's iteratively reweighted least squares toward the
minimax relative error, then expanded to monomials for Horner evaluation.
Run:  python fit_special.py   (prints the max relative error of each piece
evaluated in float32 arithmetic).
"""
import os

import numpy as np
from numpy.polynomial import chebyshev as C
from numpy.polynomial import polynomial as P
from scipy import special

HERE = os.path.dirname(os.path.abspath(__file__))
OUT = os.path.join(HERE, "special_f32.cuh")
LOG2E = 1.4426950408889634
K_T = 1.0 / (2.0 * np.sqrt(2.0))  # t = 1 / (1 + z K_T)
Z_MAX = 38.0
W1_HI = 8.0  # first quantile piece: w in [0, 8], i.e. r > 8.4e-5


def lawson_cheb(u, f, deg, iters=60, rel=True):
    """Chebyshev fit on u in [-1,1] minimising max |err| (relative if rel)."""
    V = C.chebvander(u, deg)
    scale = np.abs(f) if rel else np.ones_like(f)
    w = np.full(u.shape, 1.0 / u.size)
    for _ in range(iters):
        sw = np.sqrt(w) / scale
        c, *_ = np.linalg.lstsq(V * sw[:, None], f * sw, rcond=None)
        err = (V @ c - f) / scale
        w = w * np.abs(err) + 1e-30
        w /= w.sum()
    return c, float(np.max(np.abs(err)))


def to_monomial(c):
    return C.cheb2poly(c)


def horner_f32(coef, u):
    """Evaluate a monomial polynomial in float32 with one rounding per fma."""
    u64 = u.astype(np.float32).astype(np.float64)
    cf = coef.astype(np.float32).astype(np.float64)
    acc = np.full(u.shape, cf[-1])
    for a in cf[-2::-1]:
        acc = (acc * u64 + a).astype(np.float32).astype(np.float64)
    return acc


def fit_phi(deg=9):
    z = np.linspace(0.0, Z_MAX, 200001)
    t = 1.0 / (1.0 + z * K_T)
    tlo, thi = 1.0 / (1.0 + Z_MAX * K_T), 1.0
    u = (2.0 * t - (thi + tlo)) / (thi - tlo)
    # log2 Phi(-z) = log2(erfcx(z/sqrt2)/2) - z^2 log2(e)/2
    target = np.log2(0.5 * special.erfcx(z / np.sqrt(2.0))) - np.log2(t)
    c, err = lawson_cheb(u, target, deg, rel=False)
    # expanded from u = a t + b into monomials of t itself (coefficients of
    # magnitude <= 3 on t in [0.07, 1]: no cancellation to speak of), so the
    # kernel needs no map of t
    a, b = 2.0 / (thi - tlo), -(thi + tlo) / (thi - tlo)
    mono_u = to_monomial(c)
    mono = np.zeros(1)
    for k in range(len(mono_u) - 1, -1, -1):
        mono = P.polyadd(P.polymul(mono, [b, a]), [mono_u[k]])
    got = horner_f32(mono, t)
    err32 = float(np.max(np.abs(got - target))) * np.log(2.0)  # relative error of Phi
    return dict(name="PHI", a=1.0, b=0.0, coef=mono, fit_err=err * np.log(2.0), f32_err=err32,
                note="log2 exponent as a polynomial in t itself; relative error of Phi")


def finv_target(w):
    y = np.sqrt(-np.expm1(-w))
    r = np.exp(-w) / (1.0 + y) / 2.0  # (1 - y) / 2
    ei = np.where(w < 5.0, special.erfinv(np.minimum(y, 1 - 1e-16)), -special.ndtri(r) / np.sqrt(2.0))
    return ei / y


def fit_inv(name, lo, hi, var, deg):
    w = np.linspace(lo, hi, 200001)
    w[0] = max(w[0], 1e-14)
    f = finv_target(w)
    x = w if var == "w" else np.sqrt(w)
    xlo, xhi = (lo, hi) if var == "w" else (np.sqrt(lo), np.sqrt(hi))
    u = (2.0 * x - (xhi + xlo)) / (xhi - xlo)
    c, err = lawson_cheb(u, f, deg, rel=True)
    mono = to_monomial(c) * np.sqrt(2.0)
    got = horner_f32(mono, u)
    err32 = float(np.max(np.abs(got - f * np.sqrt(2.0)) / np.abs(f * np.sqrt(2.0))))
    return dict(name=name, a=2.0 / (xhi - xlo), b=-(xhi + xlo) / (xhi - xlo), coef=mono, fit_err=err,
                f32_err=err32, note="sqrt(2) erfinv(y)/y on %s in [%g, %g]" % (var, xlo, xhi))


def fit_inv1_scaled(deg=10):
    """The central quantile piece for callers that carry 16 p and 16 q.

    With pk = 16 p and qk = 16 q (exact power-of-two scalings of p and q),
    L' = log2(pk qk) = log2(r (1 - r)) + 8 and w = -ln 2 (L' - 6).  Fitted on
    w in [0, 12 ln 2], the map to [-1, 1] is u = -L'/6 with no offset, so the
    polynomial is re-expressed in L' itself (coefficients c_k (-1/6)^k) and
    divided by 16: Phi^{-1}(p) = (pk - qk) f16(L') needs no map of L'."""
    hi = 12.0 * np.log(2.0)
    p = fit_inv("INV1S", 0.0, hi, "w", deg)
    k = np.arange(len(p["coef"]))
    coef = p["coef"] * (-1.0 / 6.0) ** k / 16.0
    w = np.linspace(0.0, hi, 200001)
    w[0] = 1e-14
    Lp = (6.0 - w / np.log(2.0)).astype(np.float32).astype(np.float64)
    got = horner_f32(coef, Lp)
    f = finv_target(w) * np.sqrt(2.0) / 16.0
    err32 = float(np.max(np.abs(got - f) / np.abs(f)))
    return dict(name="INV1S", a=1.0, b=0.0, coef=coef, fit_err=p["fit_err"], f32_err=err32,
                note="sqrt(2) erfinv(y)/y / 16 as a polynomial in L' = log2(256 r (1-r)), w in [0, %g]" % hi)


def emit(pieces):
    lines = [
        "// special_f32.cuh -- generated by fit_special.py; do not edit by hand.",
        "// Coefficients of the FP32 normal CDF / quantile pieces used by the mixed",
        "// Genz kernel (forms and fitting method described in fit_special.py).",
        "// Each piece: u = a*x + b maps its interval to [-1, 1]; value = sum_k c_k u^k.",
        "#pragma once",
        "",
        "namespace vk {",
        "namespace special {",
        "",
        "constexpr float kLog2e = 1.44269504088896341f;",
        "constexpr float kKt = %.9ef;  // t = 1 / (1 + z kKt)" % K_T,
        "constexpr float kZmax = %.1ff;" % Z_MAX,
        "",
    ]
    inv1 = [p for p in pieces if p["name"] == "INV1"][0]
    ln2 = np.log(2.0)
    lines.append("// INV1 from L = log2(r (1-r)): u = kINV1LA L + kINV1LB, valid for L > kINV1Lmin")
    lines.append("constexpr float kINV1LA = %.9ef, kINV1LB = %.9ef, kINV1Lmin = %.9ef;" % (
        -inv1["a"] * ln2, inv1["b"] - 2.0 * inv1["a"] * ln2, -W1_HI / ln2 - 2.0))
    lines.append("")
    lines.append("// INV1S from L' = log2(256 r (1-r)), Horner in L' itself, valid for L' > kINV1SLmin")
    lines.append("constexpr float kINV1SLmin = -6.0f;")
    lines.append("")
    for p in pieces:
        lines.append("// %s: %s; fit max error %.2e, in float32 %.2e" % (p["name"], p["note"], p["fit_err"],
                                                                         p["f32_err"]))
        lines.append("constexpr float k%sA = %.9ef, k%sB = %.9ef;" % (p["name"], p["a"], p["name"], p["b"]))
        cs = ", ".join("%.9ef" % v for v in p["coef"])
        lines.append("constexpr int k%sN = %d;" % (p["name"], len(p["coef"])))
        lines.append("__device__ constexpr float k%sC[%d] = {%s};" % (p["name"], len(p["coef"]), cs))
        lines.append("")
    lines += ["}  // namespace special", "}  // namespace vk", ""]
    with open(OUT, "w") as f:
        f.write("\n".join(lines))


def main():
    pieces = [
        fit_phi(9),
        fit_inv("INV1", 0.0, W1_HI, "w", 10),
        fit_inv1_scaled(10),
        fit_inv("INV2", W1_HI, 36.0, "s", 9),
        fit_inv("INV3", 36.0, 130.0, "s", 8),
        fit_inv("INV4", 130.0, 700.0, "s", 8),
    ]
    for p in pieces:
        print("%-5s fit %.3e  float32 %.3e  (%s)" % (p["name"], p["fit_err"], p["f32_err"], p["note"]))
    emit(pieces)
    print("wrote", OUT)


if __name__ == "__main__":
    main()
