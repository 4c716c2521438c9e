"""Tables of the FP64 normal tail used by the FP64 Genz kernel.

Writes special_f64.cuh next to this script.  The form: for a >= 0,

    Phi(-a) = exp(-a^2 / 2) R(a),   R(a) = erfcx(a / sqrt 2) / 2,

with R (smooth and slowly varying: 1/2 at 0, ~ 1/(a sqrt(2 pi)) for large a)
a piecewise polynomial and the Gaussian factor a table-driven exponential:

  * R on the intervals centred at a_i = i/8, |a - a_i| <= 1/16, i = 0..310
    (a < 38.75; beyond, Phi(-a) is below the smallest double): a degree-8
    polynomial in d = a - a_i per interval, fitted in the Chebyshev sense by
    mpmath (chebyfit) against R evaluated at 40 digits, rounded to doubles;
  * exp(x), x = -a^2/2 <= 0: k = round(x 256 / ln 2), r = x - k ln2/256 by
    Cody and Waite's two-constant reduction (the first constant has 34
    significant bits, so k times it is exact for |k| < 2^19), exp(r) by its
    Taylor polynomial to r^4 (|r| <= ln2/512: the dropped term is below
    4e-17), times 2^(j/256) (j = k mod 256, a table of 256 doubles) and 2^(k div 256).

Each table entry is the exact mathematical value rounded to the nearest
double (mpmath at 40 digits).  Run:  python fit_special64.py  (prints the
worst relative error of each R piece in exact arithmetic and in double
arithmetic without fused multiply-adds).
"""
import os

import mpmath as mp
import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))
OUT = os.path.join(HERE, "special_f64.cuh")
mp.mp.dps = 40

H = 0.125         # interval width in a
NINT = 311        # centres 0, 1/8, ..., 38.75
DEG = 8
EXP_BITS = 8      # 2^(j/256) table


def R(a):
    x = mp.mpf(a) / mp.sqrt(2)
    return mp.erfc(x) * mp.exp(x * x) / 2


def fit_R():
    rows, worst_exact, worst_f64 = [], 0.0, 0.0
    for i in range(NINT):
        c = mp.mpf(i) * H
        poly, err = mp.chebyfit(lambda d: R(c + d), [-H / 2, H / 2], DEG + 1, error=True)
        coef = [float(v) for v in reversed(poly)]  # c_0 .. c_DEG
        ds = np.linspace(-H / 2, H / 2, 257)
        if i == 0:
            ds = ds[ds >= 0]
        for d in ds:
            acc = coef[-1]
            for k in range(DEG - 1, -1, -1):
                acc = acc * float(d) + coef[k]
            ref = R(c + mp.mpf(float(d)))
            worst_f64 = max(worst_f64, float(abs((mp.mpf(acc) - ref) / ref)))
        worst_exact = max(worst_exact, float(err / R(c)))
        rows.append(coef + [float(-c), 0.0])  # offset: d = a + (-a_i)
    return rows, worst_exact, worst_f64


def exp_constants():
    step = mp.log(2) / 2 ** EXP_BITS
    hi = float(step)
    m, e = np.frexp(hi)
    hi = float(np.ldexp(np.floor(np.ldexp(m, 34)), e - 34))  # 34 significant bits
    lo = float(step - mp.mpf(hi))
    table = [float(mp.mpf(2) ** (mp.mpf(j) / 2 ** EXP_BITS)) for j in range(2 ** EXP_BITS)]
    inv = float(2 ** EXP_BITS / mp.log(2))
    return hi, lo, inv, table


def fmt(v):
    return "%.17e" % v


def emit(rows, hi, lo, inv, table, worst_exact, worst_f64):
    L = [
        "// special_f64.cuh -- generated by fit_special64.py; do not edit by hand.",
        "// Tables of the FP64 normal tail Phi(-a) = exp(-a^2/2) R(a) (form and",
        "// fitting method described in fit_special64.py).",
        "#pragma once",
        "",
        "namespace vk {",
        "namespace special64 {",
        "",
        "// R(a) on |a - i h| <= h/2, h = %g: sum_k kR[i][k] d^k, d = a + kR[i][%d]; worst relative" % (H, DEG + 1),
        "// error %.2e (exact arithmetic), %.2e (double, no fma)" % (worst_exact, worst_f64),
        "constexpr int kRIntervals = %d, kRDeg = %d, kRStride = %d;" % (NINT, DEG, DEG + 3),
        "constexpr double kRScale = %s;  // 1 / width" % fmt(1.0 / H),
        "__device__ constexpr double kR[%d][%d] = {" % (NINT, DEG + 3),
    ]
    for r in rows:
        L.append("    {" + ", ".join(fmt(v) for v in r) + "},")
    L += [
        "};",
        "",
        "// exp(x) = 2^(k >> %d) 2^((k & %d) / %d) exp(r),  k = round(x kExpInv)," % (EXP_BITS, 2 ** EXP_BITS - 1,
                                                                                 2 ** EXP_BITS),
        "// r = (x - k kExpHi) - k kExpLo",
        "constexpr int kExpBits = %d;" % EXP_BITS,
        "constexpr double kExpInv = %s;" % fmt(inv),
        "constexpr double kExpHi = %s;  // 34 significant bits" % fmt(hi),
        "constexpr double kExpLo = %s;" % fmt(lo),
        "__device__ constexpr double kExp2Frac[%d] = {" % len(table),
    ]
    for k in range(0, len(table), 4):
        L.append("    " + ", ".join(fmt(v) for v in table[k:k + 4]) + ",")
    L += ["};", "", "}  // namespace special64", "}  // namespace vk", ""]
    with open(OUT, "w") as f:
        f.write("\n".join(L))


def main():
    rows, we, wf = fit_R()
    hi, lo, inv, table = exp_constants()
    print("R pieces: worst relative error %.3e exact, %.3e in double" % (we, wf))
    emit(rows, hi, lo, inv, table, we, wf)
    print("wrote", OUT)


if __name__ == "__main__":
    main()
