"""The arithmetic claims behind the mixed full-D factor's tensor-core update,
checked on the CPU with exact integers and rationals (no GPU, no library
code): a row of the block column written as 2^e times seven balanced
base-256 digits of round(x 2^56) has digits exact in bf16 (|s_0| <= 256,
|s_i| <= 128), the digit products of one significance over 32 columns sum
below 2^24 (so an FP32 accumulator holds them exactly), and the recombined
value V 2^(e_r + e_c - 56), subtracted with one rounding, is within a few
2^-53 of sum_t |L_rt L_ct| of the exact update."""
import math
from fractions import Fraction

import numpy as np
import pytest

K = 32      # columns of a block column
NS = 7      # digits a value


def row_exponent(row):
    mb = max(abs(v) for v in row)
    if mb == 0.0:
        return 0
    return max(math.frexp(mb)[1], -900)  # |x| 2^-e < 1


def digits(x, e):
    X = int(np.rint(math.ldexp(x, 56 - e)))
    d = [0] * NS
    for i in range(NS - 1, 0, -1):
        d[i] = ((X + 128) & 255) - 128
        X = (X - d[i]) >> 8
    d[0] = X
    return d


def bf16_exact(v):
    """An integer is exact in bf16 when its significand needs at most 8 bits."""
    v = abs(v)
    while v and v % 2 == 0:
        v //= 2
    return v < 256


def sliced_update(a0, Lr, Lc):
    er, ec = row_exponent(Lr), row_exponent(Lc)
    dr = [digits(v, er) for v in Lr]
    dc = [digits(v, ec) for v in Lc]
    G = []
    for g in range(NS):
        G.append(sum(dr[t][i] * dc[t][g - i] for i in range(g + 1) for t in range(K)))
    V = G[0]
    for g in range(1, NS - 1):
        V = V * 256 + G[g]
    V += G[NS - 1] >> 8
    return float(Fraction(a0) - Fraction(float(V)) * Fraction(2) ** (er + ec - 56)), dr, dc, G, V


@pytest.mark.parametrize("seed", range(6))
def test_digits_are_exact_in_bf16_and_reconstruct_the_row(seed):
    rng = np.random.default_rng(seed)
    row = rng.standard_normal(K) * 10.0 ** rng.uniform(-8, 3, K)
    e = row_exponent(row)
    for x in row:
        d = digits(float(x), e)
        assert abs(d[0]) <= 256 and all(-128 <= v <= 127 for v in d[1:])
        assert all(bf16_exact(v) for v in d)
        back = sum(Fraction(v) * Fraction(2) ** (-8 * (i + 1)) for i, v in enumerate(d)) * Fraction(2) ** e
        assert abs(back - Fraction(float(x))) <= Fraction(2) ** (e - 57)


@pytest.mark.parametrize("seed", range(12))
def test_sums_fit_fp32_and_update_is_fp64_accurate(seed):
    rng = np.random.default_rng(100 + seed)
    sr, sc = 10.0 ** rng.uniform(-4, 2), 10.0 ** rng.uniform(-4, 2)
    Lr = rng.standard_normal(K) * sr * 10.0 ** rng.uniform(-6, 0, K)
    Lc = rng.standard_normal(K) * sc
    if seed % 3 == 0:  # equal rows: the diagonal entries of the update
        Lc = Lr.copy()
    a0 = float(rng.standard_normal() * sr * sc * K)
    got, dr, dc, G, V = sliced_update(a0, [float(v) for v in Lr], [float(v) for v in Lc])
    for g in range(NS):
        assert abs(G[g]) < 2 ** 24  # exact in an FP32 accumulator
    assert abs(V) < 2 ** 63
    exact = Fraction(a0) - sum(Fraction(float(x)) * Fraction(float(y)) for x, y in zip(Lr, Lc))
    mag = sum(abs(Fraction(float(x)) * Fraction(float(y))) for x, y in zip(Lr, Lc))
    # one rounding of V, the dropped products and digits, and the final rounding
    assert abs(Fraction(got) - exact) <= 4 * Fraction(2) ** -53 * (mag + abs(exact))


def test_zero_row_gives_no_update():
    got, _, _, G, V = sliced_update(1.5, [0.0] * K, [1.0] * K)
    assert V == 0 and got == 1.5 and all(g == 0 for g in G)
