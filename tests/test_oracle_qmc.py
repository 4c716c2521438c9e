"""Pins of the oracle's randomisation (Philox shifts) and rank-1 lattice.

Genz QMC (Sec. 2.2, Sec. 3) uses a lattice rule with random shifts; the
paper names no generator.  Philox4x32-10 is pinned to its published
known-answer vectors; the lattice criterion is pinned to its dual-lattice
(Fourier) definition, an independent route to the same number.
"""
import math
import os

import numpy as np
import pytest

import oracle as O

GOLDEN = os.path.join(os.path.dirname(__file__), "golden", "philox4x32_10_kat.txt")


def _kat():
    rows = []
    for line in open(GOLDEN):
        line = line.strip()
        if not line or line.startswith("#"):
            continue
        v = [int(x, 16) for x in line.split()]
        rows.append((v[0:4], v[4:6], v[6:10]))
    return rows


@pytest.mark.parametrize("ctr,key,out", _kat())
def test_philox_known_answers(ctr, key, out):
    assert list(O.philox4x32_10(ctr, key)) == out


def test_shifts_are_53bit_uniforms():
    d = O.shifts(12345, 64, 30)
    assert d.shape == (64, 30)
    assert np.all(d >= 0.0) and np.all(d < 1.0)
    ints = d * 2.0 ** 53
    assert np.all(ints == np.floor(ints))
    assert len(np.unique(d)) == d.size
    # mean and variance of 1920 uniforms
    assert abs(d.mean() - 0.5) < 4 * math.sqrt(1 / 12 / d.size)
    assert abs(d.var() - 1 / 12) < 0.01


def test_shifts_prefix_stable_and_seeded():
    a = O.shifts(7, 8, 10)
    b = O.shifts(7, 16, 31)
    assert np.array_equal(a, b[:8, :10])
    assert not np.array_equal(a, O.shifts(8, 8, 10))
    # high 32 bits of the seed reach the key
    assert not np.array_equal(O.shifts(7, 2, 2), O.shifts(7 + (1 << 32), 2, 2))


def _p2_dual(N, g, gammas, H):
    """P2 as the weighted sum over the dual lattice {h != 0 : h.g = 0 mod N}
    of prod_j w_j(h_j), w(0) = 1, w(h) = gamma/h^2, truncated at |h_j| <= H."""
    h = np.arange(-H, H + 1)
    hs = np.where(h == 0, 1, h).astype(np.float64)
    w = [np.where(h == 0, 1.0, gm / hs ** 2) for gm in gammas]
    if len(g) == 2:
        dot = (h[:, None] * g[0] + h[None, :] * g[1]) % N
        W = w[0][:, None] * w[1][None, :]
        mask = dot == 0
        mask[H, H] = False
        return W[mask].sum()
    raise NotImplementedError


@pytest.mark.parametrize("N,a", [(31, 12), (32, 7), (50, 13)])
def test_p2_matches_dual_lattice_sum(N, a):
    g = [1, a % N]
    H = 3000
    ref = _p2_dual(N, g, [1.0, 0.25], H)
    got = O.p2(N, a, 2)
    # truncation error of the dual sum is O(gamma / H)
    assert got == pytest.approx(ref, rel=3e-3)


def test_korobov_multiplier_is_the_argmin():
    for N in [61, 64, 100]:
        a = O.korobov_a(N)
        cands = [b for b in range(2, N // 2 + 1) if math.gcd(b, N) == 1]
        vals = {b: O.p2(N, b, 30) for b in cands}
        best = min(vals.values())
        assert vals[a] == best
        assert a == min(b for b in cands if vals[b] == best)


@pytest.mark.parametrize("N", [2000, 2048, 4096, 8192])
def test_lattice_vectors(N):
    a = O.korobov_a(N)
    assert 2 <= a <= N // 2 and math.gcd(a, N) == 1
    g = O.lattice_c(N, 40)
    assert g[0] == 1
    for j in range(1, 40):
        assert g[j] == (int(g[j - 1]) * a) % N
    assert np.array_equal(g, O.lattice(N, 40))


def test_lattice_rule_integrates_trig_polynomials():
    # A rank-1 lattice integrates exp(2 pi i h.x) exactly (to 0) unless h is in
    # the dual lattice; low-degree modes are absent for a good multiplier.
    N = 4096
    g = O.lattice(N, 4).astype(np.int64)
    k = np.arange(N)
    x = (np.outer(k, g) % N) / N
    for h in [(1, 0, 0, 0), (0, 1, 0, 0), (1, 1, 0, 0), (2, -1, 1, 0), (1, 1, 1, 1)]:
        v = np.exp(2j * np.pi * (x @ np.array(h))).mean()
        assert abs(v) < 1e-10
