"""Pins of the oracle's univariate normal CDF and quantile (CPU only).

Phi and Phi^{-1} are the per-coordinate maps of Genz's separation of
variables (Sec. 2.2 evaluates every low-dimensional CDF with it).  They are
pinned to printed quantiles, to scipy's independent ndtr/ndtri, and to the
round trip Phi(Phi^{-1}(p)) = p.
"""
import os

import numpy as np
import pytest
from scipy import special

import oracle as O

GOLDEN = os.path.join(os.path.dirname(__file__), "golden", "normal_quantiles.txt")


def _golden():
    rows = []
    for line in open(GOLDEN):
        line = line.strip()
        if not line or line.startswith("#"):
            continue
        p, z = line.split()
        rows.append((float(p), float(z)))
    return rows


@pytest.mark.parametrize("p,z", _golden())
def test_printed_quantiles(p, z):
    assert O.Phiinv(p) == pytest.approx(z, rel=1e-15, abs=1e-300)


def test_quantile_vs_scipy_ndtri_lower_tail():
    ps = np.concatenate([10.0 ** -np.linspace(300, 1, 300), np.linspace(0.01, 0.5, 50)])
    for p in ps:
        z = O.Phiinv(p)
        assert z == pytest.approx(special.ndtri(p), rel=2e-15, abs=1e-15), p


def test_round_trip_relative():
    ps = 10.0 ** -np.linspace(300, np.log10(2.0), 400)
    for p in ps:
        assert O.Phi(O.Phiinv(p)) == pytest.approx(p, rel=1e-14), p


def test_symmetry_from_complement():
    for p in [1e-200, 1e-30, 1e-6, 0.013, 0.2, 0.49]:
        assert O.Phiinv_pq(1.0 - p, p) == -O.Phiinv(p)


def test_pq_uses_smaller_tail():
    # p = 1 - 1e-20 is not representable; with q given the quantile is exact.
    z = O.Phiinv_pq(1.0, 1e-20)
    assert z == pytest.approx(-special.ndtri(1e-20), rel=1e-15)


def test_clamp_floor():
    z0 = O.Phiinv_pq(0.0, 1.0)
    assert z0 == pytest.approx(special.ndtri(2.0 ** -1000), rel=1e-14)
    assert O.Phiinv_pq(1.0, 0.0) == -z0


def test_phi_vs_scipy():
    # erfc at argument a has condition number ~2 a^2: the rounding of x/sqrt(2)
    # alone moves Phi(x) by ~x^2 ulps in the far tail.
    xs = np.linspace(-38, 38, 761)
    for x in xs:
        rel = 2.3e-16 * max(32.0, 2.0 * x * x)
        assert O.Phi(x) == pytest.approx(special.ndtr(x), rel=rel, abs=1e-300)
        assert O.Phi_tail(x) == pytest.approx(special.ndtr(-abs(x)), rel=rel, abs=1e-300)
