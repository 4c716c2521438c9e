"""Pins of the oracle's general Vecchia terms: joint groups of p sites with a
conditioning set each (Sec. 3.2), random conditioning sets, the anisotropic
exponential covariance (Sec. 4.1), and neighbour counts above 31 (Sec. 3).

  - the conditional Genz sums: num is the d-dim estimate of genz_sums and den
    the c-dim estimate of the leading block, bit for bit;
  - p = 1 with the nearest-neighbour sets is the classic Vecchia estimate;
  - groups conditioned on every earlier site telescope to the full Genz
    estimate (Eq. cascading-conditional-cdf with multivariate factors);
  - independent sites: every term is a product of univariate Phi;
  - Floyd's sampler draws each subset with equal frequency;
  - the Mahalanobis covariance is the isotropic one on rotated, stretched
    coordinates.
"""
import itertools
import math

import numpy as np
import pytest
from scipy import special

import oracle as O
from paper_2007_15195_gb300 import inputs


def _ordered(prob):
    perm = O.order(prob.sites, O.ORDER_MAXMIN)
    return prob.sites[perm], prob.u[perm]


def _lattice(N, S, dim, seed):
    return O.lattice(N, dim), O.shifts(seed, S, dim)


@pytest.mark.parametrize("d", [1, 2, 5, 12])
def test_genz_sums_c_splits_num_and_den(d):
    prob = inputs.small_random(d, 7 + d, m=0)
    Sig = O.cov_matrix(prob.sites, O.COV_EXPONENTIAL, 1.0, 0.4)
    u = prob.u
    N, S = 512, 3
    g, dl = _lattice(N, S, max(d - 1, 1), 5)
    num_ref, den_ref = O.genz_sums(Sig, u, N, S, g, dl)
    for c in range(d):
        num, den = O.genz_sums_c(Sig, u, c, N, S, g, dl)
        assert np.array_equal(num, num_ref)
        if c == d - 1:
            assert np.array_equal(den, den_ref)
        if c == 0:
            assert np.all(den == 1.0)
        else:  # the c-dim estimate of the leading block, same lattice coordinates
            lead, _ = O.genz_sums(Sig[:c, :c], u[:c], N, S, g, dl)
            assert np.array_equal(den, lead)


def test_groups_of_one_are_classic_vecchia():
    prob = inputs.small_random(70, 3, m=6)
    s, u = _ordered(prob)
    nbr = O.neighbors(s, 6)
    cond, cnt = O.group_cond_nearest(s, 1, 6, 6)
    assert np.array_equal(cond, nbr)
    assert np.array_equal(cnt, np.minimum(np.arange(70), 6))
    lp, se, t = O.grouped_log_cdf(s, 1, cond, prob.cov, u, 256, 4, 9, return_terms=True)
    lp0, se0, t0 = O.log_cdf(s, nbr, 6, prob.cov, u, 256, 4, 9, return_terms=True)
    assert np.array_equal(t, t0) and lp == lp0 and se == se0


@pytest.mark.parametrize("D,p", [(10, 3), (12, 4), (9, 2)])
def test_groups_conditioned_on_everything_telescope(D, p):
    prob = inputs.small_random(D, 40 + D, m=0, cov=(O.COV_EXPONENTIAL, 1.0, 0.5, 0.5, 0.0))
    s, u = _ordered(prob)
    cond, cnt = O.group_cond_nearest(s, p, D, D)
    assert all(cnt[k] == k * p for k in range(len(cnt)))
    lp, se = O.grouped_log_cdf(s, p, cond, prob.cov, u, 512, 4, 3)
    lpf, sef = O.full_genz(s, prob.cov, u, 512, 4, 3)
    assert lp == pytest.approx(lpf, rel=1e-12, abs=1e-12)
    assert se == pytest.approx(sef, rel=1e-9, abs=1e-14)


def test_independent_groups_are_products_of_univariate():
    prob = inputs.small_random(30, 5, m=0, cov=(O.COV_EXPONENTIAL, 1.0, 1e-6, 0.5, 0.0))
    s, u = _ordered(prob)
    cond, _ = O.group_cond_nearest(s, 3, 4, 12)
    lp, _ = O.grouped_log_cdf(s, 3, cond, prob.cov, u, 128, 3, 1)
    ref = sum(math.log(special.ndtr(x)) for x in u)
    assert lp == pytest.approx(ref, rel=1e-12)


def test_nearest_union_by_brute_force():
    s = inputs.uniform_sites(23, 4)
    p, m = 4, 3
    cond, cnt = O.group_cond_nearest(s, p, m, p * m)
    q = O.quantize(s).astype(np.int64)
    for k in range((23 + p - 1) // p):
        i0 = k * p
        want = set()
        for i in range(i0, min(i0 + p, 23)):
            d2 = [((q[i] - q[j]) ** 2).sum() for j in range(i0)]
            want |= set(sorted(range(i0), key=lambda j: (d2[j], j))[:m])
        assert cond[k, :cnt[k]].tolist() == sorted(want)
        assert np.all(cond[k, cnt[k]:] == -1)


def test_nearest_union_overflow_is_an_error():
    s = inputs.uniform_sites(40, 1)
    with pytest.raises(O.OracleError):
        O.group_cond_nearest(s, 4, 5, 10)


def test_random_sets_are_valid_and_cover_everything_when_asked():
    cond, cnt = O.group_cond_random(50, 2, 7, 123, 7)
    for k in range(25):
        c = cond[k, :cnt[k]]
        assert cnt[k] == min(7, 2 * k)
        assert np.all(np.diff(c) > 0) and (len(c) == 0 or (c[0] >= 0 and c[-1] < 2 * k))
        assert np.all(cond[k, cnt[k]:] == -1)
    full, cf = O.group_cond_random(20, 1, 25, 5, 25)
    for k in range(20):
        assert full[k, :cf[k]].tolist() == list(range(k))


def test_floyd_subsets_are_uniform():
    """Group 5 of size 1 draws 2 of the 5 earlier sites: all 10 pairs equally often."""
    counts = {}
    n_seeds = 3000
    for seed in range(n_seeds):
        cond, cnt = O.group_cond_random(6, 1, 2, seed, 2)
        key = tuple(cond[5].tolist())
        counts[key] = counts.get(key, 0) + 1
    assert set(counts) == set(itertools.combinations(range(5), 2))
    exp = n_seeds / 10
    chi2 = sum((v - exp) ** 2 / exp for v in counts.values())
    assert chi2 < 30.0  # 9 degrees of freedom: p < 1e-3


def test_anisotropic_is_isotropic_on_transformed_coordinates():
    s = inputs.uniform_sites(25, 6)
    angle, aspect, rho = 0.7, 2.5, 0.3
    c, sn = math.cos(angle), math.sin(angle)
    t = np.stack([s[:, 0] * c - s[:, 1] * sn, aspect * (s[:, 0] * sn + s[:, 1] * c)], axis=1)
    A = O.cov_matrix_t(s, (O.COV_ANISO_EXP, 1.3, rho, 0.5, 0.01, angle, aspect))
    B = O.cov_matrix(t, O.COV_EXPONENTIAL, 1.3, rho, 0.5, 0.01)
    assert np.allclose(A, B, rtol=1e-13, atol=1e-15)
    # no rotation, unit aspect: the plain exponential
    E = O.cov_matrix_t(s, (O.COV_ANISO_EXP, 1.0, rho, 0.5, 0.0, 0.0, 1.0))
    assert np.array_equal(E, O.cov_matrix(s, O.COV_EXPONENTIAL, 1.0, rho))
    # a quarter turn swaps the axes
    assert O.aniso_h(1.0, 0.0, math.pi / 2, 3.0) == pytest.approx(3.0, rel=1e-15)
    assert O.aniso_h(0.0, 1.0, 0.0, 3.0) == pytest.approx(3.0, rel=1e-15)


@pytest.mark.parametrize("m", [40, 50])
def test_many_neighbours_telescope_on_small_problems(m):
    """m >= D - 1 beyond 31 neighbours: still the full Genz estimate."""
    D = m + 1
    prob = inputs.small_random(D, m, m=m, cov=(O.COV_EXPONENTIAL, 1.0, 0.2, 0.5, 0.0))
    s, u = _ordered(prob)
    nbr = O.neighbors(s, m)
    lp, _ = O.log_cdf(s, nbr, m, prob.cov, u, 64, 3, 2)
    lpf, _ = O.full_genz(s, prob.cov, u, 64, 3, 2)
    assert lp == pytest.approx(lpf, rel=1e-12, abs=1e-12)
