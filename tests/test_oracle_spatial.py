"""Pins of the oracle's covariance, Cholesky, ordering and neighbour search.

Sec. 2.1: the conditioning set N_i of site i is its m nearest previously
ordered sites, |N_i| = min(m, i-1); Sec. 3 uses isotropic exponential
covariances on regular grids.  Neighbour sets are pinned to scipy's k-d tree
on tie-free inputs; the covariance to the general Matern formula through the
modified Bessel function K_nu.
"""
import math

import numpy as np
import pytest
from scipy import special
from scipy.spatial import cKDTree

import oracle as O
from paper_2007_15195_gb300 import inputs


def _matern_bessel(h, var, rho, nu):
    """Rasmussen-Williams Matern via K_nu: var 2^{1-nu}/Gamma(nu) (a)^nu K_nu(a), a = sqrt(2 nu) h / rho."""
    if h == 0:
        return var
    a = math.sqrt(2 * nu) * h / rho
    return var * 2 ** (1 - nu) / special.gamma(nu) * a ** nu * special.kv(nu, a)


@pytest.mark.parametrize("nu", [0.5, 1.5, 2.5])
def test_matern_closed_forms_match_bessel(nu):
    for h in [0.0, 1e-6, 0.01, 0.05, 0.1, 0.37, 1.2]:
        got = O.cov(O.COV_MATERN, 1.7, 0.13, nu, h)
        assert got == pytest.approx(_matern_bessel(h, 1.7, 0.13, nu), rel=1e-12)


def test_exponential_is_matern_half():
    for h in [0.0, 0.02, 0.5, 3.0]:
        assert O.cov(O.COV_EXPONENTIAL, 2.0, 0.3, 9.9, h) == O.cov(O.COV_MATERN, 2.0, 0.3, 0.5, h)
        assert O.cov(O.COV_EXPONENTIAL, 2.0, 0.3, 0.0, h) == pytest.approx(2.0 * math.exp(-h / 0.3),
                                                                            rel=1e-15)


def test_unsupported_nu_rejected():
    assert math.isnan(O.cov(O.COV_MATERN, 1.0, 0.1, 1.0, 0.3))


def test_cov_matrix_nugget_and_symmetry():
    s = inputs.uniform_sites(20, 3)
    A = O.cov_matrix(s, O.COV_MATERN, 1.3, 0.2, 1.5, nugget=0.01)
    assert np.allclose(A, A.T, rtol=0, atol=0)
    assert np.allclose(np.diag(A), 1.31)


def test_cholesky_matches_numpy():
    s = inputs.uniform_sites(31, 5)
    A = O.cov_matrix(s, O.COV_MATERN, 1.0, 0.1, 1.5)
    L = O.cholesky(A)
    assert np.allclose(L @ L.T, A, rtol=0, atol=1e-13)
    assert np.allclose(L, np.linalg.cholesky(A), rtol=1e-9, atol=1e-12)
    assert np.all(np.triu(L, 1) == 0)


def test_cholesky_not_pd():
    A = np.array([[1.0, 1.0], [1.0, 1.0]])
    with pytest.raises(O.OracleError) as e:
        O.cholesky(A)
    assert e.value.status == O.ERR_NOT_PD
    with pytest.raises(O.OracleError):
        O.cholesky(np.array([[1.0, 2.0], [2.0, 1.0]]))


def test_quantize_rule():
    s = inputs.grid_sites(9)  # coordinates k/8: exact dyadic
    q = O.quantize(s)
    assert q.min() == 0 and q.max() == 2 ** 30
    assert np.array_equal(q, np.rint(s * 2 ** 30).astype(np.int64))
    # the longer axis sets the scale; the shorter one is not stretched
    s2 = np.array([[0.0, 0.0], [2.0, 0.5], [1.0, 0.25]])
    q2 = O.quantize(s2)
    assert q2.tolist() == [[0, 0], [2 ** 30, 2 ** 28], [2 ** 29, 2 ** 27]]
    # all sites equal: all zeros
    assert not O.quantize(np.ones((4, 2))).any()


def test_order_xy_is_lexsort():
    r = inputs.rng(1, 99)
    s = np.round(r.random((300, 2)) * 8) / 8  # many exact ties in x and in (x, y)
    perm = O.order(s, O.ORDER_XY)
    ref = np.lexsort((np.arange(300), s[:, 1], s[:, 0]))
    assert np.array_equal(perm, ref)


def test_order_identity():
    assert np.array_equal(O.order(np.zeros((7, 2)), O.ORDER_IDENTITY), np.arange(7))


def test_order_maxmin_property():
    s = inputs.uniform_sites(250, 11)
    perm = O.order(s, O.ORDER_MAXMIN)
    assert sorted(perm.tolist()) == list(range(250))
    q = O.quantize(s)
    d2 = ((q[:, None, :] - q[None, :, :]) ** 2).sum(-1)
    # first: nearest to the centre of the quantised bounding box
    c = 2 * q - q.max(0)
    cd = (c ** 2).sum(1)
    assert perm[0] == int(np.flatnonzero(cd == cd.min())[0])
    chosen = [perm[0]]
    mind = d2[perm[0]].copy()
    for pos in range(1, 250):
        cand = np.setdiff1d(np.arange(250), chosen)
        best = mind[cand].max()
        assert perm[pos] == cand[mind[cand] == best][0]
        chosen.append(perm[pos])
        mind = np.minimum(mind, d2[perm[pos]])


def test_order_maxmin_small_by_hand():
    # square corners + centre: the centre first; every corner is then at the
    # same minimum distance (to the centre), so the corners follow in index order
    s = np.array([[0.0, 0.0], [1.0, 0.0], [0.5, 0.5], [0.0, 1.0], [1.0, 1.0]])
    assert O.order(s, O.ORDER_MAXMIN).tolist() == [2, 0, 1, 3, 4]
    # points on a line: 0 is the centre; then the far end 4 (ties with -4 go to
    # the smaller index), then the other end, then the midpoints
    x = np.array([0.0, 1.0, 2.0, 3.0, 4.0, -1.0, -2.0, -3.0, -4.0])
    s = np.stack([x, np.zeros_like(x)], axis=1)
    assert O.order(s, O.ORDER_MAXMIN).tolist() == [0, 4, 8, 2, 6, 1, 3, 5, 7]


@pytest.mark.parametrize("m", [1, 5, 20, 31])
def test_neighbors_match_kdtree_on_tie_free_sites(m):
    s = inputs.uniform_sites(400, 21)
    nbr = O.neighbors(s, m)
    for i in range(400):
        q = min(m, i)
        row = nbr[i]
        assert np.all(row[q:] == -1)
        got = row[:q]
        assert np.all(np.diff(got) > 0)
        if q == 0:
            continue
        tree = cKDTree(s[:i])
        _, idx = tree.query(s[i], k=q)
        assert set(np.atleast_1d(idx).tolist()) == set(got.tolist()), i


def test_neighbors_on_grid_ties_break_by_index():
    s = inputs.grid_sites(6)
    nbr = O.neighbors(s, 4)
    q = O.quantize(s)
    for i in range(36):
        k = min(4, i)
        keys = sorted(((int(((q[i] - q[j]) ** 2).sum()), j) for j in range(i)))[:k]
        assert nbr[i, :k].tolist() == sorted(j for _, j in keys)
    # the site at grid position (1,1) (index 7): previous sites 0..6; nearest are
    # 1 (below) and 6 (left) at distance 1, then 0 and 2 at sqrt 2
    assert nbr[7].tolist() == [0, 1, 2, 6]


def test_neighbors_of_matches_full():
    s = inputs.uniform_sites(120, 4)
    nbr = O.neighbors(s, 7)
    for i in [0, 1, 6, 7, 8, 50, 119]:
        assert np.array_equal(O.neighbors_of(s, i, 7), nbr[i])
