"""The large workload at full size: D = 100,000 sites uniform in the unit
square, exact maxmin order, Matern nu in {0.5, 1.5} with range 0.05,
u ~ U[0, 2], m = 30, N = 8,192 x S = 16.  The full mixed-precision
evaluation is checked term by term on sampled sites against the oracle's
one-site evaluation; the FP64 path at full size, its per-shift partial means
on sampled terms against the oracle's (1e-10) and its log P against the mixed
one (the mixed tolerance), and on an ordered prefix (itself a valid problem:
every neighbour of site i < K is among the first K sites)."""
import numpy as np
import pytest

import oracle as O
from paper_2007_15195_gb300 import binding as B
from paper_2007_15195_gb300 import inputs

from _prep import mixed_tol

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def ctx():
    c = B.Context(0)
    yield c
    c.close()


@pytest.fixture(scope="module")
def large_ordered():
    prob = inputs.large(nu=1.5)
    perm = B.vecchia_order(None, prob.sites, "maxmin")
    s, u = B.vecchia_apply_order(None, perm, prob.sites, prob.u)
    return prob, s, u


@pytest.mark.parametrize("nu", [1.5, 0.5])
def test_large_mixed_terms_against_oracle(ctx, large_ordered, nu):
    import torch
    prob, s, u = large_ordered
    cov = (prob.cov[0], prob.cov[1], prob.cov[2], nu, 0.0)
    ds, du = torch.from_numpy(s).cuda(), torch.from_numpy(u).cuda()
    nbr = B.vecchia_neighbors(ctx, ds, prob.m)
    lp, se, terms, num, den = B.vecchia_log_cdf_terms(ctx, ds, nbr, prob.m, cov, du, prob.N, prob.S, 0,
                                                      B.MIXED)
    assert np.isfinite(lp) and lp < 0
    terms = terms.cpu().numpy()
    rng = np.random.default_rng(7)
    idx = np.unique(np.concatenate([[0, 1, 2, 15, 30, 31, 32], rng.integers(33, prob.D, 40)]))
    nb_h = nbr.cpu().numpy()
    for i in idx[:12]:
        assert np.array_equal(nb_h[i], O.neighbors_of(s, int(i), prob.m))
    onum, oden = O.vecchia_partials(s, nb_h, prob.m, cov, u, prob.N, prob.S, 0, idx=idx)
    t_or = np.log(onum.mean(1)) - np.log(oden.mean(1))
    per_term = mixed_tol(lp) / prob.D
    assert np.max(np.abs(terms[idx] - t_or)) <= per_term, np.max(np.abs(terms[idx] - t_or))


def test_large_fp64_on_ordered_prefix(ctx, large_ordered):
    prob, s, u = large_ordered
    K = 3000
    sp, up = np.ascontiguousarray(s[:K]), np.ascontiguousarray(u[:K])
    nbr = B.vecchia_neighbors(ctx, sp, prob.m)
    full_nbr = B.vecchia_neighbors(ctx, s, prob.m)
    assert np.array_equal(nbr, full_nbr[:K])
    lp, se, terms, num, den = B.vecchia_log_cdf_terms(ctx, sp, nbr, prob.m, prob.cov, up, prob.N, prob.S, 3,
                                                      B.FP64)
    idx = np.array([0, 1, 29, 30, 31, 500, 1777, K - 1])
    onum, oden = O.vecchia_partials(sp, nbr, prob.m, prob.cov, up, prob.N, prob.S, 3, idx=idx)
    assert np.allclose(num[idx], onum, rtol=1e-10, atol=0)
    assert np.allclose(den[idx], oden, rtol=1e-10, atol=0)
    mlp, mse = B.vecchia_log_cdf(ctx, sp, nbr, prob.m, prob.cov, up, prob.N, prob.S, 3, B.MIXED)
    assert abs(mlp - lp) <= mixed_tol(lp)


def test_large_fp64_full_size(ctx, large_ordered):
    import torch
    prob, s, u = large_ordered
    ds, du = torch.from_numpy(s).cuda(), torch.from_numpy(u).cuda()
    nbr = B.vecchia_neighbors(ctx, ds, prob.m)
    lp, se, terms, num, den = B.vecchia_log_cdf_terms(ctx, ds, nbr, prob.m, prob.cov, du, prob.N, prob.S, 0,
                                                      B.FP64)
    assert np.isfinite(lp) and lp < 0
    rng = np.random.default_rng(11)
    idx = np.unique(np.concatenate([[0, 1, 2, 29, 30, 31, 32, prob.D - 1], rng.integers(33, prob.D, 32)]))
    nb_h = nbr.cpu().numpy()
    onum, oden = O.vecchia_partials(s, nb_h, prob.m, prob.cov, u, prob.N, prob.S, 0, idx=idx)
    num, den = num.cpu().numpy(), den.cpu().numpy()
    assert np.allclose(num[idx], onum, rtol=1e-10, atol=0), np.max(np.abs(num[idx] / onum - 1))
    assert np.allclose(den[idx], oden, rtol=1e-10, atol=0), np.max(np.abs(den[idx] / oden - 1))
    mlp, _ = B.vecchia_log_cdf(ctx, ds, nbr, prob.m, prob.cov, du, prob.N, prob.S, 0, B.MIXED)
    assert abs(mlp - lp) <= mixed_tol(lp), (mlp, lp)


def _last_variance_fraction(s, nbr, m, rho):
    """Per term with m neighbours: L_qq^2 / Sigma_qq of its block under the
    Matern 3/2 covariance (the last variable's conditional variance fraction;
    near 0 when a neighbour nearly duplicates the site).  numpy Cholesky of
    each block: only used to pick the worst-conditioned terms."""
    D = s.shape[0]
    idx = np.arange(m, D)
    out = np.ones(D)
    for c0 in range(0, idx.size, 8192):
        ii = idx[c0:c0 + 8192]
        blk = np.concatenate([nbr[ii, :m], ii[:, None]], axis=1)
        p = s[blk]
        r = np.sqrt(((p[:, :, None, :] - p[:, None, :, :]) ** 2).sum(-1)) * np.sqrt(3.0) / rho
        L = np.linalg.cholesky((1.0 + r) * np.exp(-r))
        out[ii] = L[:, -1, -1] ** 2
    return out


def test_large_mixed_on_the_worst_conditioned_terms(ctx, large_ordered):
    """Near-duplicate sites make a term's block nearly singular; the mixed
    path's FP64 factor and FP32 integrand must still meet the per-term bound
    on the 24 worst-conditioned terms of the D = 100,000 problem."""
    import torch
    prob, s, u = large_ordered
    ds, du = torch.from_numpy(s).cuda(), torch.from_numpy(u).cuda()
    nbr = B.vecchia_neighbors(ctx, ds, prob.m)
    nb_h = nbr.cpu().numpy()
    frac = _last_variance_fraction(s, nb_h, prob.m, prob.cov[2])
    idx = np.sort(np.argsort(frac)[:24])
    assert frac[idx].max() < 1e-4  # genuinely ill-conditioned blocks
    lp, se, terms, num, den = B.vecchia_log_cdf_terms(ctx, ds, nbr, prob.m, prob.cov, du, prob.N, prob.S, 5,
                                                      B.MIXED)
    onum, oden = O.vecchia_partials(s, nb_h, prob.m, prob.cov, u, prob.N, prob.S, 5, idx=idx)
    t_or = np.log(onum.mean(1)) - np.log(oden.mean(1))
    err = np.abs(terms.cpu().numpy()[idx] - t_or)
    assert np.max(err) <= mixed_tol(lp) / prob.D, (np.max(err), frac[idx])
