"""GPU parity: the CUDA path through the C ABI against the oracle.

Bars (element by element on the same seeded inputs):
  - neighbour sets: bit-exact;
  - FP64 path: relative error <= 1e-10 on log P (and on every per-shift
    partial num[i,s], den[i,s]);
  - mixed path: |d log P| <= 1e-4 max(1, |log P|).
Sizes span several CTAs and ragged lattice tails; the full-size 50x50 grid
cases are checked in full at m = 20 and on sampled terms at other m.
"""
import math

import numpy as np
import pytest

import oracle as O
from paper_2007_15195_gb300 import binding as B
from paper_2007_15195_gb300 import inputs

from _prep import mixed_tol, oracle_prepare

pytestmark = pytest.mark.gpu

FP64_TOL = 1e-10


@pytest.fixture(scope="module")
def ctx():
    import torch
    assert torch.cuda.is_available()
    c = B.Context(0)
    yield c
    c.close()


def _gpu_prepare(ctx, prob):
    perm = B.vecchia_order(ctx, prob.sites, prob.order)
    s = np.ascontiguousarray(prob.sites[perm])
    u = np.ascontiguousarray(prob.u[perm])
    nbr = B.vecchia_neighbors(ctx, s, prob.m) if prob.m > 0 else np.zeros((s.shape[0], 0), np.int32)
    return perm, s, u, nbr


# ----------------------------------------------------------------------------
# neighbours
# ----------------------------------------------------------------------------

@pytest.mark.parametrize("n,m", [(10, 10), (50, 5), (50, 10), (50, 20), (50, 30), (50, 31)])
def test_knn_grid_bit_exact(ctx, n, m):
    s = inputs.grid_sites(n)
    assert np.array_equal(B.vecchia_neighbors(ctx, s, m), O.neighbors(s, m))


@pytest.mark.parametrize("D,m,seed", [(1, 5, 0), (2, 31, 0), (33, 31, 1), (3000, 20, 2), (4100, 1, 3)])
def test_knn_uniform_maxmin_bit_exact(ctx, D, m, seed):
    s = inputs.uniform_sites(D, seed)
    perm = O.order(s, O.ORDER_MAXMIN)
    so = np.ascontiguousarray(s[perm])
    assert np.array_equal(B.vecchia_neighbors(ctx, so, m), O.neighbors(so, m))


def test_knn_large_sampled(ctx):
    """100,000 uniform sites (the large workload's size), m = 30, in maxmin
    order: sampled sites against the oracle's one-site search."""
    D, m = 100_000, 30
    s = inputs.uniform_sites(D, 0)
    perm = B.vecchia_order(None, s, "maxmin")
    so = np.ascontiguousarray(s[perm])
    import torch
    nb = B.vecchia_neighbors(ctx, torch.from_numpy(so).cuda(), m).cpu().numpy()
    rng = np.random.default_rng(5)
    sample = np.unique(np.concatenate([np.arange(40), rng.integers(0, D, 160), [D - 1]]))
    for i in sample:
        assert np.array_equal(nb[i], O.neighbors_of(so, int(i), m)), i


def test_knn_degenerate_geometry(ctx):
    # all sites equal: every squared distance is 0, ties go to the smaller index
    s = np.ones((40, 2))
    assert np.array_equal(B.vecchia_neighbors(ctx, s, 6), O.neighbors(s, 6))
    # collinear, exactly repeated coordinates, random order
    x = np.repeat(np.arange(30) / 29.0, 3)
    s = np.stack([x, np.zeros_like(x)], axis=1)[inputs.rng(0, 1).permutation(90)]
    s = np.ascontiguousarray(s)
    assert np.array_equal(B.vecchia_neighbors(ctx, s, 8), O.neighbors(s, 8))
    # ring search with many ties on a large regular grid (beyond the brute-force prefix)
    g = inputs.grid_sites(70)
    assert np.array_equal(B.vecchia_neighbors(ctx, g, 12), O.neighbors(g, 12))


def test_knn_device_arrays(ctx):
    import torch
    s = inputs.uniform_sites(2500, 9)
    nb_h = B.vecchia_neighbors(ctx, s, 10)
    nb_d = B.vecchia_neighbors(ctx, torch.from_numpy(s).cuda(), 10)
    assert nb_d.is_cuda and np.array_equal(nb_d.cpu().numpy(), nb_h)


# ----------------------------------------------------------------------------
# log-CDF: FP64 and mixed against the oracle
# ----------------------------------------------------------------------------

CASES = [
    # (name, problem factory)
    ("grid10", lambda: inputs.grid10()),
    ("rand_m0", lambda: inputs.small_random(64, 1, m=0, N=256, S=4)),
    ("rand_m1_ragged", lambda: inputs.small_random(300, 2, m=1, N=1000, S=3)),
    ("rand_m7_matern25", lambda: inputs.small_random(
        200, 3, m=7, cov=(O.COV_MATERN, 1.5, 0.2, 2.5, 0.0), N=777, S=2)),
    ("rand_m15_nugget", lambda: inputs.small_random(
        257, 4, m=15, cov=(O.COV_MATERN, 1.0, 0.15, 1.5, 0.05), N=512, S=5)),
    ("rand_m23", lambda: inputs.small_random(150, 5, m=23, N=300, S=4)),
    ("rand_m31", lambda: inputs.small_random(120, 6, m=31, N=256, S=3)),
    ("D_lt_m", lambda: inputs.small_random(9, 7, m=20, N=640, S=6)),
    ("D1", lambda: inputs.small_random(1, 8, m=5, N=64, S=2)),
    ("S64_max_shifts", lambda: inputs.small_random(100, 9, m=10, N=128, S=64)),
    ("N1_one_point", lambda: inputs.small_random(40, 10, m=5, N=1, S=2)),
    ("N3_odd", lambda: inputs.small_random(60, 11, m=6, N=3, S=3)),
    ("m63_max", lambda: inputs.small_random(80, 12, m=63, N=128, S=2)),
]


@pytest.fixture(scope="module")
def oracle_results():
    return {}


def _oracle(cache, name, prob):
    if name not in cache:
        _, s, u, nbr = oracle_prepare(prob)
        num, den = O.vecchia_partials(s, nbr, prob.m, prob.cov, u, prob.N, prob.S, prob.seed)
        lp, se, terms = O.vecchia_reduce(num, den)
        cache[name] = (s, u, nbr, num, den, lp, se, terms)
    return cache[name]


@pytest.mark.parametrize("name,factory", CASES, ids=[c[0] for c in CASES])
def test_fp64_matches_oracle(ctx, oracle_results, name, factory):
    prob = factory()
    s, u, nbr, num, den, lp, se, terms = _oracle(oracle_results, name, prob)
    _, gs, gu, gnbr = _gpu_prepare(ctx, prob)
    assert np.array_equal(gs, s) and np.array_equal(gnbr, nbr)
    glp, gse, gterms, gnum, gden = B.vecchia_log_cdf_terms(ctx, gs, gnbr, prob.m, prob.cov, gu, prob.N,
                                                           prob.S, prob.seed, B.FP64)
    assert abs(glp - lp) <= FP64_TOL * abs(lp), (glp, lp)
    assert np.allclose(gnum, num, rtol=FP64_TOL, atol=0)
    assert np.allclose(gden, den, rtol=FP64_TOL, atol=0)
    assert np.allclose(gterms, terms, rtol=1e-9, atol=1e-12)
    if se > 0:
        assert abs(gse - se) <= 1e-7 * se
    else:
        assert gse <= 1e-12


@pytest.mark.parametrize("name,factory", CASES, ids=[c[0] for c in CASES])
def test_mixed_matches_oracle(ctx, oracle_results, name, factory):
    prob = factory()
    s, u, nbr, num, den, lp, se, terms = _oracle(oracle_results, name, prob)
    glp, gse = B.vecchia_log_cdf(ctx, s, nbr, prob.m, prob.cov, u, prob.N, prob.S, prob.seed, B.MIXED)
    assert abs(glp - lp) <= mixed_tol(lp), (glp, lp)
    # the standard error is a spread statistic: same order of magnitude
    assert gse == pytest.approx(se, rel=0.05, abs=1e-6)


def test_identity_m_full_against_oracle_full_genz(ctx):
    """m = D - 1 (D = 32): the Vecchia product telescopes to the full Genz
    estimate (Eq. cascading-conditional-cdf); the FP64 GPU path reproduces the
    oracle's full 32-dimensional estimate."""
    prob = inputs.small_random(32, 10, m=31, N=1024, S=4)
    _, s, u, nbr = oracle_prepare(prob)
    full, full_se = O.full_genz(s, prob.cov, u, prob.N, prob.S, prob.seed)
    glp, gse = B.vecchia_log_cdf(ctx, s, nbr, 31, prob.cov, u, prob.N, prob.S, prob.seed, B.FP64)
    assert abs(glp - full) <= FP64_TOL * abs(full)
    assert gse == pytest.approx(full_se, rel=1e-7)


# ----------------------------------------------------------------------------
# the 50x50 grid (Matern 1.5, range 0.1, N = 4096, S = 16) at full size
# ----------------------------------------------------------------------------

@pytest.fixture(scope="module")
def grid50_m20():
    prob = inputs.grid50(m=20)
    _, s, u, nbr = oracle_prepare(prob)
    num, den = O.vecchia_partials(s, nbr, 20, prob.cov, u, prob.N, prob.S, prob.seed)
    lp, se, terms = O.vecchia_reduce(num, den)
    return prob, s, u, nbr, num, den, lp, se, terms


def test_grid50_m20_full_both_paths(ctx, grid50_m20):
    prob, s, u, nbr, num, den, lp, se, terms = grid50_m20
    import torch
    ds, du, dn = (torch.from_numpy(x).cuda() for x in (s, u, nbr))
    glp, gse, gterms, gnum, gden = B.vecchia_log_cdf_terms(ctx, ds, dn, 20, prob.cov, du, prob.N,
                                                           prob.S, prob.seed, B.FP64)
    assert abs(glp - lp) <= FP64_TOL * abs(lp)
    assert np.allclose(gnum.cpu().numpy(), num, rtol=FP64_TOL, atol=0)
    mlp, mse = B.vecchia_log_cdf(ctx, ds, dn, 20, prob.cov, du, prob.N, prob.S, prob.seed, B.MIXED)
    assert abs(mlp - lp) <= mixed_tol(lp), (mlp, lp)


def test_grid50_m20_benchmark_call(ctx, grid50_m20):
    """The call and configuration bench.py times (raw sites on the device,
    vecchia_log_cdf_unordered, XY order, mixed and FP64) against the oracle."""
    prob, s, u, nbr, num, den, lp, se, terms = grid50_m20
    import torch
    rs, ru = torch.from_numpy(prob.sites).cuda(), torch.from_numpy(prob.u).cuda()
    mlp, mse = B.vecchia_log_cdf_unordered(ctx, rs, ru, 20, prob.cov, prob.N, prob.S, prob.seed, B.MIXED)
    assert abs(mlp - lp) <= mixed_tol(lp), (mlp, lp)
    flp, fse = B.vecchia_log_cdf_unordered(ctx, rs, ru, 20, prob.cov, prob.N, prob.S, prob.seed, B.FP64)
    assert abs(flp - lp) <= FP64_TOL * abs(lp) and fse == pytest.approx(se, rel=1e-8)


@pytest.mark.parametrize("m", [5, 10, 30])
def test_grid50_sampled_terms(ctx, m):
    prob = inputs.grid50(m=m)
    _, s, u, nbr = oracle_prepare(prob)
    gnbr = B.vecchia_neighbors(ctx, s, m)
    assert np.array_equal(gnbr, nbr)
    idx = np.unique(np.concatenate([np.arange(m + 2), np.linspace(m + 2, 2499, 40).astype(int)]))
    num, den = O.vecchia_partials(s, nbr, m, prob.cov, u, prob.N, prob.S, prob.seed, idx=idx)
    t_or = np.log(num.mean(1)) - np.log(den.mean(1))
    glp, gse, gterms, gnum, gden = B.vecchia_log_cdf_terms(ctx, s, nbr, m, prob.cov, u, prob.N, prob.S,
                                                           prob.seed, B.FP64)
    assert np.allclose(gnum[idx], num, rtol=FP64_TOL, atol=0)
    assert np.allclose(gden[idx], den, rtol=FP64_TOL, atol=0)
    mlp, mse, mterms, _, _ = B.vecchia_log_cdf_terms(ctx, s, nbr, m, prob.cov, u, prob.N, prob.S,
                                                     prob.seed, B.MIXED)
    # sufficient per-term bound for the log-P tolerance: mixed_tol(log P) / D
    per_term = mixed_tol(glp) / s.shape[0]
    assert np.max(np.abs(mterms[idx] - t_or)) <= per_term
    assert abs(mlp - glp) <= mixed_tol(glp)


# ----------------------------------------------------------------------------
# boundary behaviour
# ----------------------------------------------------------------------------

def test_d1_exact(ctx):
    s = np.array([[0.3, 0.4]])
    for prec in (B.FP64, B.MIXED):
        lp, se = B.vecchia_log_cdf(ctx, s, np.zeros((1, 3), np.int32), 3, (B.COV_EXPONENTIAL, 4.0, 0.2, 0.5, 0.0),
                                   np.array([1.0]), 128, 4, 0, prec)
        assert lp == pytest.approx(math.log(O.Phi(0.5)), rel=1e-14)
        assert se == 0.0


def test_not_pd_reports_site(ctx):
    s = np.array([[0.0, 0.0], [0.5, 0.5], [0.5, 0.5], [1.0, 0.0], [0.2, 0.9]])
    nbr = O.neighbors(s, 2)
    for prec in (B.FP64, B.MIXED):
        with pytest.raises(B.VecchiaError) as e:
            B.vecchia_log_cdf(ctx, s, nbr, 2, (B.COV_EXPONENTIAL, 1.0, 0.3, 0.5, 0.0), np.zeros(5), 64, 4, 0,
                              prec)
        assert e.value.status == B.ERR_NOT_PD and e.value.site == 2


def test_argument_errors(ctx):
    s = inputs.uniform_sites(10, 0)
    nbr = O.neighbors(s, 3)
    cov = (B.COV_EXPONENTIAL, 1.0, 0.3, 0.5, 0.0)
    u = np.zeros(10)
    bad = [
        dict(S=1), dict(S=65), dict(N=0), dict(cov=(B.COV_MATERN, 1.0, 0.3, 1.0, 0.0)),
        dict(cov=(B.COV_EXPONENTIAL, -1.0, 0.3, 0.5, 0.0)), dict(cov=(7, 1.0, 0.3, 0.5, 0.0)),
        dict(u=np.array([0.0] * 9 + [np.nan])), dict(precision=5),
    ]
    for b in bad:
        args = dict(S=4, N=64, cov=cov, u=u, precision=B.FP64)
        args.update(b)
        with pytest.raises(B.VecchiaError) as e:
            B.vecchia_log_cdf(ctx, s, nbr, 3, args["cov"], args["u"], args["N"], args["S"], 0,
                              args["precision"])
        assert e.value.status == B.ERR_ARG, b
    with pytest.raises(B.VecchiaError) as e:
        B.vecchia_neighbors(ctx, s, B.MAX_M + 1)
    assert e.value.status == B.ERR_UNSUPPORTED
    # a neighbour list that is not ascending / not previous
    bad_nbr = nbr.copy()
    bad_nbr[5, 0] = 7
    with pytest.raises(B.VecchiaError) as e:
        B.vecchia_log_cdf(ctx, s, bad_nbr, 3, cov, u, 64, 4, 0, B.FP64)
    assert e.value.status == B.ERR_ARG and e.value.site == 5


def test_host_and_device_pointers_agree_and_repeat(ctx):
    import torch
    prob = inputs.small_random(700, 11, m=12, N=1024, S=6)
    _, s, u, nbr = oracle_prepare(prob)
    for prec in (B.FP64, B.MIXED):
        a = B.vecchia_log_cdf(ctx, s, nbr, 12, prob.cov, u, prob.N, prob.S, 3, prec)
        b = B.vecchia_log_cdf(ctx, torch.from_numpy(s).cuda(), torch.from_numpy(nbr).cuda(), 12, prob.cov,
                              torch.from_numpy(u).cuda(), prob.N, prob.S, 3, prec)
        c = B.vecchia_log_cdf(ctx, s, nbr, 12, prob.cov, u, prob.N, prob.S, 3, prec)
        assert a == b == c  # bit-identical: fixed reduction order


def test_tiles_change_only_sum_order(ctx):
    prob = inputs.small_random(500, 12, m=20, N=2048, S=8)
    _, s, u, nbr = oracle_prepare(prob)
    for prec in (B.FP64, B.MIXED):
        B.vecchia_reset_tiles(ctx)
        ref = B.vecchia_log_cdf(ctx, s, nbr, 20, prob.cov, u, prob.N, prob.S, 1, prec)
        for warps, points, slices, groups in [(1, 1, 1, 1), (8, 2, 1, 8), (4, 2, 4, 2), (16, 1, 2, 3), (2, 2, 1, 3)]:
            B.vecchia_set_tile(ctx, prec, -1, warps, points, slices, groups)
            lp, se = B.vecchia_log_cdf(ctx, s, nbr, 20, prob.cov, u, prob.N, prob.S, 1, prec)
            if slices == 1:  # same points per lane in the same order: bit-identical
                assert (lp, se) == ref
            else:  # other point subsets per lane: FP64 sums reorder at 1e-16, FP32 Kahan at ~1e-9
                assert lp == pytest.approx(ref[0], rel=1e-12 if prec == B.FP64 else 1e-8)
        B.vecchia_reset_tiles(ctx)


@pytest.mark.parametrize("m,N", [(3, 1000), (8, 77), (12, 4096), (16, 129), (20, 1000), (28, 333)])
def test_two_points_per_lane_equal_one(ctx, m, N):
    """Two points per lane compute, point by point, the arithmetic of one
    point per lane: the per-shift partial means agree bit for bit, with point
    counts that leave the last pass of a lane ragged."""
    prob = inputs.small_random(300, 14 + m, m=m, N=N, S=4)
    _, s, u, nbr = oracle_prepare(prob)
    out = {}
    for pts in (1, 2):
        B.vecchia_set_tile(ctx, B.MIXED, -1, 4, pts, 1, 1)
        out[pts] = B.vecchia_log_cdf_terms(ctx, s, nbr, m, prob.cov, u, prob.N, prob.S, 2, B.MIXED)
    B.vecchia_reset_tiles(ctx)
    assert out[1][0] == out[2][0] and out[1][1] == out[2][1]
    assert np.array_equal(np.asarray(out[1][3]), np.asarray(out[2][3]))
    assert np.array_equal(np.asarray(out[1][4]), np.asarray(out[2][4]))


def test_last_round_split_leaves_results_unchanged(ctx):
    """2,500 terms on the grid outnumber the resident CTAs, so the launch cuts
    the sites of its last, partial round into more shift groups; with one
    shift per item (16 groups) nothing is cut.  A shift's partial means come
    from one warp either way: both precisions agree bit for bit."""
    prob = inputs.grid50(m=20, N=512, S=16)
    _, s, u, nbr = oracle_prepare(prob)
    for prec in (B.FP64, B.MIXED):
        out = []
        for groups in (1, 16):
            B.vecchia_set_tile(ctx, prec, -1, 4, 1 if prec == B.FP64 else 2, 1, groups)
            out.append(B.vecchia_log_cdf_terms(ctx, s, nbr, prob.m, prob.cov, u, prob.N, prob.S, 4, prec))
        B.vecchia_reset_tiles(ctx)
        assert out[0][0] == out[1][0] and out[0][1] == out[1][1]
        assert np.array_equal(np.asarray(out[0][3]), np.asarray(out[1][3]))
        assert np.array_equal(np.asarray(out[0][4]), np.asarray(out[1][4]))


def test_mixed_underflow_falls_back_to_log_space(ctx):
    """Thresholds far below the mean: FP32 conditional probabilities underflow
    in the fast mixed form, whose lattice means then fall below 2^-40; those
    terms are flagged and re-evaluated by the log-space FP32 form (probabilities
    carried as log2 below 2^-64), so the mixed result stays within the mixed
    tolerance of the oracle (and of the FP64 path)."""
    prob = inputs.small_random(60, 13, m=6, u_mean=-14.0, u_sd=0.5, N=256, S=4)
    _, s, u, nbr = oracle_prepare(prob)
    ref, _ = O.log_cdf(s, nbr, 6, prob.cov, u, prob.N, prob.S, 0)
    lp64, se64 = B.vecchia_log_cdf(ctx, s, nbr, 6, prob.cov, u, prob.N, prob.S, 0, B.FP64)
    lpm, sem = B.vecchia_log_cdf(ctx, s, nbr, 6, prob.cov, u, prob.N, prob.S, 0, B.MIXED)
    assert math.isfinite(lpm) and ref < -100.0  # deep in the tail
    assert abs(lp64 - ref) <= 1e-10 * abs(ref)
    assert abs(lpm - ref) <= mixed_tol(ref)
    assert abs(lpm - lp64) <= mixed_tol(lp64)


def test_batch_equals_single_calls(ctx):
    probs = [inputs.small_random(40 + 37 * k, 20 + k, m=[0, 3, 10, 20, 31][k % 5], N=[256, 500][k % 2],
                                 S=[2, 4, 8][k % 3]) for k in range(12)]
    prepared = [oracle_prepare(p) for p in probs]
    items = [dict(sites=s, nbr=nbr, m=p.m, cov=p.cov, u=u, N=p.N, S=p.S, seed=p.seed)
             for p, (_, s, u, nbr) in zip(probs, prepared)]
    # one failing problem in the middle (duplicated sites)
    bad_s = np.array([[0.0, 0.0], [0.5, 0.5], [0.5, 0.5], [1.0, 0.0]])
    items.insert(5, dict(sites=bad_s, nbr=O.neighbors(bad_s, 2), m=2, cov=(0, 1.0, 0.3, 0.5, 0.0),
                         u=np.zeros(4), N=64, S=4, seed=0))
    for prec in (B.FP64, B.MIXED):
        lp, se, st = B.vecchia_log_cdf_batch(ctx, items, prec)
        assert st[5] == B.ERR_NOT_PD and math.isnan(lp[5])
        for k, it in enumerate(items):
            if k == 5:
                continue
            assert st[k] == B.OK
            ref = B.vecchia_log_cdf(ctx, it["sites"], it["nbr"], it["m"], it["cov"], it["u"], it["N"],
                                    it["S"], it["seed"], prec)
            assert (lp[k], se[k]) == pytest.approx(ref, rel=1e-13, abs=1e-15)
