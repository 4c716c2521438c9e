"""GPU parity of the general Vecchia terms (Sec. 3.2, Sec. 3, Sec. 4.1):

  - neighbour sets for m up to 63 (the paper's m = 50): bit-exact;
  - conditioning rows of joint groups, nearest (union) and random (Floyd on
    Philox draws): bit-exact;
  - the grouped log-CDF, the classic one with m = 40, 50, and the anisotropic
    exponential covariance: FP64 <= 1e-10 relative, mixed <= 1e-4 max(1, |log P|);
  - groups of one with the nearest-neighbour rows: equal to the classic path
    bit for bit; grouped problems inside a batch: equal to single calls.
"""
import math

import numpy as np
import pytest

import oracle as O
from paper_2007_15195_gb300 import binding as B
from paper_2007_15195_gb300 import inputs

from _prep import mixed_tol

pytestmark = pytest.mark.gpu

FP64_TOL = 1e-10


@pytest.fixture(scope="module")
def ctx():
    c = B.Context(0)
    yield c
    c.close()


def _ordered(D, seed, m=0, cov=(O.COV_EXPONENTIAL, 1.0, 0.3, 0.5, 0.0), u_mean=0.3):
    prob = inputs.small_random(D, seed, m=m, cov=cov, u_mean=u_mean)
    perm = O.order(prob.sites, O.ORDER_MAXMIN)
    return np.ascontiguousarray(prob.sites[perm]), np.ascontiguousarray(prob.u[perm]), prob.cov


def _check(got, ref, prec):
    tol = FP64_TOL * abs(ref) if prec == B.FP64 else mixed_tol(ref)
    assert abs(got - ref) <= tol, (got, ref, prec)


@pytest.mark.parametrize("D,m", [(600, 32), (600, 33), (3000, 40), (3000, 50), (700, 63)])
def test_knn_many_neighbours_bit_exact(ctx, D, m):
    s, _, _ = _ordered(D, 100 + m)
    got = B.vecchia_neighbors(ctx, s, m)
    assert np.array_equal(got, O.neighbors(s, m))


@pytest.mark.parametrize("D,p,m", [(1500, 1, 10), (1500, 3, 5), (2200, 4, 7), (900, 16, 2), (5, 2, 3)])
def test_nearest_group_rows_bit_exact(ctx, D, p, m):
    s, _, _ = _ordered(D, 7 * p + m)
    cond, cnt = B.vecchia_group_conditioning(ctx, s, p, m, B.COND_NEAREST)
    rc, rn = O.group_cond_nearest(s, p, m, p * m)
    assert np.array_equal(cond, rc) and np.array_equal(cnt, rn)
    if p == 1:
        assert np.array_equal(cond, B.vecchia_neighbors(ctx, s, m))


def test_nearest_group_rows_on_device(ctx):
    import torch
    s, _, _ = _ordered(1200, 5)
    cond, cnt = B.vecchia_group_conditioning(ctx, torch.from_numpy(s).cuda(), 3, 6, B.COND_NEAREST)
    rc, rn = O.group_cond_nearest(s, 3, 6, 18)
    assert np.array_equal(cond.cpu().numpy(), rc) and np.array_equal(cnt.cpu().numpy(), rn)


@pytest.mark.parametrize("D,p,k,seed", [(1000, 1, 20, 3), (1000, 5, 30, 4), (64, 2, 63, 5)])
def test_random_group_rows_bit_exact(ctx, D, p, k, seed):
    s, _, _ = _ordered(D, seed)
    cmax = min(k, 64 - p)
    k = min(k, cmax)
    cond, cnt = B.vecchia_group_conditioning(ctx, s, p, k, B.COND_RANDOM, seed=seed, cmax=cmax)
    rc, rn = O.group_cond_random(D, p, k, seed, cmax)
    assert np.array_equal(cond, rc) and np.array_equal(cnt, rn)


def test_union_overflow_is_an_argument_error(ctx):
    s, _, _ = _ordered(400, 9)
    with pytest.raises(B.VecchiaError) as e:
        B.vecchia_group_conditioning(ctx, s, 4, 5, B.COND_NEAREST, cmax=8)
    assert e.value.status == B.ERR_ARG


@pytest.mark.parametrize("prec", [B.FP64, B.MIXED])
@pytest.mark.parametrize("D,p,m,method", [(240, 3, 5, B.COND_NEAREST), (200, 4, 20, B.COND_RANDOM),
                                          (150, 10, 4, B.COND_NEAREST), (130, 2, 31, B.COND_NEAREST)])
def test_grouped_log_cdf_against_oracle(ctx, prec, D, p, m, method):
    s, u, cov = _ordered(D, 11 * p + m)
    cmax = p * m if method == B.COND_NEAREST else m
    cond, cnt = B.vecchia_group_conditioning(ctx, s, p, m, method, seed=3, cmax=cmax)
    rc, _ = (O.group_cond_nearest(s, p, m, cmax) if method == B.COND_NEAREST
             else O.group_cond_random(D, p, m, 3, cmax))
    assert np.array_equal(cond, rc)
    ref, ref_se = O.grouped_log_cdf(s, p, rc, cov, u, 512, 4, 17)
    lp, se = B.vecchia_grouped_log_cdf(ctx, s, p, cond, cov, u, 512, 4, seed=17, precision=prec)
    _check(lp, ref, prec)
    if prec == B.FP64:
        assert se == pytest.approx(ref_se, rel=1e-8)


@pytest.mark.parametrize("prec", [B.FP64, B.MIXED])
def test_groups_of_one_equal_classic_bit_for_bit(ctx, prec):
    s, u, cov = _ordered(500, 21, m=12)
    nbr = B.vecchia_neighbors(ctx, s, 12)
    a = B.vecchia_log_cdf(ctx, s, nbr, 12, cov, u, 1024, 8, 4, prec)
    b = B.vecchia_grouped_log_cdf(ctx, s, 1, nbr, cov, u, 1024, 8, seed=4, precision=prec)
    assert a == b


@pytest.mark.parametrize("prec", [B.FP64, B.MIXED])
@pytest.mark.parametrize("m", [40, 50])
def test_many_neighbours_log_cdf_against_oracle(ctx, prec, m):
    s, u, cov = _ordered(260, 30 + m, cov=(O.COV_EXPONENTIAL, 1.0, 0.5, 0.5, 0.0))
    nbr = B.vecchia_neighbors(ctx, s, m)
    rn = O.neighbors(s, m)
    assert np.array_equal(nbr, rn)
    ref, _ = O.log_cdf(s, rn, m, cov, u, 256, 4, 8)
    lp, _ = B.vecchia_log_cdf(ctx, s, nbr, m, cov, u, 256, 4, 8, prec)
    _check(lp, ref, prec)


def test_many_neighbours_per_shift_partials_fp64(ctx):
    s, u, cov = _ordered(120, 77)
    m = 45
    nbr = B.vecchia_neighbors(ctx, s, m)
    ro = O.neighbors(s, m)
    assert np.array_equal(nbr, ro)
    idx = np.array([0, 1, 44, 45, 46, 90, 119])
    rn, rd = O.vecchia_partials(s, ro, m, cov, u, 333, 3, 2, idx=idx)
    _, _, _, num, den = B.vecchia_log_cdf_terms(ctx, s, nbr, m, cov, u, 333, 3, 2, B.FP64)
    assert np.allclose(num[idx], rn, rtol=FP64_TOL, atol=0) and np.allclose(den[idx], rd, rtol=FP64_TOL, atol=0)


@pytest.mark.parametrize("prec", [B.FP64, B.MIXED])
def test_anisotropic_covariance_against_oracle(ctx, prec):
    cov = (B.COV_ANISO_EXP, 1.5, 0.2, 0.5, 0.01, 0.6, 2.5)
    s, u, _ = _ordered(300, 41)
    nbr = B.vecchia_neighbors(ctx, s, 10)
    ref, _ = O.grouped_log_cdf(s, 1, O.neighbors(s, 10), cov, u, 512, 4, 5)
    lp, _ = B.vecchia_log_cdf(ctx, s, nbr, 10, cov, u, 512, 4, 5, prec)
    _check(lp, ref, prec)


def test_deep_tail_with_large_blocks_uses_log_space_form(ctx):
    """u = -3 everywhere at m = 40: terms far below 2^-40 go through the
    log-space re-evaluation (instantiated for 64 variables)."""
    s, _, cov = _ordered(160, 61, cov=(O.COV_EXPONENTIAL, 1.0, 0.3, 0.5, 0.0))
    u = np.full(160, -3.0)
    nbr = B.vecchia_neighbors(ctx, s, 40)
    ref, _ = O.log_cdf(s, O.neighbors(s, 40), 40, cov, u, 256, 4, 1)
    lp, _ = B.vecchia_log_cdf(ctx, s, nbr, 40, cov, u, 256, 4, 1, B.MIXED)
    _check(lp, ref, B.MIXED)


def test_grouped_and_classic_problems_in_one_batch(ctx):
    s1, u1, cov1 = _ordered(300, 2)
    s2, u2, cov2 = _ordered(200, 3)
    nbr1 = B.vecchia_neighbors(ctx, s1, 20)
    cond2, _ = B.vecchia_group_conditioning(ctx, s2, 5, 8, B.COND_NEAREST)
    probs = [dict(sites=s1, nbr=nbr1, m=20, cov=cov1, u=u1, N=512, S=8, seed=1),
             dict(sites=s2, nbr=cond2, m=cond2.shape[1], cov=cov2, u=u2, N=512, S=8, seed=2, group=5)]
    for prec in (B.FP64, B.MIXED):
        lp, se, st = B.vecchia_log_cdf_batch(ctx, probs, prec)
        assert np.all(st == B.OK)
        a = B.vecchia_log_cdf(ctx, s1, nbr1, 20, cov1, u1, 512, 8, 1, prec)
        b = B.vecchia_grouped_log_cdf(ctx, s2, 5, cond2, cov2, u2, 512, 8, seed=2, precision=prec)
        assert (lp[0], se[0]) == a and (lp[1], se[1]) == b


def test_malformed_group_row_names_the_group(ctx):
    s, u, cov = _ordered(60, 4)
    cond, _ = B.vecchia_group_conditioning(ctx, s, 3, 4, B.COND_NEAREST)
    bad = cond.copy()
    k = 7
    bad[k, 0], bad[k, 1] = bad[k, 1], bad[k, 0]  # not ascending
    with pytest.raises(B.VecchiaError) as e:
        B.vecchia_grouped_log_cdf(ctx, s, 3, bad, cov, u, 128, 4, precision=B.MIXED)
    assert e.value.status == B.ERR_ARG and B.vecchia_last_error_site(ctx) == k


# ---- exact maxmin ordering on the device (Sec. 3.2 ordering by distance) ----

@pytest.mark.parametrize("D,kind", [(1, "u"), (2, "u"), (33, "u"), (1000, "u"), (2500, "grid"),
                                    (20000, "u"), (600, "dup")])
def test_device_maxmin_equals_oracle(ctx, D, kind):
    import torch
    if kind == "u":
        s = inputs.uniform_sites(D, D + 3)
    elif kind == "grid":
        s = inputs.grid_sites(int(round(math.sqrt(D))))
    else:  # every site three times: ties everywhere
        s = np.repeat(inputs.uniform_sites(D // 3, 8), 3, axis=0)
    ref = O.order(s, O.ORDER_MAXMIN)
    got = B.vecchia_order(ctx, s, "maxmin")
    assert np.array_equal(got, ref)
    got_d = B.vecchia_order(ctx, torch.from_numpy(s).cuda(), "maxmin")
    assert np.array_equal(got_d.cpu().numpy(), ref)


def test_device_maxmin_equals_host_ordering_at_large_size(ctx):
    s = inputs.large().sites[:100_000]
    assert np.array_equal(B.vecchia_order(ctx, s, "maxmin"), B.vecchia_order(None, s, "maxmin"))


# ---- full D-dimensional Genz (the m = D - 1 limit) --------------------------

@pytest.mark.parametrize("prec", [B.FP64, B.MIXED])
@pytest.mark.parametrize("D,N,S", [(1, 256, 4), (2, 256, 4), (150, 512, 4), (600, 300, 4)])
def test_full_genz_against_oracle(ctx, prec, D, N, S):
    s, u, cov = _ordered(D, 500 + D, cov=(O.COV_EXPONENTIAL, 1.0, 0.3, 0.5, 0.0))
    ref, ref_se = O.full_genz(s, cov, u, N, S, 3)
    lp, se = B.vecchia_full_genz(ctx, s, cov, u, N, S, seed=3, precision=prec)
    _check(lp, ref, prec)
    if prec == B.FP64 and D > 1:
        assert se == pytest.approx(ref_se, rel=1e-6)


@pytest.mark.parametrize("D,N,S", [(64, 224, 2),    # one full panel, one exact tile of points
                                   (65, 225, 3),    # two panels (the pair's own chunks only), a ragged tile
                                   (129, 448, 2),   # three panels: the last pair has one panel
                                   (256, 100, 4),   # four panels, one partial tile per shift
                                   (321, 673, 2)])  # five panels, three tiles per shift, ragged
def test_full_genz_panel_pairs_against_oracle(ctx, D, N, S):
    """The mixed recursion on the tensor cores takes panels of 64 variables in
    pairs over tiles of 224 points: panel counts odd and even, tiles exact and
    ragged."""
    s, u, cov = _ordered(D, 900 + D, cov=(B.COV_MATERN, 1.0, 0.25, 1.5, 0.0))
    ref, _ = O.full_genz(s, cov, u, N, S, 7)
    lp, _ = B.vecchia_full_genz(ctx, s, cov, u, N, S, seed=7, precision=B.MIXED)
    _check(lp, ref, B.MIXED)


@pytest.mark.parametrize("prec", [B.FP64, B.MIXED])
def test_full_genz_equals_vecchia_with_every_neighbour(ctx, prec):
    """Eq. (vecchia-cdf) with m = D - 1 telescopes to the full estimate."""
    D = 60
    s, u, cov = _ordered(D, 77, cov=(B.COV_MATERN, 1.0, 0.2, 1.5, 0.0))
    nbr = B.vecchia_neighbors(ctx, s, D - 1)
    a, _ = B.vecchia_log_cdf(ctx, s, nbr, D - 1, cov, u, 1024, 8, 5, prec)
    b, _ = B.vecchia_full_genz(ctx, s, cov, u, 1024, 8, seed=5, precision=prec)
    assert abs(a - b) <= (1e-10 * abs(b) if prec == B.FP64 else mixed_tol(b))


def test_full_genz_singular_covariance_is_not_pd(ctx):
    """Sites 0 and 1 equal, no nugget: the second pivot is exactly 0."""
    s, u, cov = _ordered(40, 12)
    s[1] = s[0]
    with pytest.raises(O.OracleError):
        O.full_genz(s, cov, u, 256, 4, 0)
    with pytest.raises(B.VecchiaError) as e:
        B.vecchia_full_genz(ctx, s, cov, u, 256, 4, precision=B.FP64)
    assert e.value.status == B.ERR_NOT_PD and B.vecchia_last_error_site(ctx) == 1


@pytest.mark.parametrize("D,kind", [(1, "u"), (3, "u"), (2500, "grid"), (5000, "u"), (8192, "u"), (8193, "u"),
                                    (999, "dup")])
def test_device_xy_order_equals_oracle(ctx, D, kind):
    import torch
    if kind == "grid":
        s = inputs.grid_sites(50)[::-1].copy()  # many equal x: y and then the index decide
    elif kind == "dup":
        s = np.repeat(inputs.uniform_sites(D // 3, 5), 3, axis=0)
    else:
        s = inputs.uniform_sites(D, D)
    ref = O.order(s, O.ORDER_XY)
    got = B.vecchia_order(ctx, torch.from_numpy(s).cuda(), "xy")
    assert np.array_equal(got.cpu().numpy(), ref)


@pytest.mark.parametrize("order,D,m,device", [("xy", 2500, 20, True), ("xy", 2500, 20, False), ("maxmin", 1500, 12, True),
                                              ("identity", 700, 8, False), ("xy", 9000, 5, True)])
def test_unordered_call_equals_the_four_calls(ctx, order, D, m, device):
    """vecchia_log_cdf_unordered gives exactly the results of order, apply_order,
    neighbors and log_cdf called one after the other."""
    import torch
    prob = inputs.grid50(m=m) if D == 2500 else inputs.small_random(D, D, m=m, N=512, S=4)
    s, u = prob.sites, prob.u
    if device:
        s, u = torch.from_numpy(s).cuda(), torch.from_numpy(u).cuda()
    perm = B.vecchia_order(ctx if device else None, s, order)
    so, uo = B.vecchia_apply_order(ctx if device else None, perm, s, u)
    nbr = B.vecchia_neighbors(ctx, so, m)
    ref = B.vecchia_log_cdf(ctx, so, nbr, m, prob.cov, uo, prob.N, prob.S, 3, B.MIXED)
    got_perm = np.zeros(D, np.int32)
    got = B.vecchia_log_cdf_unordered(ctx, s, u, m, prob.cov, prob.N, prob.S, 3, B.MIXED, order=order,
                                      perm_out=got_perm)
    assert got == ref
    p_ref = perm.cpu().numpy() if device else perm
    assert np.array_equal(got_perm, p_ref)


def test_grouped_block_size_from_the_longest_row(ctx):
    """Grouped rows are often far shorter than their width: the grouped call
    sizes its kernel by the longest row (cond_max), and a batch with the
    hint equals one without it bit for bit; a hint shorter than a row makes
    that group fail with VECCHIA_ERR_ARG."""
    import torch
    prob = inputs.grid50(m=5, N=512, S=4)  # on the grid in xy order the members' neighbours overlap
    perm = O.order(prob.sites, O.ORDER_XY)
    s = torch.from_numpy(np.ascontiguousarray(prob.sites[perm])).cuda()
    u = torch.from_numpy(np.ascontiguousarray(prob.u[perm])).cuda()
    p, m = 5, 5
    cond, cnt = B.vecchia_group_conditioning(ctx, s, p, m, B.COND_NEAREST, seed=1, cmax=p * m)
    cmax_used = int(cnt.max().item())
    assert 1 + p < cmax_used + p <= 21 < p * m + p  # a smaller kernel than the row width asks for
    for prec in (B.FP64, B.MIXED):
        lp, se = B.vecchia_grouped_log_cdf(ctx, s, p, cond, prob.cov, u, prob.N, prob.S, seed=3, precision=prec)
        item = dict(sites=s, nbr=cond, m=p * m, cov=prob.cov, u=u, N=prob.N, S=prob.S, seed=3, group=p)
        ref = B.vecchia_log_cdf_batch(ctx, [item], prec)             # bucket from the row width
        hint = B.vecchia_log_cdf_batch(ctx, [dict(item, cond_max=cmax_used)], prec)
        assert (lp, se) == (ref[0][0], ref[1][0]) == (hint[0][0], hint[1][0])
        short = B.vecchia_log_cdf_batch(ctx, [dict(item, cond_max=1), item], prec)  # a 9-variable kernel
        assert short[2][0] == B.ERR_ARG and short[2][1] == B.OK and short[0][1] == lp
