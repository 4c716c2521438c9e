"""Batched evaluation: many independent problems in one launch sequence, and
plans (a batch kept resident and replayed as a CUDA graph with new seeds or
covariance parameters, as a likelihood optimiser would call it, Sec. 4.1).

The batched workload: problems with D log-uniform in [50, 2000], sites
uniform in the unit square, maxmin order, exponential covariance with range
~ U[0.05, 0.5], u = Phi^{-1}(0.9), m = 20, N = 2,048 x S = 8."""
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


def _gpu_items(ctx, probs, device=True):
    import torch
    items = []
    for p in probs:
        perm = B.vecchia_order(None, p.sites, p.order)
        s, u = B.vecchia_apply_order(None, perm, p.sites, p.u)
        if device:
            s, u = torch.from_numpy(s).cuda(), torch.from_numpy(u).cuda()
        nbr = B.vecchia_neighbors(ctx, s, p.m)
        items.append(dict(sites=s, nbr=nbr, m=p.m, cov=p.cov, u=u, N=p.N, S=p.S, seed=p.seed))
    return items


@pytest.fixture(scope="module")
def batch256(ctx):
    probs = inputs.batch_problems(256)
    return probs, _gpu_items(ctx, probs)


def test_batch_matches_oracle_on_sampled_problems(ctx, batch256):
    probs, items = batch256
    lp, se, st = B.vecchia_log_cdf_batch(ctx, items, B.MIXED)
    assert np.all(st == B.OK)
    assert np.all(np.isfinite(lp)) and np.all(lp < 0)
    order = np.argsort([p.D for p in probs])
    for k in list(order[:3]) + [order[len(order) // 2]]:
        p = probs[k]
        perm = O.order(p.sites, O.ORDER_MAXMIN)
        s, u = p.sites[perm], p.u[perm]
        nbr = O.neighbors(s, p.m)
        assert np.array_equal(nbr, items[k]["nbr"].cpu().numpy())
        ref, ref_se = O.log_cdf(s, nbr, p.m, p.cov, u, p.N, p.S, p.seed)
        assert abs(lp[k] - ref) <= mixed_tol(ref), (k, lp[k], ref)


def test_plan_equals_batch_and_replays(ctx, batch256):
    probs, items = batch256
    sub = items[:64]
    ref = B.vecchia_log_cdf_batch(ctx, sub, B.MIXED)
    plan = B.Plan(ctx, sub, B.MIXED)
    try:
        assert np.all(plan.status == B.OK)
        got = plan.run()
        assert np.array_equal(got[0], ref[0]) and np.array_equal(got[1], ref[1])
        # new seeds and a new range for every problem, as an optimiser step would
        seeds = np.arange(64, dtype=np.uint64) + 1000
        covs = [(B.COV_EXPONENTIAL, 1.0, 0.8 * it["cov"][2], 0.5, 0.0) for it in sub]
        got2 = plan.run(seeds=seeds, covs=covs)
        moved = [dict(it, seed=int(sd), cov=cv) for it, sd, cv in zip(sub, seeds, covs)]
        ref2 = B.vecchia_log_cdf_batch(ctx, moved, B.MIXED)
        assert np.array_equal(got2[0], ref2[0]) and np.array_equal(got2[1], ref2[1])
        assert not np.array_equal(got2[0], got[0])
        # and back
        got3 = plan.run(seeds=np.array([it["seed"] for it in sub], dtype=np.uint64),
                        covs=[it["cov"] for it in sub])
        assert np.array_equal(got3[0], ref[0])
    finally:
        plan.close()


def test_plan_fp64_and_bad_cov(ctx, batch256):
    probs, items = batch256
    sub = items[:4]
    plan = B.Plan(ctx, sub, B.FP64)
    try:
        got = plan.run()
        ref = B.vecchia_log_cdf_batch(ctx, sub, B.FP64)
        assert np.array_equal(got[0], ref[0])
        with pytest.raises(B.VecchiaError) as e:
            plan.run(covs=[(B.COV_MATERN, 1.0, 0.1, 0.7, 0.0)] * 4)
        assert e.value.status == B.ERR_ARG
    finally:
        plan.close()


def test_plan_with_host_inputs_is_resident(ctx):
    probs = inputs.batch_problems(8, workload_seed=3, d_hi=300)
    items = _gpu_items(ctx, probs, device=False)
    plan = B.Plan(ctx, items, B.MIXED)
    try:
        ref = B.vecchia_log_cdf_batch(ctx, items, B.MIXED)
        for it in items:  # the plan copied host inputs at creation
            it["sites"][:] = 0.0
        got = plan.run()
        assert np.array_equal(got[0], ref[0])
    finally:
        plan.close()


def test_autotune_picks_and_caches_a_tile(ctx, batch256, tmp_path):
    from paper_2007_15195_gb300 import autotune
    probs, items = batch256
    sub = items[:32]
    cands = [(4, 1, 1, 1), (8, 1, 1, 2), (2, 2, 1, 1)]
    path = str(tmp_path / "tiles.json")
    r = autotune.tune(ctx, sub, B.MIXED, candidates=cands, reps=1, cache_path=path)
    assert not r["cached"] and tuple(r["tile"]) in cands and len(r["timings"]) == 3
    lp_tuned = B.vecchia_log_cdf_batch(ctx, sub, B.MIXED)[0]
    r2 = autotune.tune(ctx, sub, B.MIXED, candidates=cands, reps=1, cache_path=path)
    assert r2["cached"] and tuple(r2["tile"]) == tuple(r["tile"])
    B.vecchia_reset_tiles(ctx)
    lp_default = B.vecchia_log_cdf_batch(ctx, sub, B.MIXED)[0]
    assert np.array_equal(lp_tuned, lp_default)  # slices = 1: bit-identical


@pytest.mark.parametrize("prec", [B.FP64, B.MIXED])
def test_mixture_log_cdf_against_oracle(ctx, prec):
    """Sec. 4 scale mixture: n_nodes Vecchia log-CDFs with scaled covariance in
    one batch, combined by the quadrature rule."""
    prob = inputs.small_random(150, 23, m=10, N=512, S=4)
    perm = O.order(prob.sites, O.ORDER_MAXMIN)
    s, u = prob.sites[perm], prob.u[perm] + 1.0
    nbr = O.neighbors(s, 10)
    ref = O.mixture_log_cdf(s, nbr, 10, prob.cov, u, 512, 4, 5, 0.6, 1.2, 10)
    lg, se = B.vecchia_mixture_log_cdf(ctx, s, nbr, 10, prob.cov, u, 512, 4, 5, beta=0.6, gamma=1.2,
                                       n_nodes=10, precision=prec)
    tol = 1e-10 * abs(ref) if prec == B.FP64 else mixed_tol(ref)
    assert abs(lg - ref) <= tol, (lg, ref)
    assert se > 0
