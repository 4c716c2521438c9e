"""The continuous-batching loop on the GPU: requests of different D, m and
covariance parameters arriving over time are admitted under an HBM budget,
advanced together chunk by chunk, and each result equals the one computed
alone (bit for bit: a term's partial sums do not depend on the mix)."""
import numpy as np
import pytest

from paper_2007_15195_gb300 import binding as B
from paper_2007_15195_gb300 import inputs
from paper_2007_15195_gb300.serve import Server, footprint_bytes, requests_from_stream

from _prep import mixed_tol

pytestmark = pytest.mark.gpu


def test_results_alone_equal_results_in_the_mix():
    stream = inputs.serving_stream(n_requests=24, rate_hz=400.0, d_lo=100, d_hi=3000, N=1024, S=8)
    reqs = requests_from_stream(stream)
    budget = sum(sorted(footprint_bytes(r.D, r.m, r.S) for r in reqs)[-6:])  # forces queueing
    with B.Context(0) as ctx:
        srv = Server(ctx, B.MIXED, hbm_budget_bytes=budget, max_active=8, chunk_sites=256,
                     iter_sites=2048)
        stats = srv.run(reqs)
        srv.close()
        assert stats["completed"] == len(reqs) and stats["ok"] == len(reqs)
        assert stats["peak_resident_bytes"] <= budget
        assert stats["iterations"] > len(reqs)  # requests were split across iterations
        # some requests were admitted while others were still running
        overlapped = sum(1 for a in reqs for b in reqs
                         if a.rid != b.rid and a.t_admit < b.t_admit < a.t_done)
        assert overlapped > 0
        for r in reqs:
            perm = B.vecchia_order(None, r.sites, r.order)
            s, u = B.vecchia_apply_order(None, perm, r.sites, r.u)
            nbr = B.vecchia_neighbors(ctx, s, r.m)
            lp, se = B.vecchia_log_cdf(ctx, s, nbr, r.m, r.cov, u, r.N, r.S, r.seed, B.MIXED)
            assert abs(r.log_p - lp) <= mixed_tol(lp)
            assert r.log_p == lp and r.std_err == se


def test_fp64_serving_and_a_failing_request():
    stream = inputs.serving_stream(n_requests=6, rate_hz=1000.0, d_lo=100, d_hi=600, N=256, S=4)
    reqs = requests_from_stream(stream)
    bad = reqs[2]
    bad.sites = bad.sites.copy()
    bad.sites[5] = bad.sites[4]  # duplicated site: a covariance block is singular
    with B.Context(0) as ctx:
        srv = Server(ctx, B.FP64, chunk_sites=128, iter_sites=512)
        stats = srv.run(reqs)
        srv.close()
        assert stats["completed"] == len(reqs)
        assert bad.status == B.ERR_NOT_PD and np.isnan(bad.log_p)
        for r in reqs:
            if r is bad:
                continue
            perm = B.vecchia_order(None, r.sites, r.order)
            s, u = B.vecchia_apply_order(None, perm, r.sites, r.u)
            nbr = B.vecchia_neighbors(ctx, s, r.m)
            lp, se = B.vecchia_log_cdf(ctx, s, nbr, r.m, r.cov, u, r.N, r.S, r.seed, B.FP64)
            assert r.status == B.OK and r.log_p == lp
