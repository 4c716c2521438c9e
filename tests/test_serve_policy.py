"""Host-side policy of the continuous-batching loop (no GPU): admission by
device footprint and free slots, and the round-robin share of an iteration."""
from paper_2007_15195_gb300.serve import admit, footprint_bytes, plan_iteration


def test_footprint_counts_resident_arrays():
    D, m, S = 1000, 20, 8
    assert footprint_bytes(D, m, S) == 16 * D + 8 * D + 4 * D * m + 16 * D * S + 32


def test_admit_is_fifo_and_respects_budget_and_slots():
    ready = [("a", 100), ("b", 300), ("c", 50), ("d", 10)]
    assert admit(ready, 0, 1000, 0, 10) == ["a", "b", "c", "d"]
    # budget stops at b; c and d do not overtake it
    assert admit(ready, 700, 1000, 0, 10) == ["a"]
    assert admit(ready, 0, 1000, 8, 10) == ["a", "b"]
    assert admit(ready, 0, 1000, 10, 10) == []
    assert admit([], 0, 10, 0, 1) == []


def test_plan_iteration_round_robin_caps():
    active = [("x", 10_000, 0), ("y", 500, 400), ("z", 3000, 2990)]
    plan = plan_iteration(active, chunk_sites=2048, iter_sites=100_000)
    assert plan == [("x", 0, 2048), ("y", 400, 100), ("z", 2990, 10)]
    # total cap, rotating start
    plan = plan_iteration(active, chunk_sites=2048, iter_sites=2100, start=1)
    assert plan == [("y", 400, 100), ("z", 2990, 10), ("x", 0, 1990)]
    assert sum(c for _, _, c in plan) == 2100


def test_plan_iteration_covers_every_site_exactly_once():
    D = {"p": 7001, "q": 123, "r": 4096}
    pos = {k: 0 for k in D}
    seen = {k: [] for k in D}
    start = 0
    while any(pos[k] < D[k] for k in D):
        active = [(k, D[k], pos[k]) for k in sorted(D) if pos[k] < D[k]]
        for k, b, c in plan_iteration(active, 1000, 2500, start):
            assert b == pos[k]
            seen[k].append((b, c))
            pos[k] = b + c
        start += 1
    for k in D:
        covered = sorted(seen[k])
        assert covered[0][0] == 0 and sum(c for _, c in covered) == D[k]
        for (b1, c1), (b2, _) in zip(covered, covered[1:]):
            assert b1 + c1 == b2
