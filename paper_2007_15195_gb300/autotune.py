"""Tile autotuner for the fused Genz kernel.

A tile is (warps per CTA, points per lane, lattice slices per shift, shift
groups per site): it changes only the launch shape, so results are identical
for equal `slices` (and equal up to FP summation order otherwise).  The tuner
times every candidate on the caller's own workload with the library's CUDA
events around the Genz launches (vecchia_genz_time_ms), keeps the fastest,
and caches it per (device, precision, bucket, N, S, size class) in a JSON file
so later processes start from the tuned tile.
"""
import json
import math
import os
import time

import numpy as np

from . import binding as B

# DMAX of each bucket (a problem whose largest term has d variables -- m + 1,
# or m + p for groups of p -- uses the first DMAX >= d)
BUCKET_DMAX = (9, 13, 17, 21, 25, 29, 32, 48, 64)

DEFAULT_CANDIDATES = [(w, p, 1, g) for w in (2, 4, 8) for p in (1, 2) for g in (1, 2, 4, 8)]


def bucket_of(m, group=0):
    need = m + (group if group > 0 else 1)
    for b, d in enumerate(BUCKET_DMAX):
        if need <= d:
            return b
    raise ValueError("terms of more than 64 variables")


def default_cache_path():
    base = os.environ.get("XDG_CACHE_HOME", os.path.join(os.path.expanduser("~"), ".cache"))
    return os.path.join(base, "paper_2007_15195_gb300", "tiles.json")


def _device_name(device):
    try:
        import torch
        return torch.cuda.get_device_name(device)
    except Exception:  # pragma: no cover
        return "cuda:%d" % device


def _key(ctx, precision, problems):
    buckets = sorted({bucket_of(int(p["m"]), int(p.get("group", 0))) for p in problems})
    Ns = sorted({int(p["N"]) for p in problems})
    Ss = sorted({int(p["S"]) for p in problems})
    sites = sum(int(p["sites"].shape[0]) for p in problems)
    size_class = 1 << max(0, int(math.ceil(math.log2(max(sites, 1)))))
    return "|".join([_device_name(ctx.device), "mixed" if precision == B.MIXED else "fp64",
                     "b" + ",".join(map(str, buckets)), "N" + ",".join(map(str, Ns)),
                     "S" + ",".join(map(str, Ss)), "sites<=%d" % size_class])


def _load(path):
    try:
        with open(path) as f:
            return json.load(f)
    except (OSError, ValueError):
        return {}


def _save(path, cache):
    os.makedirs(os.path.dirname(path), exist_ok=True)
    tmp = path + ".tmp%d" % os.getpid()
    with open(tmp, "w") as f:
        json.dump(cache, f, indent=1, sort_keys=True)
    os.replace(tmp, path)


def _time_tile(ctx, problems, precision, tile, reps):
    B.vecchia_set_tile(ctx, precision, -1, *tile)
    run = (lambda: B.vecchia_log_cdf_batch(ctx, problems, precision)) if len(problems) > 1 else \
        (lambda: B.vecchia_log_cdf(ctx, problems[0]["sites"], problems[0]["nbr"], problems[0]["m"],
                                   problems[0]["cov"], problems[0]["u"], problems[0]["N"],
                                   problems[0]["S"], problems[0].get("seed", 0), precision))
    run()  # first call may grow buffers
    ts = []
    for _ in range(reps):
        run()
        ts.append(B.vecchia_genz_time_ms(ctx))
    return float(np.median(ts))


def tune(ctx, problems, precision=B.MIXED, candidates=None, reps=3, cache_path=None, force=False,
         budget_s=None):
    """Pick the fastest tile for this workload and set it on ctx.

    problems: list of dicts (sites, nbr, m, cov, u, N, S, seed) as for
    vecchia_log_cdf_batch.  Returns {"tile": (warps, points, slices, groups),
    "ms": genz ms, "key": cache key, "cached": bool, "timings": [...]}.
    """
    cache_path = cache_path or default_cache_path()
    key = _key(ctx, precision, problems)
    cache = _load(cache_path)
    if not force and key in cache:
        tile = tuple(cache[key]["tile"])
        B.vecchia_set_tile(ctx, precision, -1, *tile)
        return {"tile": tile, "ms": cache[key]["ms"], "key": key, "cached": True, "timings": []}
    B.vecchia_set_timing(ctx, True)
    cands = list(candidates or DEFAULT_CANDIDATES)
    if precision == B.FP64:
        cands = sorted({(w, 1, s, g) for (w, p, s, g) in cands})
    timings = []
    t0 = time.perf_counter()
    for tile in cands:
        ms = _time_tile(ctx, problems, precision, tile, reps)
        timings.append((ms, tile))
        if budget_s is not None and time.perf_counter() - t0 > budget_s:
            break
    timings.sort()
    best_ms, best = timings[0]
    B.vecchia_set_tile(ctx, precision, -1, *best)
    cache[key] = {"tile": list(best), "ms": best_ms, "when": time.time()}
    _save(cache_path, cache)
    return {"tile": best, "ms": best_ms, "key": key, "cached": False,
            "timings": [(ms, list(t)) for ms, t in timings]}
