"""Continuous-batching request loop for Vecchia log-CDF evaluations.

Requests (sites, thresholds, covariance, m, N, S, seed) arrive over time, as
a likelihood optimiser or many concurrent ones would issue them (Sec. 4.1).
The loop keeps every admitted request's sites, thresholds, neighbour lists
and partial sums resident on the device and advances all of them together:

  * host preparation (ordering, applying it) runs on a thread pool as soon as
    a request arrives;
  * admission: a prepared request enters when its device footprint fits the
    HBM budget next to the resident requests and a slot is free (first come,
    first served); its upload and neighbour search are queued on the stream;
  * iteration: every active request contributes its next chunk of sites to
    one vecchia_partials_async call (the Genz terms of all of them in one set
    of launches); requests whose last chunk is in the iteration get their
    log-sum (vecchia_reduce_async) and a copy of their result slot behind it;
  * up to `max_in_flight` iterations are queued at once, so a request that
    arrives while others run is admitted and joins the next iteration, and its
    work overlaps theirs on the device;
  * a finished request frees its memory, which admits the next ones.

A term's partial sums do not depend on which chunks or neighbours-in-the-mix
it was launched with, so every result equals the one computed alone.
"""
import time
from concurrent.futures import ThreadPoolExecutor
from dataclasses import dataclass, field
from typing import List, Optional

import numpy as np

from . import binding as B

RESULT_BYTES = 32


@dataclass
class ServeRequest:
    rid: int
    arrival_s: float
    sites: np.ndarray
    u: np.ndarray
    cov: tuple
    m: int
    N: int
    S: int
    seed: int = 0
    order: str = "xy"
    # filled by the server
    t_ready: Optional[float] = None
    t_admit: Optional[float] = None
    t_done: Optional[float] = None
    log_p: float = float("nan")
    std_err: float = float("nan")
    status: Optional[int] = None

    @property
    def D(self):
        return int(self.sites.shape[0])


def footprint_bytes(D, m, S):
    """Device bytes a resident request holds: sites, thresholds, neighbours,
    per-shift partial sums and its result slot."""
    return 16 * D + 8 * D + 4 * D * max(m, 1) + 16 * D * S + RESULT_BYTES


def admit(ready, resident_bytes, budget_bytes, n_active, max_active):
    """First come, first served: the longest prefix of `ready` (list of
    (key, footprint)) that fits the budget and the free slots."""
    out = []
    for key, fp in ready:
        if n_active + len(out) >= max_active or resident_bytes + fp > budget_bytes:
            break
        out.append(key)
        resident_bytes += fp
    return out


def plan_iteration(active, chunk_sites, iter_sites, start=0):
    """Round-robin share of one iteration: active is a list of (key, D, pos)
    with pos < D; returns [(key, begin, count)], at most chunk_sites per
    request and iter_sites in total, starting at index `start`."""
    out = []
    budget = iter_sites
    n = len(active)
    for k in range(n):
        if budget <= 0:
            break
        key, D, pos = active[(start + k) % n]
        cnt = min(chunk_sites, D - pos, budget)
        if cnt > 0:
            out.append((key, pos, cnt))
            budget -= cnt
    return out


@dataclass
class _Live:
    req: ServeRequest
    sites: object = None
    u: object = None
    nbr: object = None
    num: object = None
    den: object = None
    result: object = None
    host_result: object = None
    pinned: list = field(default_factory=list)
    pos: int = 0
    footprint: int = 0


class Server:
    def __init__(self, ctx, precision=B.MIXED, hbm_budget_bytes=16 << 30, max_active=256,
                 chunk_sites=2048, iter_sites=65536, max_in_flight=2, prep_workers=8):
        import torch
        self.torch = torch
        self.ctx = ctx
        self.precision = precision
        self.budget = int(hbm_budget_bytes)
        self.max_active = int(max_active)
        self.chunk = int(chunk_sites)
        self.iter_sites = int(iter_sites)
        self.max_in_flight = int(max_in_flight)
        self.dev = torch.device("cuda", ctx.device)
        self.stream = torch.cuda.current_stream(self.dev)
        self.pool = ThreadPoolExecutor(prep_workers)

    # -- host preparation (thread pool) --
    @staticmethod
    def _prepare(req):
        perm = B.vecchia_order(None, req.sites, req.order)
        s, u = B.vecchia_apply_order(None, perm, req.sites, req.u)
        return s, u

    def _admit_one(self, live, prepared):
        torch = self.torch
        req = live.req
        s_np, u_np = prepared
        D, m, S = req.D, req.m, req.S
        s_pin = torch.from_numpy(s_np).pin_memory()
        u_pin = torch.from_numpy(u_np).pin_memory()
        live.pinned = [s_pin, u_pin]  # alive until the copies have run
        live.sites = s_pin.to(self.dev, non_blocking=True)
        live.u = u_pin.to(self.dev, non_blocking=True)
        live.nbr = torch.empty((D, max(m, 1)), dtype=torch.int32, device=self.dev)
        if m > 0:
            B.vecchia_neighbors_async(self.ctx, live.sites, m, out=live.nbr)
        live.num = torch.empty((D, S), dtype=torch.float64, device=self.dev)
        live.den = torch.empty((D, S), dtype=torch.float64, device=self.dev)
        live.result = torch.empty(RESULT_BYTES, dtype=torch.uint8, device=self.dev)
        live.host_result = torch.empty(RESULT_BYTES, dtype=torch.uint8, pin_memory=True)
        B.vecchia_result_init(self.ctx, live.result, 1)
        live.footprint = footprint_bytes(D, m, S)

    def _segment(self, live, begin, count):
        r = live.req
        return B.make_segment(live.sites, live.nbr, live.u, r.m, r.cov, r.N, r.S, r.seed, live.num,
                              live.den, live.result.data_ptr(), begin, count)

    def run(self, requests: List[ServeRequest], time_scale=1.0, max_wall_s=None):
        """Serve `requests` (sorted by arrival_s, seconds from start, scaled by
        time_scale).  Returns a stats dict; the requests are filled in place."""
        torch = self.torch
        reqs = sorted(requests, key=lambda r: r.arrival_s)
        t0 = time.perf_counter()
        clock = lambda: time.perf_counter() - t0
        nxt = 0                      # next request to arrive
        preparing = {}               # rid -> (live, future)
        ready = []                   # [(live, prepared)] FIFO
        active: List[_Live] = []
        in_flight = []               # [(event, [live finishing])]
        resident = peak_resident = 0
        rr = 0
        n_iter = 0
        done = 0
        while done < len(reqs):
            now = clock()
            if max_wall_s is not None and now > max_wall_s:
                break
            while nxt < len(reqs) and reqs[nxt].arrival_s * time_scale <= now:
                r = reqs[nxt]
                preparing[r.rid] = (_Live(r), self.pool.submit(self._prepare, r))
                nxt += 1
            for rid in [k for k, (_, f) in preparing.items() if f.done()]:
                live, f = preparing.pop(rid)
                live.req.t_ready = clock()
                ready.append((live, f.result()))
            ready.sort(key=lambda x: x[0].req.arrival_s)
            keys = admit([(i, footprint_bytes(lv.req.D, lv.req.m, lv.req.S)) for i, (lv, _) in enumerate(ready)],
                         resident, self.budget, len(active), self.max_active)
            for i in keys:
                live, prepared = ready[i]
                self._admit_one(live, prepared)
                live.req.t_admit = clock()
                resident += live.footprint
                active.append(live)
            ready = [x for i, x in enumerate(ready) if i not in set(keys)]
            peak_resident = max(peak_resident, resident)
            # queue an iteration
            if active and len(in_flight) < self.max_in_flight:
                plan = plan_iteration([(i, lv.req.D, lv.pos) for i, lv in enumerate(active)], self.chunk,
                                      self.iter_sites, rr)
                if plan:
                    rr = (rr + 1) % max(len(active), 1)
                    segs = [self._segment(active[i], b, c) for i, b, c in plan]
                    B.vecchia_partials_async(self.ctx, segs, self.precision)
                    finishing = []
                    for i, b, c in plan:
                        active[i].pos = b + c
                        if active[i].pos >= active[i].req.D:
                            finishing.append(active[i])
                    if finishing:
                        B.vecchia_reduce_async(self.ctx, [self._segment(lv, 0, 0) for lv in finishing])
                        for lv in finishing:
                            lv.host_result.copy_(lv.result, non_blocking=True)
                    ev = torch.cuda.Event()
                    ev.record(self.stream)
                    in_flight.append((ev, finishing))
                    active = [lv for lv in active if lv.pos < lv.req.D]
                    n_iter += 1
                    continue
            # retire finished iterations
            progressed = False
            while in_flight and in_flight[0][0].query():
                _, finishing = in_flight.pop(0)
                t = clock()
                for lv in finishing:
                    rec = np.frombuffer(lv.host_result.numpy().tobytes(), dtype=B.RESULT_DTYPE)[0]
                    r = lv.req
                    r.status = int(rec["status"])
                    r.log_p = float(rec["log_p"]) if r.status == 0 else float("nan")
                    r.std_err = float(rec["std_err"]) if r.status == 0 else float("nan")
                    r.t_done = t
                    resident -= lv.footprint
                    done += 1
                progressed = True
            if progressed:
                continue
            if in_flight and (not active or len(in_flight) >= self.max_in_flight):
                in_flight[0][0].synchronize()
            elif not in_flight and not active:
                if nxt < len(reqs):
                    wait = reqs[nxt].arrival_s * time_scale - clock()
                    if wait > 0:
                        time.sleep(min(wait, 0.001))
                elif preparing:
                    time.sleep(0.0002)
        wall = clock()
        fin = [r for r in reqs if r.t_done is not None]
        lat = np.array([r.t_done - r.arrival_s * time_scale for r in fin]) if fin else np.zeros(0)
        wait = np.array([r.t_admit - r.arrival_s * time_scale for r in fin]) if fin else np.zeros(0)
        t_first = reqs[0].arrival_s * time_scale if reqs else 0.0
        t_last = max((r.t_done for r in fin), default=t_first)
        return {
            "completed": len(fin), "submitted": len(reqs), "iterations": n_iter, "wall_s": wall,
            "throughput_rps": len(fin) / max(t_last - t_first, 1e-9),
            "p50_ms": float(np.percentile(lat, 50) * 1e3) if len(lat) else None,
            "p99_ms": float(np.percentile(lat, 99) * 1e3) if len(lat) else None,
            "wait_p50_ms": float(np.percentile(wait, 50) * 1e3) if len(wait) else None,
            "wait_p99_ms": float(np.percentile(wait, 99) * 1e3) if len(wait) else None,
            "peak_resident_bytes": int(peak_resident), "budget_bytes": self.budget,
            "ok": int(sum(1 for r in fin if r.status == 0)),
        }

    def close(self):
        self.pool.shutdown(wait=True)


def requests_from_stream(stream, order="xy"):
    """ServeRequests from paper_2007_15195_gb300.inputs.serving_stream()."""
    out = []
    for k, rq in enumerate(stream):
        p = rq.problem
        out.append(ServeRequest(rid=k, arrival_s=rq.arrival_s, sites=p.sites, u=p.u, cov=p.cov, m=p.m,
                                N=p.N, S=p.S, seed=p.seed, order=order))
    return out
