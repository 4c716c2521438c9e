"""Sharding across ranks (CPU, world size 2, gloo): the Vecchia terms are
independent given sites, order and neighbour lists (Sec. 3.1), so ranks take
contiguous ranges of sites, compute their per-shift partial means, and one
all-gather plus an ordered reduction gives the unsplit result bit for bit.
This is the layout a multi-GPU deployment uses; the oracle stands in for the
per-rank device work."""
import os
import socket

import numpy as np
import pytest
import torch
import torch.distributed as dist
import torch.multiprocessing as mp

import oracle as O
from paper_2007_15195_gb300 import inputs


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _problem():
    prob = inputs.small_random(240, 17, m=6, N=128, S=4)
    perm = O.order(prob.sites, O.ORDER_MAXMIN)
    s, u = prob.sites[perm], prob.u[perm]
    return prob, s, u, O.neighbors(s, prob.m)


def _worker(rank, world, port, out_path):
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    prob, s, u, nbr = _problem()
    D = s.shape[0]
    lo, hi = D * rank // world, D * (rank + 1) // world
    num, den = O.vecchia_partials(s, nbr, prob.m, prob.cov, u, prob.N, prob.S, prob.seed,
                                  idx=np.arange(lo, hi))
    part = torch.from_numpy(np.concatenate([num.ravel(), den.ravel()]))
    # ranks hold ranges of different length: gather padded to the longest
    longest = (D // world + 1) * prob.S * 2
    padded = torch.zeros(longest, dtype=torch.float64)
    padded[: part.numel()] = part
    bufs = [torch.zeros(longest, dtype=torch.float64) for _ in range(world)]
    dist.all_gather(bufs, padded)
    if rank == 0:
        nums, dens = [], []
        for r, b in enumerate(bufs):
            n_r = (D * (r + 1) // world - D * r // world) * prob.S
            nums.append(b[:n_r].numpy().reshape(-1, prob.S))
            dens.append(b[n_r:2 * n_r].numpy().reshape(-1, prob.S))
        lp, se, _ = O.vecchia_reduce(np.concatenate(nums), np.concatenate(dens))
        np.save(out_path, np.array([lp, se]))
    dist.barrier()
    dist.destroy_process_group()


def test_two_rank_shard_and_reduce_equals_unsplit(tmp_path):
    out = str(tmp_path / "res.npy")
    mp.spawn(_worker, args=(2, _free_port(), out), nprocs=2, join=True)
    lp, se = np.load(out)
    prob, s, u, nbr = _problem()
    ref = O.log_cdf(s, nbr, prob.m, prob.cov, u, prob.N, prob.S, prob.seed)
    assert lp == ref[0] and se == ref[1]
