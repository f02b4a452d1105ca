"""DM-trial sharding across ranks, one GPU per rank (weak scaling).

Every DM trial is an independent search of its own dedispersed series
(Section 2: the acceleration search runs once per DM trial), so a survey's
trial list is cut into contiguous blocks, one per rank, and each rank
searches its block with its own plan.  Series are tagged with their global
DM-trial index as `trial_id`, so the per-rank candidate lists concatenate
into the global (trial, harmonic stage, z, r) order.  No step of the search
exchanges data between ranks: the only collectives here are the timing
reduction and the optional gather of candidate lists on one rank, both on
the host side of a finished search.
"""
from __future__ import annotations

import numpy as np

CANDIDATE_ORDER = ("trial_id", "harm", "iz", "ir")


def trial_block(n_trials: int, rank: int, world: int) -> tuple[int, int]:
    """[start, stop) of the DM trials rank `rank` of `world` searches.

    Blocks are contiguous, cover [0, n_trials) exactly once and differ in
    size by at most one (the first n_trials % world ranks take one more).
    """
    if world < 1 or not 0 <= rank < world or n_trials < 0:
        raise ValueError(f"bad shard request: n_trials={n_trials}, rank={rank}, world={world}")
    q, r = divmod(n_trials, world)
    start = rank * q + min(rank, r)
    return start, start + q + (1 if rank < r else 0)


def max_over_ranks(value: float, dist=None, device=None) -> float:
    """The maximum of `value` over all ranks (the value itself without a
    process group).  `device` is where the reduction tensor lives (a CUDA
    device for NCCL, None for gloo)."""
    if dist is None or not dist.is_initialized() or dist.get_world_size() == 1:
        return float(value)
    import torch
    t = torch.tensor([float(value)], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def weak_scaling_throughput(units_per_rank: list[int] | int, world: int, ms_max: float) -> float:
    """Units per second of the whole job: every unit all ranks processed over
    the slowest rank's time."""
    total = units_per_rank * world if isinstance(units_per_rank, int) else sum(units_per_rank)
    if ms_max <= 0:
        raise ValueError("elapsed time must be positive")
    return total / (ms_max / 1000.0)


def merge_candidates(lists, order=CANDIDATE_ORDER) -> np.ndarray:
    """Concatenate per-rank candidate arrays (structured, same dtype) and
    sort them by `order`; with globally numbered trials this is the order a
    single search over all trials returns."""
    lists = [np.asarray(a) for a in lists if a is not None]
    if not lists:
        return np.zeros(0)
    allc = np.concatenate(lists)
    return np.sort(allc, order=list(order), kind="stable")


def gather_candidates(cands: np.ndarray, dist=None, dst: int = 0, order=CANDIDATE_ORDER):
    """Merged candidate list of all ranks on rank `dst` (None elsewhere).

    Uses an object gather over the process group after the search, so it
    works with gloo and NCCL alike; without a process group it sorts the
    local list.
    """
    if dist is None or not dist.is_initialized() or dist.get_world_size() == 1:
        return merge_candidates([cands], order)
    world = dist.get_world_size()
    rank = dist.get_rank()
    got = [None] * world if rank == dst else None
    dist.gather_object(cands, got, dst=dst)
    return merge_candidates(got, order) if rank == dst else None
