"""The N > 1 path on CPU: DM-trial shards over two gloo ranks.

Each rank searches its contiguous block of DM trials (here with the FP64
oracle standing in for a rank's GPU plan; the split, the trial numbering,
the max-over-ranks timing and the candidate gather are the host logic
bench.py and a multi-GPU survey run), and rank 0's merged candidate list
must equal the list of one search over all trials.
"""
import json
import os
import socket
from datetime import timedelta

import numpy as np
import pytest

import oracle as O
import synthetic as S
from paper_2211_13517_gb300 import shard

N, ZMAX, ZSTEP, H = 1 << 13, 8.0, 2.0, 4
ORDER = ("trial", "harm", "iz", "ir")


def _series(i):
    return S.sinusoid_series(n=N, seed=70 + i, r0=300.3 + 211 * i, z0=4.0 - 2 * i, amp=0.5)


def _search(i):
    return O.search(_series(i), ZMAX, ZSTEP, H, trial=i)["candidates"]


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _worker(rank, world, port, n_trials, out_dir, fail_rank):
    import torch.distributed as dist
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world, timeout=timedelta(seconds=30))
    try:
        if rank == fail_rank:
            raise RuntimeError("planted failure before the gather")
        start, stop = shard.trial_block(n_trials, rank, world)
        local = [_search(i) for i in range(start, stop)]
        local = np.concatenate(local) if local else np.zeros(0, dtype=O.CAND_DTYPE)
        merged = shard.gather_candidates(local, dist, dst=0, order=ORDER)
        ms = shard.max_over_ranks(100.0 + 7 * rank, dist)
        sizes = [b - a for a, b in (shard.trial_block(n_trials, r, world) for r in range(world))]
        value = shard.weak_scaling_throughput(sizes, world, ms)
        if rank == 0:
            np.save(os.path.join(out_dir, "merged.npy"), merged)
            with open(os.path.join(out_dir, "rank0.json"), "w") as f:
                json.dump({"ms": ms, "value": value, "block": [start, stop]}, f)
        else:
            assert merged is None
    finally:
        dist.destroy_process_group()


@pytest.mark.parametrize("n, world", [(0, 1), (1, 2), (5, 2), (7, 3), (256, 8), (1000, 7)])
def test_trial_blocks_partition_the_trials(n, world):
    blocks = [shard.trial_block(n, r, world) for r in range(world)]
    assert blocks[0][0] == 0 and blocks[-1][1] == n
    assert all(a[1] == b[0] for a, b in zip(blocks, blocks[1:]))
    sizes = [b - a for a, b in blocks]
    assert max(sizes) - min(sizes) <= 1 and sum(sizes) == n


def test_trial_block_rejects_bad_requests():
    for args in ((4, 2, 2), (4, -1, 2), (4, 0, 0), (-1, 0, 1)):
        with pytest.raises(ValueError):
            shard.trial_block(*args)


def test_single_process_helpers():
    assert shard.max_over_ranks(3.5) == 3.5
    assert shard.weak_scaling_throughput(10, 4, 2000.0) == 20.0
    assert shard.weak_scaling_throughput([3, 2], 2, 500.0) == 10.0
    a = np.array([(2, 1, 3, 4), (1, 2, 0, 0), (1, 1, 5, 9)],
                 dtype=[("trial_id", "u4"), ("harm", "u2"), ("iz", "u2"), ("ir", "u4")])
    m = shard.merge_candidates([a[:1], a[1:]])
    assert m.tolist() == sorted(a.tolist())


def test_two_gloo_ranks_reproduce_the_single_search(tmp_path):
    import torch.multiprocessing as mp
    n_trials = 5                                    # uneven: blocks of 3 and 2
    mp.spawn(_worker, args=(2, _free_port(), n_trials, str(tmp_path), -1), nprocs=2, join=True)
    merged = np.load(tmp_path / "merged.npy")
    want = np.sort(np.concatenate([_search(i) for i in range(n_trials)]), order=list(ORDER))
    assert len(want) > 0 and set(np.unique(want["trial"])) == set(range(n_trials))
    assert merged.dtype == want.dtype and merged.tolist() == want.tolist()
    r0 = json.loads((tmp_path / "rank0.json").read_text())
    assert r0["ms"] == 107.0                          # max over ranks, not rank 0's own
    assert r0["value"] == pytest.approx(n_trials / 0.107)
    assert r0["block"] == [0, 3]


def test_a_failing_rank_is_reported_not_hung(tmp_path):
    """A rank that raises before the gather: the other rank's collective ends
    with an error within the process-group timeout, and spawn reports it."""
    import torch.multiprocessing as mp
    with pytest.raises(Exception):
        mp.spawn(_worker, args=(2, _free_port(), 2, str(tmp_path), 1), nprocs=2, join=True)
    assert not (tmp_path / "merged.npy").exists()
