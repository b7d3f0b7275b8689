"""Multi-rank work split (no GPU): partition properties, and the two-rank path
over gloo -- each rank takes its share of a ragged batch and the timing is
reduced with a maximum, as the benchmark does under torchrun."""
import os
import socket

import numpy as np
import pytest

import workloads as W
from paper_2504_07264_gb300 import sharding as SH


@pytest.mark.parametrize("batch,world", [(0, 1), (7, 1), (7, 2), (65536, 4), (5, 8)])
def test_uniform_blocks_cover_exactly(batch, world):
    seen = []
    counts = []
    for r in range(world):
        s, c = SH.shard_uniform(batch, r, world)
        seen += list(range(s, s + c))
        counts.append(c)
    assert seen == list(range(batch))
    assert max(counts) - min(counts) <= 1


def test_ragged_partition_and_balance():
    lengths, _ = W.ragged_lengths(10000, 3, 16, 4)
    for world in (1, 2, 4, 8):
        parts = SH.shard_ragged(lengths, world)
        allidx = np.sort(np.concatenate(parts))
        assert np.array_equal(allidx, np.arange(lengths.size))
        loads = [sum(SH.transform_cost(int(lengths[t])) for t in p) for p in parts]
        biggest = max(SH.transform_cost(int(n)) for n in lengths)
        assert max(loads) - min(loads) <= biggest


def test_bad_requests():
    with pytest.raises(ValueError):
        SH.shard_uniform(4, 2, 2)
    with pytest.raises(ValueError):
        SH.shard_ragged([8, 16], 0)
    assert SH.max_over_ranks(3.5) == 3.5


def _free_port() -> int:
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank_main(rank, world, port, out_dir):
    import torch.distributed as dist
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        lengths, _ = W.ragged_lengths(500, 3, 16, 4)
        mine = SH.shard_ragged(lengths, world)[rank]
        # every rank derives the same split on its own: check against the others
        import torch
        gathered = [None] * world
        dist.all_gather_object(gathered, mine.tolist())
        fake_ms = 1.0 + rank                       # this rank's step time
        worst = SH.max_over_ranks(fake_ms, dist)
        points = float(lengths[mine].sum())
        total = torch.tensor([points], dtype=torch.float64)
        dist.all_reduce(total)
        np.save(os.path.join(out_dir, f"rank{rank}.npy"),
                np.array([worst, total.item()] + [len(g) for g in gathered], dtype=np.float64))
        allidx = sorted(i for g in gathered for i in g)
        assert allidx == list(range(lengths.size))
    finally:
        dist.destroy_process_group()


def test_two_ranks_over_gloo(tmp_path):
    import torch.multiprocessing as mp
    world = 2
    mp.spawn(_rank_main, args=(world, _free_port(), str(tmp_path)), nprocs=world, join=True)
    lengths, _ = W.ragged_lengths(500, 3, 16, 4)
    for r in range(world):
        res = np.load(tmp_path / f"rank{r}.npy")
        assert res[0] == 2.0                     # max over ranks of 1.0 and 2.0
        assert res[1] == float(lengths.sum())    # the shares add up to the whole batch
