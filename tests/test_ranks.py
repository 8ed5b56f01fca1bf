"""The multi-GPU host logic on CPU (no GPU): the batch partition across ranks
and, with two gloo processes on 127.0.0.1, the barrier, the max over ranks and
the agreement of every rank on its share of a batch."""
import os
import socket

import pytest
import torch.multiprocessing as mp

from paper_1307_7820_b300 import ranks, synth


def test_partition_covers_every_sequence_once_and_balances():
    lens = synth.log_uniform_lengths(4096, 64, 3000, 17)
    for world in (1, 2, 3, 8):
        parts = ranks.partition_lpt(lens, world)
        assert len(parts) == world
        flat = sorted(k for p in parts for k in p)
        assert flat == list(range(len(lens)))
        work = [sum(ranks.fold_work(int(lens[k])) for k in p) for p in parts]
        # longest-processing-time first: no rank exceeds the mean by more than the largest item
        assert max(work) - sum(work) / world <= max(ranks.fold_work(int(n)) for n in lens)
    assert ranks.partition_lpt([5, 5, 5, 5], 2) == [[0, 2], [1, 3]]
    assert ranks.partition_lpt([], 3) == [[], [], []]
    with pytest.raises(ValueError):
        ranks.partition_lpt([1], 0)


def _worker(rank, world, port, out_dir):
    os.environ.update({"MASTER_ADDR": "127.0.0.1", "MASTER_PORT": str(port), "RANK": str(rank),
                       "WORLD_SIZE": str(world), "LOCAL_RANK": str(rank)})
    r = ranks.Ranks(backend="gloo", device="cpu")
    assert r.rank == rank and r.world == world
    r.barrier()
    assert r.max(10.0 * rank + 1.0) == 10.0 * (world - 1) + 1.0
    lens = synth.log_uniform_lengths(300, 64, 3000, 5)
    mine = ranks.partition_lpt(lens, world)[rank]
    import torch.distributed as dist
    got = [None] * world
    dist.all_gather_object(got, mine)
    flat = sorted(k for p in got for k in p)
    assert flat == list(range(len(lens)))
    with open(os.path.join(out_dir, f"rank{rank}.ok"), "w") as f:
        f.write(str(len(mine)))
    r.close()


def test_gloo_two_ranks(tmp_path):
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        port = s.getsockname()[1]
    mp.spawn(_worker, args=(2, port, str(tmp_path)), nprocs=2, join=True)
    assert sorted(os.listdir(tmp_path)) == ["rank0.ok", "rank1.ok"]
