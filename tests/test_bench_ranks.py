"""bench.py's multi-rank totals on two gloo ranks (CPU only).

With N > 1 every rank runs its own replica of the contact stage; the whole-job line takes the
slowest rank's timed seconds and the pairs and candidates of all ranks.  The aggregation is
run here by two CPU processes over gloo, rendezvous on 127.0.0.1.
"""
import json
import os
import socket

import pytest

torch = pytest.importorskip("torch")
mp = pytest.importorskip("torch.multiprocessing")


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank(rank, world, port, out_dir):
    import torch.distributed as dist

    import bench
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        # rank r: 1.5 + r seconds, 100 (r + 1) pairs, 10 (r + 1) candidates
        got = bench.across_ranks(1.5 + rank, 100.0 * (rank + 1), 10.0 * (rank + 1), world, torch.device("cpu"))
        with open(os.path.join(out_dir, f"rank{rank}.json"), "w") as f:
            json.dump(got, f)
        dist.barrier()
    finally:
        dist.destroy_process_group()


def test_two_gloo_ranks_take_the_slowest_time_and_all_pairs(tmp_path):
    world = 2
    mp.spawn(_rank, args=(world, _free_port(), str(tmp_path)), nprocs=world, join=True)
    for r in range(world):
        with open(tmp_path / f"rank{r}.json") as f:
            s, p, c = json.load(f)
        assert s == 2.5 and p == 300.0 and c == 30.0


def test_one_rank_passes_its_values_through():
    import bench
    assert bench.across_ranks(1.25, 7.0, 3.0, 1, None) == (1.25, 7.0, 3.0)
