"""The multi-rank path of bench.py on CPU: two gloo ranks.

Ranks solve independent cells (weak scaling): each rank's cell seed differs,
and the only collectives are the reductions of the timed region (maximum over
ranks) and of the pair counts (sum), from which the whole-job throughput is
formed.  The GPU work itself is not needed to check this logic.
"""
import json
import os
import socket
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank_main(rank, world, port, out_dir):
    sys.path.insert(0, ROOT)
    import torch.distributed as dist

    import bench
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    elapsed = 100.0 + 50.0 * rank           # rank 1 is the slow one
    n_pairs = 1000 + 7 * rank               # independent cells have different pair counts
    el, pairs = bench.reduce_over_ranks(elapsed, n_pairs, dist, "cpu")
    dist.barrier()
    with open(os.path.join(out_dir, f"r{rank}.json"), "w") as f:
        json.dump({"elapsed": el, "pairs": pairs, "seed": bench.rank_seed(rank)}, f)
    dist.destroy_process_group()


def test_two_gloo_ranks_reduce_time_and_pairs(tmp_path):
    mp = pytest.importorskip("torch.multiprocessing")
    port = _free_port()
    mp.spawn(_rank_main, args=(2, port, str(tmp_path)), nprocs=2, join=True)
    r = [json.load(open(tmp_path / f"r{k}.json")) for k in range(2)]
    for x in r:
        assert x["elapsed"] == 150.0          # the slowest rank's timed region
        assert x["pairs"] == 2007              # all ranks' pairs
    assert r[0]["seed"] != r[1]["seed"]
    sys.path.insert(0, ROOT)
    import bench
    import paper_2011_07209_gb300.synth as synth
    # rank 0 solves exactly the single-GPU benchmark cell
    assert bench.rank_seed(0) == synth.SEED_BASE + 2


def test_single_rank_needs_no_collective():
    sys.path.insert(0, ROOT)
    import bench
    assert bench.reduce_over_ranks(12.5, 42, None, "cpu") == (12.5, 42)
