"""Host logic of the multi-rank bench (independent replicas, one per rank):
two gloo ranks on the CPU reduce their timings and work the way the GPU
ranks do over NCCL."""
import json
import os
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _rank_main(rank, world, port, out_dir):
    import torch.distributed as dist
    sys.path.insert(0, ROOT)
    import bench
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    elapsed = [2.5, 3.25][rank]
    work = [1.0e12, 3.0e12][rank]
    e, k = bench.aggregate_ranks(elapsed, work, "cpu")
    with open(os.path.join(out_dir, f"r{rank}.json"), "w") as f:
        json.dump({"elapsed": e, "interactions": k}, f)
    dist.barrier()
    dist.destroy_process_group()


def test_two_gloo_ranks_take_max_time_and_summed_work(tmp_path):
    torch = pytest.importorskip("torch")
    import socket
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        port = s.getsockname()[1]
    torch.multiprocessing.spawn(_rank_main, args=(2, port, str(tmp_path)), nprocs=2, join=True)
    for r in range(2):
        d = json.loads((tmp_path / f"r{r}.json").read_text())
        assert d == {"elapsed": 3.25, "interactions": 4.0e12}


def test_single_process_returns_local_figures():
    sys.path.insert(0, ROOT)
    import bench
    assert bench.aggregate_ranks(1.5, 7.0) == (1.5, 7.0)
