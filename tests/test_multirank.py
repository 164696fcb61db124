"""Host-side multi-rank path of bench.py on CPU (gloo, world size 2).

The path does not shard a cluster: every rank runs an independent lattice
(seed + rank) and the only collective is the host-side reduction of the
timing (max over ranks) and of the flipped-spin count (sum)."""
import os
import socket

import pytest

torch = pytest.importorskip("torch")
import torch.distributed as dist  # noqa: E402
import torch.multiprocessing as mp  # noqa: E402


def _free_port():
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    port = s.getsockname()[1]
    s.close()
    return port


def _worker(rank, world, port, out):
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    import sys
    sys.path.insert(0, os.path.dirname(os.path.dirname(os.path.abspath(__file__))))
    import bench
    dist.init_process_group("gloo", rank=rank, world_size=world)
    ms = [12.5, 20.0][rank]
    flips = [1000, 2345][rank]
    t, f = bench.aggregate_ranks(ms, flips, "cpu")
    out[rank] = (t, f, bench.rank_seed(2, rank))
    dist.barrier()
    dist.destroy_process_group()


def test_two_ranks_reduce_time_and_flips():
    port = _free_port()
    with mp.Manager() as m:
        out = m.dict()
        mp.start_processes(_worker, args=(2, port, out), nprocs=2, join=True,
                           start_method="spawn")
        res = dict(out)
    for rank in (0, 1):
        t, f, seed = res[rank]
        assert t == 20.0 and f == 3345.0
        assert seed == 2 + rank
