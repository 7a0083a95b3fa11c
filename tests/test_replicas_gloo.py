"""Multi-process replica path of bench.py on CPU ranks (gloo, world size 2).

Each rank evaluates its own designs (no data exchange between ranks); the job's step time is
the slowest rank's and the throughput counts every rank's k-points.  Checked here without a
GPU: the ranks get disjoint, reproducible designs, and the cross-rank reduction gives the
maximum step time and the whole-job throughput on every rank.
"""
import os
import socket
import sys

import numpy as np
import pytest

torch = pytest.importorskip("torch")
ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _free_port() -> int:
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _worker(rank: int, world: int, port: int, out_dir: str) -> None:
    sys.path.insert(0, ROOT)
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    import torch.distributed as dist
    import bench
    dist.init_process_group("gloo", rank=rank, world_size=world)
    ds = bench.designs(2, rank, workload="sc16_M2_grf")
    seeds = [d.seed for d in ds]
    gathered = [None] * world
    dist.all_gather_object(gathered, seeds)
    local_ms = [120.0, 180.0][rank]
    ms = bench.replica_max(local_ms, world, torch.device("cpu"))
    value = bench.replica_throughput(ms, ds[0].nk, world)
    np.save(os.path.join(out_dir, f"rank{rank}.npy"),
            np.array([ms, value] + [s for g in gathered for s in g], dtype=np.float64))
    dist.barrier()
    dist.destroy_process_group()


def test_two_gloo_ranks(tmp_path):
    import torch.multiprocessing as mp
    world = 2
    mp.spawn(_worker, args=(world, _free_port(), str(tmp_path)), nprocs=world, join=True)
    r0 = np.load(tmp_path / "rank0.npy")
    r1 = np.load(tmp_path / "rank1.npy")
    np.testing.assert_array_equal(r0, r1)  # every rank sees the same reduced numbers
    ms, value = r0[0], r0[1]
    assert ms == 180.0                       # the slowest rank
    sys.path.insert(0, ROOT)
    import workloads as wl
    nk = wl.sc16_grf().nk
    assert value == pytest.approx(world * nk / 0.180)
    seeds = r0[2:].astype(int)
    assert len(set(seeds.tolist())) == len(seeds)  # disjoint designs across ranks
    assert seeds.tolist() == [wl.sc16_grf(design=r * 1000 + i).seed for r in range(world) for i in range(2)]
