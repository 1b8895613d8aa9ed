"""The multi-rank (replicas) path of bench.py on CPU: two gloo ranks, the whole-job aggregation
(slowest rank's time, all ranks' units) and per-rank inputs that differ."""
import os
import socket
import sys

import pytest

torch = pytest.importorskip("torch")
import torch.distributed as dist  # noqa: E402
import torch.multiprocessing as mp  # noqa: E402

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank_main(rank, world, port, out):
    sys.path.insert(0, ROOT)
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    import bench
    ms, units = bench.aggregate_ranks(10.0 + rank, 100 * (rank + 1), dist, device="cpu")
    out[rank] = (ms, units)
    dist.barrier()
    dist.destroy_process_group()


def test_two_gloo_ranks_aggregate_to_the_whole_job():
    world = 2
    port = _free_port()
    with mp.Manager() as mgr:
        out = mgr.dict()
        mp.spawn(_rank_main, args=(world, port, out), nprocs=world, join=True)
        res = dict(out)
    assert res[0] == res[1] == (11.0, 300)


def test_single_rank_aggregation_is_identity():
    sys.path.insert(0, ROOT)
    import bench
    assert bench.aggregate_ranks(12.5, 7, None) == (12.5, 7)


def test_replicas_draw_their_own_inputs():
    """Each rank's systems come from its own seeds (batched) and its own Philox stream (sys_id)."""
    sys.path.insert(0, ROOT)
    import bench

    class _Args:
        workload = "batched64"
    wl = bench.make_workload(_Args())
    assert isinstance(wl, bench.Batched)
    seeds = {r: [wl.system_seed(r, i) for i in range(wl.nsys)] for r in range(4)}
    flat = [s for v in seeds.values() for s in v]
    assert len(flat) == len(set(flat))
