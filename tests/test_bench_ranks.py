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
    with mp.get_context("spawn").Manager() as mgr:
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


def test_clock_summary_reads_throttle_reasons():
    """The clocks object of the bench line: median SM clock under load, the maximum clock, and the
    throttle reasons seen Active in any sample (nvidia-smi csv,noheader,nounits rows)."""
    sys.path.insert(0, ROOT)
    import bench
    clk = bench.ClockSampler(0)
    na = "Not Active"
    clk.lines = [f"0, 2070, 2070, 812.3, 0x0000000000000000, {na}, {na}, {na}, {na}",
                 f"0, 1980, 2070, 1390.0, 0x0000000000000004, {na}, {na}, {na}, Active",
                 f"0, 2055, 2070, 1100.0, 0x0000000000000000, {na}, {na}, {na}, {na}",
                 "garbage line", "0, [N/A], 2070, 0, 0, a, b, c, d"]
    s = clk.summary()
    assert s == {"sm_mhz": 2055.0, "sm_max_mhz": 2070.0, "reasons": ["sw_power_cap"], "samples": 3}
    clk.lines.append(f"0, 1200, 2070, 1400.0, 0x0000000000000008, Active, {na}, Active, {na}")
    assert clk.summary()["reasons"] == ["hw_slowdown", "sw_power_cap", "sw_thermal_slowdown"]
    assert bench.ClockSampler(0).summary() == {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["unsampled"],
                                               "samples": 0}
