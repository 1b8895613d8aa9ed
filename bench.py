#!/usr/bin/env python
"""Benchmark of the Kaczmarz++ / CD++ block-step library on one GB300 (or N, one rank per GPU).

A step is one complete solve through the C ABI: the factor phase (kpp_factor_blocks: memoised
per-block Cholesky factors) and the iteration (cdpp_solve / kpp_solve) to |Ax-b|/|b| <= 1e-8,
confirmed by the FP64 true residual.  Inputs are resident in HBM before the timed region; L2 is
flushed (512 MiB write) between steps, and the flush is outside each step's event pair.

Workloads (synthetic, seeded; see paper_2501_11673_gb300/workloads.py):
  cdpp4096 (default): CD++ FP64 on SPD n=4096, 50 outliers 1e2..1e4 over U[1,10], s=64, lambda=1e-4
  kpp2000:            K++ FP64 on 2000x200 LS, 10 outliers 1e2..1e3 over U[1,2], s=20, lambda=1e-3

Prints one JSON line (rank 0).  `--impl reference` times the FP64 CPU oracle instead (rank 0 only).
"""
from __future__ import annotations

import argparse
import json
import os
import statistics
import subprocess
import sys
import threading
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

from paper_2501_11673_gb300 import workloads as W  # noqa: E402

METRIC = "time-to-1e-8 rel. residual & block-iters/s"


def _peaks():
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as f:
            return json.load(f)
    except Exception:
        return {}


def workload(name: str):
    if name == "cdpp4096":
        sy = W.cdpp_fp64_spd()
        desc = ("CD++ FP64, dense SPD n=4096 = U diag(sigma) U^T (U Haar; 50 outliers log-spaced 1e2..1e4 + "
                "4046 ~U[1,10]), b~N(0,I), s=64 contiguous, lambda=1e-4, tol=1e-8, x0=0")
        return sy, True, desc
    if name == "kpp2000":
        sy = W.kpp_fp64_2000x200()
        desc = ("K++ FP64, 2000x200 consistent LS A=Z D V^T (10 outliers 1e2..1e3 + 190 ~U[1,2]), s=20, "
                "lambda=1e-3, tol=1e-8, x0=0")
        return sy, False, desc
    raise SystemExit(f"unknown workload {name}")


def per_iter_cost(sy, cd: bool):
    """Algorithmic FP64 flops and HBM bytes of one block iteration (k = 1)."""
    m, n = sy.A.shape
    s = sy.s
    if cd:
        flops = 2 * s * n + 2 * s * s + 10 * n + 2 * s
        byts = 8 * (s * n + s * s + 8 * n + s)
    else:
        flops = 4 * s * n + 2 * s * s + 6 * n + 2 * s
        byts = 8 * (s * n + s * s + 4 * n + 2 * s)
    return flops, byts


class ClockSampler:
    """nvidia-smi samples of SM clock and throttle reasons during the timed region."""

    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_index: int):
        self.gpu = gpu_index
        self.proc = None
        self.lines = []

    def __enter__(self):
        try:
            self.proc = subprocess.Popen(["nvidia-smi", "-i", str(self.gpu), f"--query-gpu={self.FIELDS}",
                                          "--format=csv,noheader,nounits", "-lms", "100"],
                                         stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
            self.t = threading.Thread(target=self._read, daemon=True)
            self.t.start()
        except Exception:
            self.proc = None
        return self

    def _read(self):
        for line in self.proc.stdout:
            self.lines.append(line.strip())

    def __exit__(self, *a):
        if self.proc:
            time.sleep(0.25)
            self.proc.terminate()
            try:
                self.proc.wait(timeout=5)
            except Exception:
                self.proc.kill()

    def summary(self):
        sm, mx, reasons = [], None, set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for ln in self.lines:
            p = [v.strip() for v in ln.split(",")]
            if len(p) < 9:
                continue
            try:
                sm.append(float(p[1]))
                mx = float(p[2])
            except ValueError:
                continue
            for nm, v in zip(names, p[5:9]):
                if v.lower().startswith("active"):
                    reasons.add(nm)
        if not sm:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["unsampled"], "samples": 0}
        return {"sm_mhz": statistics.median(sm), "sm_max_mhz": mx, "reasons": sorted(reasons), "samples": len(sm)}


def run_reference(args, rank: int):
    """The FP64 CPU oracle on the host cores, each step a bounded sample of the same workload."""
    if rank != 0:
        return
    import oracle
    sy, cd, desc = workload(args.workload)
    n = sy.A.shape[1]
    L = oracle.cdpp_factor(sy.A, sy.s, sy.lam) if cd else oracle.kpp_factor(sy.A, sy.s, sy.lam)
    sample_iters = args.ref_iters
    times = []
    for i in range(args.warmup + args.steps):
        t0 = time.perf_counter()
        r = oracle.run(sy.A, sy.b, L, sy.s, cd=cd, lam=sy.lam, tol=0.0, max_iters=sample_iters, seed=1 if cd else 0)
        dt = time.perf_counter() - t0
        if i >= args.warmup:
            times.append(dt)
        assert r.iters == sample_iters
    v = sample_iters / statistics.mean(times)
    sample = f"{sample_iters} oracle block iterations of the workload per step (factor phase excluded)"
    line = {"impl": "reference", "metric": METRIC, "value": v, "unit": "block-iters/s", "n_gpus": args.gpus,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": 1e3 * statistics.mean(times),
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
            "config": {"workload": desc},
            "cpu_baseline": {"value": v, "unit": "block-iters/s", "cores": 1, "kind": "oracle", "sample": sample},
            "e2e": {"value": v, "unit": "block-iters/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)


def cpu_baseline(sy, cd: bool, budget_s: float):
    """The oracle as it stands, single-threaded, on a bounded sample (iterations, not the whole solve)."""
    import oracle
    L = oracle.cdpp_factor(sy.A, sy.s, sy.lam) if cd else oracle.kpp_factor(sy.A, sy.s, sy.lam)
    it = 256
    while True:
        t0 = time.perf_counter()
        oracle.run(sy.A, sy.b, L, sy.s, cd=cd, lam=sy.lam, tol=0.0, max_iters=it, seed=1 if cd else 0)
        dt = time.perf_counter() - t0
        if dt > budget_s / 4 or it >= (1 << 22):
            break
        it *= 4
    return {"value": it / dt, "unit": "block-iters/s", "cores": 1, "kind": "oracle",
            "sample": f"{it} block iterations of the same workload, FP64 C oracle, one host thread ({dt:.1f} s)"}


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=5)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--workload", default="cdpp4096", choices=["cdpp4096", "kpp2000"])
    ap.add_argument("--ref-iters", type=int, default=4096)
    ap.add_argument("--cpu-budget", type=float, default=20.0)
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-e2e", action="store_true")
    args = ap.parse_args()

    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))

    if args.impl == "reference":
        run_reference(args, rank)
        return

    import torch
    torch.cuda.set_device(local)
    dist = None
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl", device_id=torch.device("cuda", local))
    from paper_2501_11673_gb300 import build as kbuild
    from paper_2501_11673_gb300 import kpp
    if rank == 0:
        kbuild.build()
    if dist:
        dist.barrier()
    kpp.load()

    sy, cd, desc = workload(args.workload)
    m, n = sy.A.shape
    stream = torch.cuda.current_stream()
    Ad = torch.as_tensor(sy.A, device="cuda")
    bd = torch.as_tensor(sy.b, device="cuda")
    x = torch.zeros(n, dtype=torch.float64, device="cuda")
    P = kpp.Partition(m, sy.s)
    prm = kpp.params(lam=sy.lam, tol=sy.tol, seed=1 if cd else 0, sys_id=rank)
    flush = torch.empty(512 << 20, dtype=torch.uint8, device="cuda")
    solve = kpp.cdpp_solve if cd else kpp.kpp_solve

    def step():
        x.zero_()
        F = kpp.Factors(Ad, P, sy.lam, 1 if cd else 0)
        rep = solve(Ad, bd, x, P, F, prm)
        del F
        return rep

    for _ in range(args.warmup):
        step()
    torch.cuda.synchronize()
    step_ms, kern_ms, iters, reps = [], [], [], []
    with ClockSampler(local) as clk:
        if dist:
            dist.barrier()
        torch.cuda.synchronize()
        for _ in range(args.steps):
            flush.zero_()
            e0 = torch.cuda.Event(enable_timing=True)
            e1 = torch.cuda.Event(enable_timing=True)
            e0.record(stream)
            rep = step()
            e1.record(stream)
            e1.synchronize()
            step_ms.append(e0.elapsed_time(e1))
            kern_ms.append(rep.device_ms)
            iters.append(rep.iters)
            reps.append(rep)
        torch.cuda.synchronize()
        if dist:
            dist.barrier()
    total_ms = sum(step_ms)
    total_iters = sum(iters)
    if dist:
        t = torch.tensor([total_ms], device="cuda", dtype=torch.float64)
        dist.all_reduce(t, op=dist.ReduceOp.MAX)
        total_ms = float(t.item())
        it = torch.tensor([total_iters], device="cuda", dtype=torch.float64)
        dist.all_reduce(it, op=dist.ReduceOp.SUM)
        total_iters = int(it.item())
    value = total_iters / (total_ms / 1e3)
    assert all(r.status == kpp.OK and r.rel_res_true <= sy.tol for r in reps), [r.as_dict() for r in reps]

    flops, byts = per_iter_cost(sy, cd)
    peaks = _peaks()
    mean_iters = statistics.mean(iters)
    kms = statistics.mean(kern_ms)
    fp64_peak = 152 * 2 * 2 * peaks.get("sm_max_mhz", 2070.0) * 1e6 / 1e9  # GFLOP/s: 2 FP64 FMA/clk/SM
    ach_flops = mean_iters * flops / (kms / 1e3) / 1e9
    ach_bytes = mean_iters * byts / (kms / 1e3) / 1e9
    hbm = peaks.get("hbm_gbs", 6800.0)
    roof = {"kernel": "cd3_kernel" if cd else "solve2_kernel", "bound": "alu", "achieved": ach_flops, "peak": fp64_peak, "unit": "GFLOP/s",
            "frac": ach_flops / fp64_peak, "traffic": None,
            "per_iter": {"flops": flops, "bytes": byts},
            "hbm_view": {"achieved": ach_bytes, "peak": hbm, "unit": "GB/s", "frac": ach_bytes / hbm,
                         "peak_source": "MEASURED_PEAKS.json hbm_gbs (measured)"},
            "peak_source": "FP64 ALU: 152 SMs x 2 FMA/clk x 2 flop x sm_max_mhz (derived)"}

    line = {"metric": METRIC, "value": value, "unit": "block-iters/s", "n_gpus": world, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": total_ms / args.steps, "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
            "config": {"workload": desc, "parallelism": f"replicas x{world}",
                       "l2": "flushed between steps (512 MiB write, outside the step events)",
                       "step": "factor phase + solve to 1e-8 + FP64 residual confirmation"},
            "time_to_tol_ms": statistics.mean(step_ms), "iters_to_tol": mean_iters,
            "solve_kernel_ms": kms, "rel_res_true": reps[-1].rel_res_true,
            "gpu_launches": 5 * args.steps, "roofline": roof, "clocks": clk.summary()}

    if rank == 0 and not args.no_e2e:
        # end to end through the host-buffer entry point: copies in, factor, solve, copy back
        A_h = np.ascontiguousarray(sy.A)
        b_h = sy.b.copy()
        ets = []
        for i in range(2):
            x_h = np.zeros(n)
            t0 = time.perf_counter()
            rep = kpp.solve_host(A_h, b_h, x_h, sy.s, 1 if cd else 0, prm)
            ets.append(time.perf_counter() - t0)
            assert rep.status == kpp.OK
        line["e2e"] = {"value": rep.iters / ets[-1], "unit": "block-iters/s",
                       "h2d_bytes_per_step": A_h.nbytes + b_h.nbytes + x_h.nbytes,
                       "d2h_bytes_per_step": x_h.nbytes, "time_to_tol_ms": 1e3 * ets[-1],
                       "note": "host (pageable) buffers through kpp_solve_host"}
    if rank == 0 and not args.no_cpu_baseline:
        line["cpu_baseline"] = cpu_baseline(sy, cd, args.cpu_budget)
    if rank == 0:
        print(json.dumps(line), flush=True)
    if dist:
        dist.destroy_process_group()


if __name__ == "__main__":
    main()
