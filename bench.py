#!/usr/bin/env python
"""Benchmark of the Kaczmarz++ / CD++ block-step library on one GB300 (or N, one rank per GPU).

A step is one complete solve through the C ABI: the factor phase (memoised per-block factors,
kpp_factor_blocks) and the iteration to |Ax-b|/|b| <= 1e-8, confirmed by the FP64 true residual.
Inputs are resident in HBM before the timed region; L2 is flushed (512 MiB write) between steps,
outside each step's event pair.

Workloads (synthetic and seeded; recipes in paper_2501_11673_gb300/workloads.py):
  mixed262144 (default)  K++ on 262144x4096 LS stored BF16 (--storage f32 for FP32), 100 outliers 10..1000
                      over U[0.5,1], s=512, lambda=1e-3, FP32 iterations + FP64 refinement, b = A x*
                      (--noisy: b = A x* + 1e-6 N(0,I); the attained residual is reported, no tolerance);
                      after the timed steps the plain FP64 K++ path solves the same system once
  cdpp4096            CD++ FP64, dense SPD n=4096, 50 outliers 1e2..1e4 over U[1,10], s=64, lambda=1e-4
  kpp2000             K++ FP64, 2000x200 consistent LS, 10 outliers 1e2..1e3 over U[1,2], s=20, lambda=1e-3
  batched64           64 systems 2048x65536 FP32 (20 rows x100), 8 right-hand sides each, s=256,
                      lambda = 1e-3 median |a_i|^2, refinement; one autotuned plan replayed as a CUDA graph
  serving             1024 CD++ requests, Poisson arrivals (2 ms mean gap) over a catalog of 32 SPD matrices
                      (n log-uniform 512..8192, BF16 / FP32), k = 1..32, refinement, 120 GiB budget
  cdpp4096-f32 / -bf16  the cdpp4096 system stored FP32 / BF16 with FP64 refinement

Prints one JSON line (rank 0).  `--impl reference` times the FP64 CPU oracle on every host core on a
bounded sample of the same workload instead (rank 0 only, no GPU).
"""
from __future__ import annotations

import argparse
import json
import math
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
SERVING_METRIC = "solves/s + p99 latency"

# DRAM bytes (read + write) per launch of the dominant kernel, from one ncu capture of the kernel as
# built now, on the same workload (the ncu summaries under profiles/ give the commands).  An entry goes
# when its kernel changes; absent means not captured since (reported as null).
NCU_TRAFFIC_PER_LAUNCH = {
    # cd4_kernel, n = 4096 CD++ FP64, one launch = one solve of 23168 iterations
    # (profiles/cd4_kernel_cdpp4096.md: 7.1217e9 read + 0.0203e9 written)
    "cd4_kernel/cdpp4096": 7.142e9,
}


def _log(msg):
    print(f"[bench {time.strftime('%H:%M:%S')}] {msg}", file=sys.stderr, flush=True)


def _peaks():
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as f:
            return json.load(f)
    except Exception:
        return {}


# FP64 FMA lanes per clock per SM on this GPU, measured by a throughput probe (4+ warps issuing
# independent DFMA): a warp-wide FP64 instruction holds an SMSP's FP64 pipe for about 76 cycles.
FP64_LANES_MEASURED = 1.68
FP64_LANES_NOMINAL = 2.0


def fp64_peak_gflops(peaks, lanes=FP64_LANES_MEASURED):
    """FP64 FMA pipe: 152 SMs x lanes FMA/clk x 2 flop x the maximum SM clock."""
    return 152 * lanes * 2 * peaks.get("sm_max_mhz", 2070.0) * 1e6 / 1e9


FP64_PEAK_SOURCE = ("derived: 152 SMs x 1.68 FP64 FMA lanes/clk/SM (measured by a DFMA throughput probe on this "
                    "pool's GB300) x 2 flop x sm_max_mhz (MEASURED_PEAKS.json)")


def fp32_peak_gflops(peaks):
    """FP32 FMA pipe: 152 SMs x 128 FMA/clk x 2 flop x the maximum SM clock."""
    return 152 * 128 * 2 * peaks.get("sm_max_mhz", 2070.0) * 1e6 / 1e9


def fp64_peak_nominal(peaks):
    return {"peak": fp64_peak_gflops(peaks, FP64_LANES_NOMINAL),
            "source": "nominal: 152 SMs x 2 FP64 FMA/clk x 2 flop x sm_max_mhz"}


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


# ---------------------------------------------------------------------------------------------
# Oracle samples (cpu_baseline and the reference arm)
# ---------------------------------------------------------------------------------------------

def _oracle_iter_rate(A, b, L, s, cd, lam, seed, budget_s, it0=64):
    """Block iterations per second of the oracle as it stands (one host thread, no stop test), on a
    sample grown until it takes about a quarter of `budget_s`."""
    import oracle
    it = it0
    while True:
        t0 = time.perf_counter()
        oracle.run(A, b, L, s, cd=cd, lam=lam, tol=0.0, max_iters=it, seed=seed, confirm=False)
        dt = time.perf_counter() - t0
        if dt > budget_s / 4 or it >= (1 << 22):
            return it / dt, it, dt
        it *= 4


def _cpu_info():
    """Host cores this process may run on, and the CPU model (lscpu, else the platform's name)."""
    import platform
    cores = len(os.sched_getaffinity(0)) if hasattr(os, "sched_getaffinity") else (os.cpu_count() or 1)
    model = platform.processor() or platform.machine()
    try:
        out = subprocess.run(["lscpu"], capture_output=True, text=True, timeout=10).stdout
        for ln in out.splitlines():
            if ln.startswith("Model name:"):
                model = ln.split(":", 1)[1].strip()
                break
    except Exception:
        pass
    return cores, model


def _oracle_worker(paths, s, cd, lam, seed, sys_id, iters, barrier, q):
    """One all-cores oracle worker (spawned): maps the sample, waits for the others, times `iters`
    block iterations of its own Philox stream."""
    if ROOT not in sys.path:
        sys.path.insert(0, ROOT)
    import oracle
    A = np.load(paths[0], mmap_mode="r")
    b = np.load(paths[1])
    L = np.load(paths[2], mmap_mode="r")
    oracle.run(A, b, L, s, cd=cd, lam=lam, tol=0.0, max_iters=2, seed=seed, sys=sys_id, confirm=False)
    barrier.wait()
    t0 = time.perf_counter()
    oracle.run(A, b, L, s, cd=cd, lam=lam, tol=0.0, max_iters=iters, seed=seed, sys=sys_id, confirm=False)
    q.put(time.perf_counter() - t0)


def _oracle_rate_all_cores(A, b, L, s, cd, lam, seed, one_core_rate, budget_s):
    """Block iterations per second of the oracle as it stands on every host core: one single-threaded
    oracle process per core (spawned, so no process is forked from one that holds a CUDA context), each
    on its own Philox stream of the same sample, started together; value = all iterations / the slowest
    worker's time.  Returns (value, cores, cpu model, iterations per worker, slowest seconds)."""
    import multiprocessing as mp
    import shutil
    import tempfile
    cores, model = _cpu_info()
    iters = max(4, int(one_core_rate * budget_s / 2))
    tmp = tempfile.mkdtemp(prefix="kpp_oracle_sample_")
    try:
        paths = [os.path.join(tmp, nm) for nm in ("A.npy", "b.npy", "L.npy")]
        for pth, arr in zip(paths, (A, b, L)):
            np.save(pth, np.ascontiguousarray(arr, dtype=np.float64))
        ctx = mp.get_context("spawn")
        barrier = ctx.Barrier(cores)
        q = ctx.Queue()
        procs = [ctx.Process(target=_oracle_worker, args=(paths, s, cd, lam, seed, i, iters, barrier, q))
                 for i in range(cores)]
        for pr in procs:
            pr.start()
        times = [q.get(timeout=max(600.0, 20 * budget_s)) for _ in procs]
        for pr in procs:
            pr.join(timeout=60)
    finally:
        shutil.rmtree(tmp, ignore_errors=True)
    slow = max(times)
    return cores * iters / slow, cores, model, iters, slow


def _cpu_baseline_both(A, b, L, s, cd, lam, seed, budget_s, unit, what, it0=16):
    """The oracle on one host thread and on every host core (the line's value is the all-cores one)."""
    v1, it1, dt1 = _oracle_iter_rate(A, b, L, s, cd, lam, seed, budget_s, it0=it0)
    out = {"value": v1, "unit": unit, "cores": 1, "kind": "oracle",
           "sample": f"{it1} {what}, one host thread ({dt1:.1f} s; factor phase excluded)"}
    try:
        va, cores, model, ita, dta = _oracle_rate_all_cores(A, b, L, s, cd, lam, seed, v1, budget_s)
        out = {"value": va, "unit": unit, "cores": cores, "kind": "oracle", "cpu_model": model,
               "sample": f"{cores} x {ita} {what}, one single-threaded oracle process per host core on its own "
                         f"block sequence, started together (slowest {dta:.1f} s; factor phase excluded)",
               "one_core": out}
    except Exception as exc:  # the single-thread figure still stands
        out["all_cores_error"] = f"{type(exc).__name__}: {exc}"
    return out


def _oracle_factors(A, s, lam, cd):
    """All-block factors by the oracle (small systems)."""
    import oracle
    return oracle.cdpp_factor(A, s, lam) if cd else oracle.kpp_factor(A, s, lam)


def _factors_numpy_gram(A, s, lam):
    """K++ factors for a large sample: block Grams by numpy, Cholesky by the oracle (factor phase is
    not part of the timed oracle sample)."""
    import oracle
    m = A.shape[0]
    nb = -(-m // s)
    L = np.zeros((nb, s, s))
    for j in range(nb):
        As = A[j * s:(j + 1) * s]
        ln = As.shape[0]
        L[j].reshape(-1)[:ln * ln] = oracle.cholesky(As @ As.T + lam * np.eye(ln)).reshape(-1)
    return L


def krylov_reference(kpp, A, b, tol, method, reps=3, restart=512):
    """The library's FP64 CG (kpp_cg) or GMRES(restart) (kpp_gmres) on the same system and GPU, from
    x0 = 0, one persistent launch each; the fastest of `reps` runs by the kernel's events, with the
    paper's flop model for the method (CG 2n^2 + 11n per iteration, GMRES 2n^2 T + 4n T (T + 1))."""
    import torch
    n = A.shape[0]
    best = None
    for _ in range(reps):
        x = torch.zeros(n, dtype=torch.float64, device="cuda")
        rep = kpp.cg(A, b, x, tol=tol) if method == "cg" else kpp.gmres(A, b, x, restart=restart, tol=tol)
        if best is None or rep.kernel_ms < best.kernel_ms:
            best = rep
    T = best.iters
    flops = (2 * n * n + 11 * n) * T if method == "cg" else 2 * n * n * T + 4 * n * T * (T + 1)
    what = ("plain FP64 conjugate gradients (kpp_cg)" if method == "cg"
            else f"FP64 GMRES({restart}) with classical Gram-Schmidt + reorthogonalisation (kpp_gmres)")
    return {"what": what + ", same system and GPU, x0 = 0, one persistent launch, fastest of 3",
            "iters": T, "time_to_tol_ms": best.kernel_ms, "rel_res_true": best.rel_res_true,
            "flops_paper_model": flops,
            "flops_model": "(2 n^2 + 11 n) per iteration" if method == "cg" else "2 n^2 T + 4 n T (T + 1)"}


# ---------------------------------------------------------------------------------------------
# Workloads
# ---------------------------------------------------------------------------------------------

class Workload:
    unit = "block-iters/s"
    metric = METRIC
    dtype = "f64"
    kernel = ""

    def setup(self, kpp, torch, rank):
        raise NotImplementedError

    def step(self) -> dict:
        """One step; returns units (the metric's numerator), ok, and what the roofline needs."""
        raise NotImplementedError

    def roofline(self, steps, peaks) -> dict:
        raise NotImplementedError

    def e2e(self):
        return None

    def cpu_baseline(self, budget_s):
        return None

    def extra(self, steps) -> dict:
        return {}


def _hbm_roof(kernel, byts_per_launch, launch_ms, peaks, traffic_key, per_iter, extra=None):
    ach = byts_per_launch / (launch_ms / 1e3) / 1e9
    hbm = peaks.get("hbm_gbs", 6800.0)
    out = {"kernel": kernel, "bound": "hbm", "achieved": ach, "peak": hbm, "unit": "GB/s", "frac": ach / hbm,
           "traffic": NCU_TRAFFIC_PER_LAUNCH.get(traffic_key), "launch_ms": launch_ms, "per_iter": per_iter,
           "peak_source": "MEASURED_PEAKS.json hbm_gbs (measured)"}
    out.update(extra or {})
    return out


class SingleFP64(Workload):
    """One FP64 system, factor + solve per step (CD++ n=4096, or K++ 2000x200)."""

    def __init__(self, name, grid_tune=False):
        self.name = name
        self.grid_tune = grid_tune
        self.cd = name.startswith("cdpp4096")
        if self.cd:
            self.sy = W.cdpp_fp64_spd()
            self.desc = ("CD++ FP64, dense SPD n=4096 = U diag(sigma) U^T (U Haar; 50 outliers log-spaced 1e2..1e4 + "
                         "4046 ~U[1,10]), b~N(0,I), s=64 contiguous, lambda=1e-4, tol=1e-8, x0=0")
            self.kernel = "cd4_kernel"
        else:
            self.sy = W.kpp_fp64_2000x200()
            self.desc = ("K++ FP64, 2000x200 consistent LS A=Z D V^T (10 outliers 1e2..1e3 + 190 ~U[1,2]), s=20, "
                         "lambda=1e-3, tol=1e-8, x0=0")
            self.kernel = "solve2_kernel"
        self.seed = 1 if self.cd else 0

    def setup(self, kpp, torch, rank):
        self.kpp, self.torch = kpp, torch
        sy = self.sy
        m, n = sy.A.shape
        self.Ad = torch.as_tensor(sy.A, device="cuda")
        self.bd = torch.as_tensor(sy.b, device="cuda")
        self.x = torch.zeros(n, dtype=torch.float64, device="cuda")
        self.P = kpp.Partition(m, sy.s)
        self.prm = kpp.params(lam=sy.lam, tol=sy.tol, seed=self.seed, sys_id=rank,
                              grid=kpp.GRID_TUNE if self.grid_tune else 0)
        if self.grid_tune:
            self.desc += "; CTAs per system chosen by the launch autotuner (during warm-up)"
        self.solve = kpp.cdpp_solve if self.cd else kpp.kpp_solve

    def step(self):
        kpp = self.kpp
        self.x.zero_()
        F = kpp.Factors(self.Ad, self.P, self.sy.lam, 1 if self.cd else 0)
        rep = self.solve(self.Ad, self.bd, self.x, self.P, F, self.prm)
        del F
        return {"units": rep.iters, "ok": rep.status == kpp.OK and rep.rel_res_true <= self.sy.tol,
                "kernel_ms": rep.kernel_ms, "kernel_launches": rep.launches, "iters": rep.iters,
                "outer": rep.outer, "rel_res": rep.rel_res_true}

    def per_iter(self):
        """Algorithmic FP64 flops and bytes of one block iteration (k = 1)."""
        m, n = self.sy.A.shape
        s = self.sy.s
        if self.cd:
            # u = W_S^T r_S from the memoised W = G^-1 A_S (s x n), R_x and R_m read + written, x_S, r_S
            return 2 * s * n + 2 * s * s + 10 * n + 2 * s, 8 * (s * n + s * s + 8 * n + s)
        # r = A_S x (s x n), w = A_S^T y (second read of A_S from L2), x and m read + written
        return 4 * s * n + 2 * s * s + 6 * n + 2 * s, 8 * (s * n + s * s + 4 * n + 2 * s)

    def roofline(self, steps, peaks):
        flops, byts = self.per_iter()
        iters = statistics.mean(st["iters"] for st in steps)
        kms = statistics.mean(st["kernel_ms"] for st in steps)
        launches = statistics.mean(st["kernel_launches"] for st in steps)
        per_launch_ms = kms / max(launches, 1)
        ach = iters / launches * flops / (per_launch_ms / 1e3) / 1e9
        achb = iters / launches * byts / (per_launch_ms / 1e3) / 1e9
        pk = fp64_peak_gflops(peaks)
        nom = fp64_peak_nominal(peaks)
        hbm = peaks.get("hbm_gbs", 6800.0)
        return {"kernel": self.kernel, "bound": "alu", "achieved": ach, "peak": pk, "unit": "GFLOP/s",
                "frac": ach / pk, "traffic": NCU_TRAFFIC_PER_LAUNCH.get(f"{self.kernel}/{self.name}"),
                "launch_ms": per_launch_ms, "per_iter": {"flops": flops, "bytes": byts},
                "peak_source": FP64_PEAK_SOURCE,
                "nominal_peak": {**nom, "frac": ach / nom["peak"]},
                "hbm_view": {"achieved": achb, "peak": hbm, "unit": "GB/s", "frac": achb / hbm,
                             "peak_source": "MEASURED_PEAKS.json hbm_gbs (measured)"}}

    def extra(self, steps):
        """CD++ only: plain FP64 CG on the same system as a reference point, and both methods' flop counts
        (CG: the paper's 2n^2 + 11n per iteration; CD++: per-iteration flops of this step times the
        iterations, plus the factor phase nb (s^3/3 + 2 s^2 n), Cholesky and the memo W = G^-1 A_S)."""
        if not self.cd:
            return {}
        n, s = self.sy.A.shape[1], self.sy.s
        nb = -(-n // s)
        iters = statistics.mean(st["iters"] for st in steps)
        out = {"cdpp_flops": {"iterations": self.per_iter()[0] * iters,
                              "factor_phase": nb * (s ** 3 / 3 + 2 * s * s * n)}}
        if not getattr(self, "run_cg_reference", True):
            return out
        for name in ("cg", "gmres"):
            try:
                out[f"{name}_reference"] = krylov_reference(self.kpp, self.Ad, self.bd, self.sy.tol, name)
            except Exception as exc:  # a failed reference point must not lose the bench line
                out[f"{name}_reference"] = {"error": f"{type(exc).__name__}: {exc}"}
        return out

    def e2e(self):
        kpp, torch = self.kpp, self.torch
        n = self.sy.A.shape[1]
        # pinned host buffers (numpy views of page-locked torch tensors, kept alive here); pageable
        # buffers if page-locking fails, said so in the note
        At = torch.as_tensor(np.ascontiguousarray(self.sy.A))
        bt = torch.as_tensor(self.sy.b.copy())
        xt = torch.zeros(n, dtype=torch.float64)
        try:
            At, bt, xt = At.pin_memory(), bt.pin_memory(), xt.pin_memory()
            kind = "pinned"
        except RuntimeError:
            kind = "pageable (page-locking failed)"
        A_h, b_h, x_h = At.numpy(), bt.numpy(), xt.numpy()
        ets = []
        for _ in range(2):
            x_h[:] = 0.0
            t0 = time.perf_counter()
            rep = kpp.solve_host(A_h, b_h, x_h, self.sy.s, 1 if self.cd else 0, self.prm)
            ets.append(time.perf_counter() - t0)
            assert rep.status == kpp.OK
        return {"value": rep.iters / ets[-1], "unit": self.unit,
                "h2d_bytes_per_step": A_h.nbytes + b_h.nbytes + x_h.nbytes, "d2h_bytes_per_step": x_h.nbytes,
                "time_to_tol_ms": 1e3 * ets[-1],
                "note": f"{kind} host buffers through kpp_solve_host (copies in, factor, solve, x back)"}

    def cpu_baseline(self, budget_s):
        L = _oracle_factors(self.sy.A, self.sy.s, self.sy.lam, self.cd)
        return _cpu_baseline_both(self.sy.A, self.sy.b, L, self.sy.s, self.cd, self.sy.lam, self.seed, budget_s,
                                  self.unit, "block iterations of the same workload (FP64 C oracle)", it0=256)


class MemoSPD(SingleFP64):
    """The cdpp4096 system solved by CD++ with the online block memoisation (random s-subsets memoised
    as they are drawn) instead of the fixed partition: kpp_solve_memo, to 1e-8."""

    def __init__(self):
        super().__init__("cdpp4096")
        self.name = "cdpp4096-memo"
        self.kernel = "memo_kernel"
        self.desc = self.desc.replace("s=64 contiguous", "s=64 random subsets memoised online (Sec. 4)")
        self.run_cg_reference = False

    def step(self):
        kpp = self.kpp
        self.x.zero_()
        rep, nb = kpp.solve_memo(self.Ad, self.bd, self.x, self.sy.s, self.prm, cd=True)
        self.nblocks = nb
        return {"units": rep.iters, "ok": rep.status == kpp.OK and rep.rel_res_true <= self.sy.tol,
                "kernel_ms": rep.kernel_ms, "kernel_launches": rep.launches, "iters": rep.iters,
                "outer": 0, "rel_res": rep.rel_res_true, "blocks": nb}

    def per_iter(self):
        """One memo CD++ step: r = A_S x - b_S from the stored rows (s x n), y = G^-1 r (s x s), x and the
        momentum on every column (read + written)."""
        n, s = self.sy.A.shape[1], self.sy.s
        return 2 * s * n + 2 * s * s + 5 * n, 8 * (s * n + s * s + 4 * n + 2 * s)

    def roofline(self, steps, peaks):
        flops, byts = self.per_iter()
        iters = statistics.mean(st["iters"] for st in steps)
        kms = statistics.mean(st["kernel_ms"] for st in steps)
        out = _hbm_roof(self.kernel, iters * byts, kms, peaks, f"{self.kernel}/{self.name}", {"bytes": byts},
                        {"note": "all window launches of the step; the stored rows of the memoised blocks "
                                 "(blocks x s x n FP64) exceed L2, so each step reads A_S from HBM"})
        return out

    def extra(self, steps):
        return {"memoised_blocks": statistics.mean(st["blocks"] for st in steps),
                "fixed_partition_blocks": -(-self.sy.A.shape[0] // self.sy.s)}

    def e2e(self):
        return None

    def cpu_baseline(self, budget_s):
        import oracle
        A, b, s = self.sy.A, self.sy.b, self.sy.s
        k = 64
        while True:
            t0 = time.perf_counter()
            oracle.run_memo(A, b, s, cd=True, lam=self.sy.lam, tol=0.0, max_iters=k, seed=self.seed)
            dt = time.perf_counter() - t0
            if dt > budget_s / 4 or k >= 1 << 20:
                break
            k *= 4
        return {"value": k / dt, "unit": self.unit, "cores": 1, "kind": "oracle",
                "sample": f"{k} steps of the oracle's memo CD++ (oracle.run_memo) on the same system, one host "
                          f"thread, new blocks factored as drawn ({dt:.1f} s)"}


class LsqrLS(Workload):
    """K++ with the inexact projection of Sec. 4.1 (sketch-preconditioned LSQR, tau = 2 s, t_max = 8) on
    large blocks of an FP64 least-squares system: the sketch preconditioners of every block, then the
    solve to 1e-8.  After the timed steps the exact K++ (Cholesky projections) solves the same system
    once, for comparison."""
    dtype = "f64"

    def __init__(self, m=65536, n=2048, s=512, t_max=8):
        self.m, self.n, self.s, self.t_max = m, n, s, t_max
        self.name = "kpp-lsqr"
        self.kernel = "lsqr_kernel"
        self.lam, self.tol = 1e-3, 1e-8
        self.desc = (f"K++ FP64 with the inexact projection (sketch-preconditioned LSQR, Sec. 4.1): {m}x{n} LS "
                     "A=Z D V^T (Z~N(0,1/m), V Haar, 100 outliers log-spaced 10..1000 + U[0.5,1]) stored FP32 and "
                     f"widened, b = A x*, s={s} contiguous, SRHT sketch tau=2s, t_max={t_max}, lambda=1e-3, "
                     "tol 1e-8 on the FP64 residual, x0=0")

    def setup(self, kpp, torch, rank):
        self.kpp, self.torch = kpp, torch
        A32, self.b, self.x_star, _ = W.torch_lowrank_ls(self.m, self.n, 100, 10.0, 1000.0, 0.5, 1.0,
                                                        seed=7 + 1000 * rank, dtype="f32")
        self.A = A32.double()
        del A32
        self.x = torch.zeros(self.n, dtype=torch.float64, device="cuda")
        self.P = kpp.Partition(self.m, self.s)
        np2 = 1 << (self.n - 1).bit_length()
        rng = np.random.default_rng(11 + rank)
        self.T = np.sort(rng.choice(np2, 2 * self.s, replace=False))
        self.d = torch.as_tensor(W.rademacher_signs(np2, 12 + rank), device="cuda")
        self.prm = kpp.params(lam=self.lam, tol=self.tol, seed=0, sys_id=rank)

    def step(self):
        kpp = self.kpp
        self.x.zero_()
        F = kpp.LsqrFactors(self.A, self.P, self.lam, self.T, self.d)
        rep = kpp.solve_lsqr(self.A, self.b, self.x, self.P, F, self.t_max, self.prm)
        del F
        return {"units": rep.iters, "ok": rep.status == kpp.OK and rep.rel_res_true <= self.tol,
                "kernel_ms": rep.kernel_ms, "kernel_launches": rep.launches, "iters": rep.iters,
                "outer": 0, "rel_res": rep.rel_res_true}

    def per_iter_bytes(self):
        """The method's bytes of one step: A_S once, L_j^{-1} twice per LSQR iteration, the n-vectors."""
        s, n = self.s, self.n
        return 8 * (s * n + 2 * self.t_max * s * s + 6 * n)

    def roofline(self, steps, peaks):
        iters = statistics.mean(st["iters"] for st in steps)
        kms = statistics.mean(st["kernel_ms"] for st in steps)
        byts = self.per_iter_bytes()
        return _hbm_roof(self.kernel, iters * byts, kms, peaks, f"{self.kernel}/{self.name}", {"bytes": byts},
                         {"note": "one launch per solve; A_S stays in L2 for the 2 t_max + 2 products of a step, "
                                  "which are counted once; the step is bound by its group barriers "
                                  "(5 per LSQR iteration)"})

    def extra(self, steps):
        kpp, torch = self.kpp, self.torch
        x = torch.zeros(self.n, dtype=torch.float64, device="cuda")
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        F = kpp.Factors(self.A, self.P, self.lam, 0)
        rep = kpp.kpp_solve(self.A, self.b, x, self.P, F, kpp.params(lam=self.lam, tol=self.tol, seed=0))
        torch.cuda.synchronize()
        dt = time.perf_counter() - t0
        stages = F.stage_ms()
        del F
        return {"exact_kpp_reference": {"what": "K++ with exact Cholesky projections (kpp_factor_blocks + "
                                                "kpp_solve) on the same system, one run after the timed steps",
                                        "time_to_tol_ms": 1e3 * dt, "iters": rep.iters,
                                        "rel_res_true": rep.rel_res_true, "factor_stages_ms": stages,
                                        "solve_kernel_ms": rep.kernel_ms}}

    def cpu_baseline(self, budget_s):
        import oracle
        rows = 8 * self.s
        A = self.A[:rows].cpu().numpy()
        b = self.b[:rows].cpu().numpy()
        d = self.d.cpu().numpy()
        Lsk = oracle.lsqr_factors(A, self.s, self.lam, self.T, d)
        k = 16
        while True:
            t0 = time.perf_counter()
            oracle.run_lsqr(A, b, Lsk, self.s, self.t_max, lam=self.lam, tol=0.0, max_iters=k, seed=0)
            dt = time.perf_counter() - t0
            if dt > budget_s / 4 or k >= 1 << 16:
                break
            k *= 4
        return {"value": k / dt, "unit": self.unit, "cores": 1, "kind": "oracle",
                "sample": f"{k} steps of the oracle's inexact-projection K++ (oracle.run_lsqr, t_max={self.t_max}) "
                          f"on the first {rows} rows of the same matrix, one host thread (preconditioners "
                          f"excluded; {dt:.1f} s)"}


class MixedSPD(SingleFP64):
    """The cdpp4096 system stored FP32 / BF16 with FP32 iterations and FP64 refinement."""

    def __init__(self, storage):
        super().__init__("cdpp4096")
        self.storage = storage
        self.name = f"cdpp4096-{storage}"
        self.dtype = "f32"
        self.desc = (f"CD++ on the n=4096 SPD system of the default workload stored {storage.upper()} "
                     "(the stored matrix is the system), FP32 iterations + FP64 refinement (inner tol 1e-3), s=64, "
                     "lambda=1e-4, tol 1e-8, x0=0")

    def setup(self, kpp, torch, rank):
        super().setup(kpp, torch, rank)
        self.Ad = self.Ad.to(torch.float32 if self.storage == "f32" else torch.bfloat16)
        self.prm = kpp.params(lam=self.sy.lam, tol=self.sy.tol, seed=1, sys_id=rank, refine=1, inner_tol=1e-3)

    def per_iter_bytes(self):
        n, s = self.sy.A.shape[1], self.sy.s
        esz = 4 if self.storage == "f32" else 2
        return s * n * esz + s * s * 4 + 4 * (8 * n + s)

    def roofline(self, steps, peaks):
        byts = self.per_iter_bytes()
        iters = statistics.mean(st["iters"] for st in steps)
        kms = statistics.mean(st["kernel_ms"] for st in steps)
        launches = statistics.mean(st["kernel_launches"] for st in steps)
        return _hbm_roof(self.kernel, iters * byts / launches, kms / launches, peaks, f"{self.kernel}/{self.name}",
                         {"bytes": byts})

    def extra(self, steps):
        return {"outer_steps": steps[-1]["outer"]}

    def e2e(self):
        return None

    def cpu_baseline(self, budget_s):
        return None


class RhtSPD(SingleFP64):
    """The cdpp4096 system with CD++'s randomized Hadamard preprocessing inside the step (Alg. 3):
    Abar = Q A Q^T and bbar = Q b on the GPU, factors and CD++ on (Abar, bbar), x = Q^T xbar."""

    def __init__(self):
        super().__init__("cdpp4096")
        self.name = "cdpp4096-rht"
        self.desc += ("; randomized Hadamard preprocessing Q = H_n diag(d) / sqrt(n) (d Rademacher, seed 7) "
                      "applied on the GPU inside every step, and x = Q^T xbar after it")

    def setup(self, kpp, torch, rank):
        super().setup(kpp, torch, rank)
        n = self.sy.A.shape[1]
        self.d = torch.as_tensor(W.rademacher_signs(n, 7), device="cuda")
        self.xbar = torch.zeros(n, dtype=torch.float64, device="cuda")

    def _solve(self, A, b):
        kpp, torch = self.kpp, self.torch
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record()
        Abar, bbar = kpp.rht_forward(self.d, A, b)
        e1.record()
        self.xbar.zero_()
        F = kpp.Factors(Abar, self.P, self.sy.lam, 1)
        rep = kpp.cdpp_solve(Abar, bbar, self.xbar, self.P, F, self.prm)
        x = kpp.rht_inverse(self.d, self.xbar)
        del F, Abar
        return rep, x, e0, e1

    def step(self):
        rep, self.x, e0, e1 = self._solve(self.Ad, self.bd)
        # the original system's FP64 residual (equal to the transformed one up to rounding: Q is orthogonal)
        res = self.kpp.rel_residual(self.Ad, self.bd, self.x)
        return {"units": rep.iters, "ok": rep.status == self.kpp.OK and res <= 1.0001 * self.sy.tol,
                "kernel_ms": rep.kernel_ms, "kernel_launches": rep.launches, "iters": rep.iters,
                "outer": rep.outer, "rel_res": res, "rht_ms": e0.elapsed_time(e1)}

    def extra(self, steps):
        n = self.sy.A.shape[1]
        rht_ms = statistics.mean(st["rht_ms"] for st in steps)
        # two streaming passes over the n x n FP64 matrix (read + write each) and the vector
        byts = 4 * 8 * n * n + 2 * 8 * n
        return {"rht_forward_ms": rht_ms, "rht_forward_gbs": byts / (rht_ms / 1e3) / 1e9,
                "rht_forward_bytes": byts}

    def cpu_baseline(self, budget_s):
        out = super().cpu_baseline(budget_s)
        out["sample"] += "; on the untransformed matrix (same sizes, same work per iteration)"
        return out

    def e2e(self):
        """Pinned host A and b in, transform + factors + CD++ + inverse transform, x out."""
        torch = self.torch
        A_h = torch.as_tensor(self.sy.A).pin_memory()
        b_h = torch.as_tensor(self.sy.b).pin_memory()
        x_h = torch.empty_like(b_h).pin_memory()
        ets = []
        for _ in range(2):
            torch.cuda.synchronize()
            t0 = time.perf_counter()
            A = A_h.to("cuda", non_blocking=True)
            b = b_h.to("cuda", non_blocking=True)
            rep, x, _, _ = self._solve(A, b)
            x_h.copy_(x, non_blocking=True)
            torch.cuda.synchronize()
            ets.append(time.perf_counter() - t0)
            assert rep.status == self.kpp.OK
            del A, b
        return {"value": rep.iters / ets[-1], "unit": self.unit,
                "h2d_bytes_per_step": A_h.numel() * 8 + b_h.numel() * 8, "d2h_bytes_per_step": x_h.numel() * 8,
                "time_to_tol_ms": 1e3 * ets[-1], "note": "pinned host A, b in and x out around the whole step"}


class MixedLS(Workload):
    """K++ on a 262144 x 4096 LS stored BF16 / FP32, FP32 iterations + FP64 refinement (the default
    workload).  After the timed steps the plain FP64 K++ path solves the same system (the stored matrix
    widened to FP64) once, for the comparison of the two forms on the same GPU."""

    def __init__(self, storage="bf16", noisy=False, m=262144, n=4096, s=512):
        self.storage, self.noisy = storage, noisy
        self.m, self.n, self.s = m, n, s
        # BF16 blocks of up to 512 rows take the W-memo kernel; FP32 storage of 512-row blocks does not fit
        # its shared memory and stays on the small-block kernel
        self.kernel = "kw_kernel" if storage == "bf16" else "solve2_kernel"
        self.name = f"mixed{m}-{storage}"
        self.lam = 1e-3
        self.tol = 1e-8
        self.dtype = "f32"  # the arithmetic of the iterations (BF16 entries are widened exactly to FP32)
        self.run_fp64_reference = True
        noise = ("b = A_stored x* + 1e-6 N(0,I) (noisy variant: attained residual reported, no tolerance)"
                 if noisy else "b = A_stored x* (noise-free headline)")
        self.desc = (f"K++ mixed precision, {m}x{n} LS A=Z D V^T stored {storage.upper()} (Z~N(0,1/m), V Haar, "
                     f"100 outliers log-spaced 10..1000 + U[0.5,1]), {noise}, s={s}, lambda=1e-3, "
                     "tensor-core block Grams, FP32 Cholesky (FP64 for blocks it finds ill-conditioned), "
                     "FP32 iterations + FP64 refinement (inner tol 1e-3), "
                     "tol 1e-8 on the FP64 residual, x0=0")

    def setup(self, kpp, torch, rank):
        self.kpp, self.torch = kpp, torch
        self.A, self.b, self.x_star, _ = W.torch_lowrank_ls(self.m, self.n, 100, 10.0, 1000.0, 0.5, 1.0,
                                                           seed=2 + 1000 * rank, dtype=self.storage,
                                                           noise=1e-6 if self.noisy else 0.0)
        self.x = torch.zeros(self.n, dtype=torch.float64, device="cuda")
        self.P = kpp.Partition(self.m, self.s)
        self.prm = kpp.params(lam=self.lam, tol=self.tol, refine=1, inner_tol=1e-3, seed=0, sys_id=rank,
                              max_outer=4 if self.noisy else 20, max_iters=20000 if self.noisy else 1000000)

    def step(self):
        kpp = self.kpp
        self.x.zero_()
        F = kpp.Factors(self.A, self.P, self.lam, 0)
        rep = kpp.kpp_solve(self.A, self.b, self.x, self.P, F, self.prm, allow_no_conv=self.noisy)
        stages = F.stage_ms()
        fp64_blocks = F.fp64_blocks
        del F
        ok = rep.rel_res_true <= self.tol if not self.noisy else math.isfinite(rep.rel_res_true)
        return {"units": rep.iters, "ok": ok, "kernel_ms": rep.kernel_ms, "kernel_launches": rep.launches,
                "iters": rep.iters, "outer": rep.outer, "rel_res": rep.rel_res_true, "stages": stages,
                "fp64_blocks": fp64_blocks}

    def per_iter_bytes(self):
        esz = 2 if self.storage == "bf16" else 4
        s, n = self.s, self.n
        # the method's bytes: A_S once, G_S^-1 (FP32), x and m read + written (FP32), r_S and y
        return s * n * esz + s * s * 4 + 4 * n * 4 + 2 * s * 4

    def per_iter_bytes_kernel(self):
        """What the block-step kernel reads besides: the memoised W_S = G_S^-1 A_S (s x n FP32) in place of
        G_S^-1 (the large-block kernel; the small-block kernel reads G_S^-1 as the method does)."""
        if self.kernel != "kw_kernel":
            return self.per_iter_bytes()
        return self.per_iter_bytes() - self.s * self.s * 4 + self.s * self.n * 4

    def block_step(self, steps, peaks):
        """The block step (S2-S6) against HBM: algorithmic bytes per iteration x iterations / the
        iteration kernel's device time (CUDA events around its launches)."""
        byts, kbyts = self.per_iter_bytes(), self.per_iter_bytes_kernel()
        iters = statistics.mean(st["iters"] for st in steps)
        kms = statistics.mean(st["kernel_ms"] for st in steps)
        launches = statistics.mean(st["kernel_launches"] for st in steps)
        out = _hbm_roof(self.kernel, iters * byts / launches, kms / launches, peaks, f"{self.kernel}/{self.name}",
                        {"bytes": byts})
        ach_k = iters * kbyts / (kms / 1e3) / 1e9
        out["us_per_iter"] = 1e3 * kms / iters
        out["with_memo_reads"] = {"bytes_per_iter": kbyts, "achieved": ach_k, "frac": ach_k / out["peak"],
                                  "note": "counting the memo W_S the kernel streams as well (s x n FP32)"}
        return out

    def roofline(self, steps, peaks):
        """The dominant kernel of the step: the Cholesky of every block (FP32, with FP64 for the blocks it
        flags), or the block-step kernel, whichever took more device time (events on the launching stream
        for both)."""
        st = steps[-1]["stages"]
        chol_ms = statistics.mean(x["stages"]["cholesky"] for x in steps)
        kms = statistics.mean(x["kernel_ms"] for x in steps)
        self._block = self.block_step(steps, peaks)
        if not (chol_ms > kms):
            return self._block
        nb = -(-self.m // self.s)
        flops = nb * self.s ** 3 / 3.0
        ach = flops / (chol_ms / 1e3) / 1e9
        pk = fp32_peak_gflops(peaks)
        return {"kernel": "cholesky_f32_kernel", "bound": "alu", "achieved": ach, "peak": pk, "unit": "GFLOP/s",
                "frac": ach / pk, "traffic": NCU_TRAFFIC_PER_LAUNCH.get(f"cholesky_f32_kernel/{self.name}"),
                "launch_ms": chol_ms, "per_launch": {"flops": flops, "blocks": nb, "s": self.s,
                                                     "count": "s^3/3 per block (the paper's Cholesky count)"},
                "launches": "cholesky_f32_kernel over every block (one CTA per block), then cholesky_kernel "
                            "(FP64) over the blocks it flagged (the others return at once); the time is the "
                            "stage's events around both",
                "fp64_blocks": steps[-1].get("fp64_blocks"),
                "peak_source": "nominal: 152 SMs x 128 FP32 FMA/clk x 2 flop x sm_max_mhz",
                "factor_stages_ms": st}

    def extra(self, steps):
        x_err = float(((self.x - self.x_star).norm() / self.x_star.norm()).item())
        stages = {k: statistics.mean(x["stages"][k] for x in steps) for k in steps[-1]["stages"]}
        out = {"outer_steps": steps[-1]["outer"], "x_rel_err_vs_x_star": x_err, "factor_stages_ms": stages,
               "fp64_cholesky_blocks": steps[-1].get("fp64_blocks"), "block_step": self._block}
        if self.noisy:
            out["attained_rel_res"] = steps[-1]["rel_res"]
        if self.run_fp64_reference and not self.noisy:
            try:
                out["fp64_reference"] = self.fp64_reference()
            except Exception as exc:  # a failed reference point must not lose the bench line
                out["fp64_reference"] = {"error": f"{type(exc).__name__}: {exc}"}
        return out

    def fp64_reference(self):
        """The plain FP64 K++ path on the same system (the stored matrix widened to FP64, the same b):
        FP64 block Grams and Cholesky, FP64 iterations to 1e-8, one run timed with events."""
        kpp, torch = self.kpp, self.torch
        A64 = self.A.double()
        x = torch.zeros(self.n, dtype=torch.float64, device="cuda")
        prm = kpp.params(lam=self.lam, tol=self.tol, seed=0)
        torch.cuda.synchronize()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record()
        F = kpp.Factors(A64, self.P, self.lam, 0)
        rep = kpp.kpp_solve(A64, self.b, x, self.P, F, prm)
        e1.record()
        e1.synchronize()
        stages = F.stage_ms()
        del F, A64
        return {"what": "plain FP64 K++ (FP64 storage of the same stored values, FP64 Grams, Cholesky and "
                        "iterations, no refinement) on the same system and GPU, one run after the timed steps",
                "time_to_tol_ms": e0.elapsed_time(e1), "iters": rep.iters, "rel_res_true": rep.rel_res_true,
                "solve_kernel_ms": rep.kernel_ms, "factor_stages_ms": stages, "status": rep.status}

    def e2e(self):
        """Host buffers (pinned) in and out around the public calls: A, b to the device, factor, solve, x back."""
        kpp, torch = self.kpp, self.torch
        A_h = self.A.cpu().pin_memory()
        b_h = self.b.cpu().pin_memory()
        x_h = torch.zeros(self.n, dtype=torch.float64).pin_memory()
        ets = []
        for _ in range(4):
            torch.cuda.synchronize()
            t0 = time.perf_counter()
            A = A_h.to("cuda", non_blocking=True)
            b = b_h.to("cuda", non_blocking=True)
            x = torch.zeros(self.n, dtype=torch.float64, device="cuda")
            F = kpp.Factors(A, self.P, self.lam, 0)
            rep = kpp.kpp_solve(A, b, x, self.P, F, self.prm, allow_no_conv=self.noisy)
            x_h.copy_(x)
            ets.append(time.perf_counter() - t0)
            del F, A
        et = statistics.median(ets[1:])  # the first run maps the buffers; the median of the other three
        return {"value": rep.iters / et, "unit": self.unit,
                "h2d_bytes_per_step": A_h.numel() * A_h.element_size() + b_h.numel() * 8,
                "d2h_bytes_per_step": self.n * 8, "time_to_tol_ms": 1e3 * et,
                "runs_ms": [1e3 * v for v in ets],
                "note": "pinned host buffers copied in and out around kpp_factor_blocks + kpp_solve; "
                        "median of runs 2-4"}

    def oracle_sample(self, blocks=16):
        """The first `blocks` blocks (blocks x s rows x n) of the stored matrix widened to FP64, with b and
        the block factors; the oracle's per-iteration work is the workload's (one s x n block)."""
        rows = blocks * self.s
        A = np.ascontiguousarray(self.A[:rows].double().cpu().numpy())
        b = np.ascontiguousarray(self.b[:rows].cpu().numpy())
        return A, b, _factors_numpy_gram(A, self.s, self.lam), rows

    def cpu_baseline(self, budget_s):
        A, b, L, rows = self.oracle_sample()
        return _cpu_baseline_both(A, b, L, self.s, False, self.lam, 0, budget_s, self.unit,
                                  f"FP64 oracle block iterations (s={self.s}, n={self.n}) on the first {rows} rows "
                                  "of the stored matrix widened to FP64", it0=16)


def host_mixed_sample(m=262144, n=4096, s=512, blocks=16, storage="bf16"):
    """A host-built sample of the mixed-precision workload for the reference arm (no GPU): `blocks`
    blocks of s rows of A = Z D V^T with Z ~ N(0, 1/m) (the full system's scaling), V Haar n x n and the
    planted spectrum, rounded to the storage type, b = A_sample x*.  Same shapes and distributions as
    the device-built system, not the same values."""
    rng = np.random.default_rng(2)
    rows = blocks * s
    z = rng.standard_normal((rows, n)) * (1.0 / math.sqrt(m))
    v = W.haar_orthogonal(n, rng)
    d = W.planted_spectrum(n, 100, 10.0, 1000.0, 0.5, 1.0, rng)
    A = W.round_to_storage(np.ascontiguousarray(z @ (d[:, None] * v.T)), storage)
    b = A @ np.random.default_rng(103).standard_normal(n)
    return A, b


class Batched(Workload):
    """64 under-determined FP32 systems with 8-column panels: factors, then one autotuned plan per step,
    captured into a CUDA graph and replayed."""

    kernel = "stream_kernel"

    def __init__(self, nsys=64, m=2048, n=65536, k=8, s=256, grid=None, tune_s=False):
        self.nsys, self.m, self.n, self.k, self.s = nsys, m, n, k, s
        self.grid = grid  # CTAs per system; None: the launch autotuner
        self.tune_s = tune_s  # pick s among 128, 256, 512 with the block-size autotuner (before the steps)
        self.s_tuning = None
        self.tol = 1e-8
        self.dtype = "f32"
        self.desc = (f"{nsys} under-determined min-norm K++ systems, each {m}x{n} FP32 i.i.d. N(0,1) with 20 seeded "
                     f"rows x100, {k} right-hand sides ~N(0,I) each, s={s}, lambda=1e-3 median |a_i|^2, FP32 "
                     "iterations + FP64 refinement (inner tol 1e-3), tol 1e-8 per column; one plan (autotuned CTAs "
                     "per system) captured in a CUDA graph and replayed")

    def setup(self, kpp, torch, rank):
        self.kpp, self.torch = kpp, torch
        self.A, self.B = [], []
        for i in range(self.nsys):
            A, B, _ = W.torch_gaussian_rows(self.m, self.n, 20, 100.0, seed=self.system_seed(rank, i), k_rhs=self.k)
            self.A.append(A)
            self.B.append(B)
        rn = (self.A[0].double() ** 2).sum(dim=1)
        self.lam = 1e-3 * float(torch.median(rn).item())
        self.X = [torch.zeros(self.n, self.k, dtype=torch.float64, device="cuda") for _ in range(self.nsys)]
        if self.tune_s:
            prm = kpp.params(lam=self.lam, tol=self.tol, refine=1, inner_tol=1e-3, seed=0, sys_id=rank * 4096)
            t0 = time.perf_counter()
            best, est = kpp.tune_block_size(self.A, self.B, [128, 256, 512], prm)
            self.s_tuning = {"candidates": {str(k): v for k, v in est.items()}, "chosen": best,
                             "tuning_s": time.perf_counter() - t0,
                             "note": "estimated ms to tol per candidate (kpp_tune_block_size), before the timed steps"}
            self.s = best
            self.desc = self.desc.replace("s=256", f"s={best} (block-size autotuner over 128, 256, 512)")
        self.P = kpp.Partition(self.m, self.s)
        self.prm = kpp.params(lam=self.lam, tol=self.tol, refine=1, inner_tol=1e-3, seed=0, sys_id=rank * 4096,
                              grid=kpp.GRID_TUNE if self.grid is None else self.grid)
        self.cap_stream = torch.cuda.Stream()

    def system_seed(self, rank, i):
        """Seed of system i on rank r: every rank of a replicas run builds its own systems."""
        return 3000 + 1000 * rank + i

    def step(self):
        kpp, torch = self.kpp, self.torch
        cur = torch.cuda.current_stream()
        F = [kpp.Factors(a, self.P, self.lam, 0) for a in self.A]
        plan = kpp.Plan(self.A, self.B, self.X, self.P, F, self.prm, stream=cur)
        n0 = kpp.launch_count()
        g = torch.cuda.CUDAGraph()
        self.cap_stream.wait_stream(cur)
        with torch.cuda.graph(g, stream=self.cap_stream):
            plan.launch(torch.cuda.current_stream())
        graph_launches = kpp.launch_count() - n0
        for x in self.X:
            x.zero_()
        g.replay()
        reps = plan.report(stream=cur)
        self.info = plan.info()
        plan.close()
        del g, F
        it = [reps[i * self.k].iters for i in range(self.nsys)]
        ok = all(r.status == kpp.OK and r.rel_res_true <= self.tol for r in reps)
        return {"units": sum(it), "ok": ok, "iters": sum(it), "max_iters": max(it),
                "outer": max(reps[i * self.k].outer for i in range(self.nsys)),
                "graph_launches": graph_launches, "rel_res": max(r.rel_res_true for r in reps)}

    def per_iter_bytes(self):
        s, n, k = self.s, self.n, self.k
        # A_S once (the second pass re-reads it from L2), X and M panels read + written, G_S^-1 (FP32)
        return s * n * 4 + 4 * n * k * 4 + s * s * 4

    def measure_kernel(self, peaks):
        """The stream kernel's launch duration is not separable inside a replayed graph: time one more
        launch of it (same systems, tuned grid, a fixed 64 steps) with events around the launch."""
        kpp, torch = self.kpp, self.torch
        F = [kpp.Factors(a, self.P, self.lam, 0) for a in self.A]
        X = [torch.zeros_like(x) for x in self.X]
        T = 64
        prm = kpp.params(lam=self.lam, tol=0.0, refine=0, max_iters=T, seed=0, grid=self.info["grid"])
        reps = kpp.kpp_solve_batched(self.A, self.B, X, self.P, F, prm, allow_no_conv=True)
        kms = reps[0].kernel_ms
        self._roof = _hbm_roof(self.kernel, self.per_iter_bytes() * self.nsys * T, kms, peaks,
                               f"{self.kernel}/batched64", {"bytes": self.per_iter_bytes()},
                               {"measured_on": f"one launch of {T} steps x {self.nsys} systems at the tuned grid "
                                               f"({self.info['grid']} CTAs per system)"})
        del F, X

    def roofline(self, steps, peaks):
        self.measure_kernel(peaks)
        return self._roof

    def extra(self, steps):
        out = {"block_size_tuning": self.s_tuning} if self.s_tuning else {}
        return {**out, "plan": self.info, "max_system_iters": steps[-1]["max_iters"], "outer_steps": steps[-1]["outer"],
                "worst_rel_res": steps[-1]["rel_res"],
                "gpu_launches_note": "host-side launches plus the captured graph's kernels (one replay per step)"}

    def e2e(self):
        """Right-hand sides in from pinned host memory and solutions out, around factor + plan + replay
        (the 32 GiB of A stay resident)."""
        kpp, torch = self.kpp, self.torch
        B_h = [b.cpu().pin_memory() for b in self.B]
        X_h = [torch.zeros(self.n, self.k, dtype=torch.float64).pin_memory() for _ in range(self.nsys)]
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        for b, bh in zip(self.B, B_h):
            b.copy_(bh, non_blocking=True)
        st = self.step()
        for x, xh in zip(self.X, X_h):
            xh.copy_(x)
        dt = time.perf_counter() - t0
        assert st["ok"]
        return {"value": st["units"] / dt, "unit": self.unit,
                "h2d_bytes_per_step": sum(b.numel() * 8 for b in B_h),
                "d2h_bytes_per_step": sum(x.numel() * 8 for x in X_h), "time_to_tol_ms": 1e3 * dt,
                "note": "B in / X out through pinned host memory; A resident in HBM"}

    def cpu_baseline(self, budget_s):
        """Oracle iterations on system 0, right-hand side 0 (FP32 entries widened to FP64); factor phase
        excluded."""
        A = np.ascontiguousarray(self.A[0].double().cpu().numpy())
        b = np.ascontiguousarray(self.B[0][:, 0].cpu().numpy())
        L = _factors_numpy_gram(A, self.s, self.lam)
        v, it, dt = _oracle_iter_rate(A, b, L, self.s, False, self.lam, 0, budget_s, it0=8)
        return {"value": v, "unit": self.unit, "cores": 1, "kind": "oracle",
                "sample": f"{it} FP64 oracle block iterations of system 0, one right-hand side, one host thread "
                          f"({dt:.1f} s; factor phase excluded; the GPU counts one iteration per system for its "
                          f"{self.k}-column panel)"}


class Serving(Workload):
    """Continuous-batching CD++ server fed by a Poisson request stream."""

    unit = "solves/s"
    metric = SERVING_METRIC
    kernel = "serve_kernel"

    def __init__(self, n_req=1024, n_mats=32, budget=120 << 30, max_concurrent=64, grid_per_solve=0):
        self.n_req, self.n_mats, self.budget = n_req, n_mats, budget
        self.max_concurrent, self.grid = max_concurrent, grid_per_solve
        self.dtype = "f32"
        self.desc = (f"{n_req} CD++ requests, Poisson arrivals (mean gap 2 ms), catalog of {n_mats} dense SPD "
                     "matrices built as the n=4096 workload (n log-uniform in [512,8192], even ids BF16, odd FP32), "
                     "k ~ U{1..32} right-hand sides ~N(0,I), s=64, lambda=1e-4, FP32 iterations + FP64 "
                     f"refinement, tol 1e-8, HBM budget {budget >> 30} GiB, device-resident request loop (one "
                     "persistent kernel; as many slots of 8 CTAs as fit, at most "
                     f"{max_concurrent}; jobs of <= 8 columns, shortest expected work first), factors "
                     "memoised per matrix across requests")

    def setup(self, kpp, torch, rank):
        self.kpp, self.torch = kpp, torch
        self.sizes = W.serving_catalog(self.n_mats)
        self.mats = []
        self.bf16_to_f32 = []
        for i, n in enumerate(self.sizes):
            dt = "bf16" if i % 2 == 0 else "f32"
            A, _ = W.torch_spd(n, 50, 1e2, 1e4, 1.0, 10.0, seed=7000 + i, dtype=dt)
            if dt == "bf16" and not W.stays_spd(A, 0.1):
                # the BF16-rounded matrix is not SPD (min eigenvalue below 0.1): store this one FP32
                dt = "f32"
                A, _ = W.torch_spd(n, 50, 1e2, 1e4, 1.0, 10.0, seed=7000 + i, dtype=dt)
                self.bf16_to_f32.append(i)
            self.mats.append((n, dt, A))
        self.reqs = W.serving_requests(self.n_req, self.n_mats, 2.0, 1, 32, seed=6000 + rank)
        self.B = [np.random.default_rng(seed).standard_normal((self.sizes[mid], k))
                  for (_, mid, k, seed) in self.reqs]
        self.sv = kpp.Server(self.budget, max_concurrent=self.max_concurrent, grid_per_solve=self.grid)
        self.ids = [self.sv.add_matrix(A, 64, 1e-4, 1) for (_, _, A) in self.mats]
        _log(f"serving: catalog of {len(self.mats)} matrices and {len(self.reqs)} requests ready")

    def step(self):
        kpp = self.kpp
        self.sv.reset_stats()
        t0 = time.perf_counter()
        rids = []
        for (arr_ms, mid, k, seed), B in zip(self.reqs, self.B):
            wait = t0 + arr_ms / 1e3 - time.perf_counter()
            if wait > 0:
                time.sleep(wait)
            prm = kpp.params(tol=1e-8, refine=1, inner_tol=1e-3, seed=seed, sys_id=seed)
            rids.append(self.sv.submit(self.ids[mid], B, prm))
        _log(f"serving: {len(rids)} requests submitted in {time.perf_counter() - t0:.2f} s")
        self.sv.wait_all(1800.0)
        st = self.sv.stats()
        _log(f"serving: done in {time.perf_counter() - t0:.2f} s, p50 {st['p50_ms']:.1f} ms, p99 {st['p99_ms']:.1f} ms")
        byts, iters, worst = 0, 0, 0.0
        for rid, (_, mid, k, _) in zip(rids, self.reqs):
            n = self.sizes[mid]
            done, rc, _, reps = self.sv.poll(rid, n, k)
            esz = 2 if self.mats[mid][1] == "bf16" else 4
            worst = max(worst, max(r.rel_res_true for r in reps))
            # the server runs a request as jobs of at most 8 columns, each its own block sequence of steps
            for c0 in range(0, k, 8):
                it, kc = reps[c0].iters, min(8, k - c0)
                iters += it
                byts += it * (64 * n * esz + 64 * 64 * 4 + 4 * n * kc * 4)
        return {"units": st["completed"], "ok": st["failed"] == 0 and st["completed"] == self.n_req,
                "span_s": st["span_s"], "p50_ms": st["p50_ms"], "p99_ms": st["p99_ms"], "max_ms": st["max_ms"],
                "loop_launches": st["loop_launches"], "loop_slots": st["loop_slots"],
                "solves_per_s": st["solves_per_s"], "peak_bytes": st["peak_bytes"], "alg_bytes": byts,
                "iters": iters, "rel_res": worst}

    def roofline(self, steps, peaks):
        last = steps[-1]
        ach = last["alg_bytes"] / last["span_s"] / 1e9
        hbm = peaks.get("hbm_gbs", 6800.0)
        return {"kernel": "every solve kernel of the mix (device level)", "bound": "hbm", "achieved": ach,
                "peak": hbm, "unit": "GB/s", "frac": ach / hbm, "traffic": None,
                "note": "algorithmic bytes of all requests' block iterations / serving span (arrivals included)",
                "peak_source": "MEASURED_PEAKS.json hbm_gbs (measured)"}

    def extra(self, steps):
        last = steps[-1]
        return {"p50_ms": last["p50_ms"], "p99_ms": last["p99_ms"], "max_ms": last["max_ms"],
                "server_solves_per_s": last["solves_per_s"], "peak_bytes": last["peak_bytes"],
                "loop_launches": last["loop_launches"], "loop_slots": last["loop_slots"],
                "block_iters_per_s": last["iters"] / last["span_s"] if last["span_s"] > 0 else None,
                "block_iters": last["iters"], "requests": self.n_req,
                "bf16_not_spd_stored_f32": [(i, self.sizes[i]) for i in self.bf16_to_f32]}

    def e2e(self):
        # every request already enters as a host panel and leaves as one: the metric is end to end
        return None

    def cpu_baseline(self, budget_s):
        """Oracle CD++ solves (FP64, one column, to 1e-8) of the first requests with n <= 2048, until about
        budget_s of CPU time; reported per request of the stream's mean width k."""
        import oracle
        t_used, cols = 0.0, 0
        for (_, mid, k, seed), B in zip(self.reqs, self.B):
            n, dt, A = self.mats[mid]
            if n > 2048:
                continue
            Ah = np.ascontiguousarray(A.double().cpu().numpy())
            L = oracle.cdpp_factor(Ah, 64, 1e-4)
            t0 = time.perf_counter()
            r = oracle.run(Ah, np.ascontiguousarray(B[:, 0]), L, 64, cd=True, lam=1e-4, tol=1e-8,
                           max_iters=2000000, seed=seed, sys=seed)
            t_used += time.perf_counter() - t0
            cols += 1
            assert r.rel_res_true <= 1e-8
            if t_used > budget_s:
                break
        mean_k = statistics.mean(k for (_, _, k, _) in self.reqs)
        v = cols / t_used / mean_k
        return {"value": v, "unit": self.unit, "cores": 1, "kind": "oracle",
                "sample": f"{cols} single-column FP64 oracle CD++ solves to 1e-8 of the first requests with "
                          f"n <= 2048 ({t_used:.1f} s, one host thread); value = columns/s / mean k ({mean_k:.1f})"}


def make_workload(args):
    if args.workload in ("cdpp4096", "kpp2000"):
        return SingleFP64(args.workload, grid_tune=getattr(args, "grid_tune", False))
    if args.workload == "mixed262144":
        return MixedLS(args.storage, args.noisy, m=args.mixed_rows)
    if args.workload == "batched64":
        return Batched(nsys=getattr(args, "systems", 64), grid=getattr(args, "batched_grid", None),
                       tune_s=getattr(args, "tune_s", False))
    if args.workload == "serving":
        return Serving(n_req=args.requests)
    if args.workload == "cdpp4096-rht":
        return RhtSPD()
    if args.workload == "kpp-lsqr":
        return LsqrLS()
    if args.workload == "cdpp4096-memo":
        return MemoSPD()
    if args.workload in ("cdpp4096-f32", "cdpp4096-bf16"):
        return MixedSPD(args.workload.split("-")[1])
    raise SystemExit(f"unknown workload {args.workload}")


# ---------------------------------------------------------------------------------------------
# Arms
# ---------------------------------------------------------------------------------------------

def aggregate_ranks(total_ms, total_units, dist=None, device="cuda"):
    """Whole-job numbers of a replicas run: the slowest rank's time and the units of all ranks."""
    if dist is None:
        return total_ms, total_units
    import torch
    t = torch.tensor([float(total_ms)], device=device, dtype=torch.float64)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    u = torch.tensor([float(total_units)], device=device, dtype=torch.float64)
    dist.all_reduce(u, op=dist.ReduceOp.SUM)
    return float(t.item()), int(u.item())


def run_reference(args, rank: int):
    """The FP64 CPU oracle on every host core, each step a bounded sample of the same workload (rank 0
    only; no GPU is touched).  A step runs one single-threaded oracle process per core, each on its own
    block sequence, started together; the step's time is the slowest process's."""
    if rank != 0:
        return
    wl = make_workload(args)
    if isinstance(wl, MixedLS):
        A, b = host_mixed_sample(wl.m, wl.n, wl.s, 16, wl.storage)
        s, cd, lam, seed, it0 = wl.s, False, wl.lam, 0, 16
        L = _factors_numpy_gram(A, s, lam)
        what = (f"FP64 oracle block iterations (s={s}, n={wl.n}) on a host-built {A.shape[0]}-row sample of the "
                f"workload (same recipe and scaling, {wl.storage.upper()}-rounded, widened to FP64)")
        dtype = wl.dtype
    elif type(wl) is SingleFP64:
        sy, cd = wl.sy, wl.cd
        A, b, s, lam, seed, it0 = sy.A, sy.b, sy.s, sy.lam, wl.seed, 256
        L = _oracle_factors(A, s, lam, cd)
        what = "FP64 oracle block iterations of the workload"
        dtype = "f64"
    else:
        print(json.dumps({"impl": "reference", "unavailable": "the oracle arm times the fixed-partition single-system "
                          "workloads (mixed262144, cdpp4096, kpp2000); the memo, LSQR, batched and serving "
                          "workloads report their oracle as cpu_baseline"}), flush=True)
        return
    v1, _, _ = _oracle_iter_rate(A, b, L, s, cd, lam, seed, 8.0, it0=it0)
    times, iters, cores, model = [], 0, 1, ""
    for i in range(args.warmup + args.steps):
        va, cores, model, ita, dta = _oracle_rate_all_cores(A, b, L, s, cd, lam, seed, v1, 8.0)
        if i >= args.warmup:
            times.append(dta)
            iters = ita
    v = cores * iters / statistics.mean(times)
    sample = (f"{cores} x {iters} {what} per step, one single-threaded oracle process per host core "
              "(factor phase excluded)")
    line = {"impl": "reference", "metric": METRIC, "value": v, "unit": "block-iters/s", "n_gpus": args.gpus,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": 1e3 * statistics.mean(times),
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": dtype, "data": "synthetic",
            "config": {"workload": wl.desc},
            "cpu_baseline": {"value": v, "unit": "block-iters/s", "cores": cores, "cpu_model": model,
                             "kind": "oracle", "sample": sample},
            "e2e": {"value": v, "unit": "block-iters/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=5)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--workload", default="mixed262144",
                    choices=["cdpp4096", "kpp2000", "mixed262144", "batched64", "serving", "cdpp4096-f32",
                             "cdpp4096-bf16", "cdpp4096-rht", "cdpp4096-memo", "kpp-lsqr"])
    ap.add_argument("--storage", default="bf16", choices=["bf16", "f32"], help="mixed262144 storage type")
    ap.add_argument("--noisy", action="store_true", help="mixed262144: b = A x* + 1e-6 N(0,I)")
    ap.add_argument("--mixed-rows", type=int, default=262144,
                    help="mixed262144: rows of the system (a smaller one for profiler captures)")
    ap.add_argument("--requests", type=int, default=1024, help="serving: requests per step")
    ap.add_argument("--grid-tune", action="store_true",
                    help="cdpp4096 / kpp2000: let the launch autotuner pick the CTAs per system")
    ap.add_argument("--systems", type=int, default=64, help="batched64: systems (fewer for profiler captures)")
    ap.add_argument("--batched-grid", type=int, default=None, help="batched64: CTAs per system (default: autotuned)")
    ap.add_argument("--tune-s", action="store_true",
                    help="batched64: choose the block size among 128, 256, 512 with the block-size autotuner")
    ap.add_argument("--host-qr", action="store_true",
                    help="Haar factors by a host QR (ncu cannot load torch's device linear algebra)")
    ap.add_argument("--ref-iters", type=int, default=4096)
    ap.add_argument("--cpu-budget", type=float, default=20.0)
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-e2e", action="store_true")
    ap.add_argument("--no-cg-reference", action="store_true",
                    help="cdpp4096: skip the plain CG reference point after the timed steps (e.g. for ncu)")
    ap.add_argument("--no-fp64-reference", action="store_true",
                    help="mixed262144: skip the plain FP64 K++ solve of the same system after the timed steps")
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

    W.HOST_QR = args.host_qr
    wl = make_workload(args)
    wl.run_cg_reference = not args.no_cg_reference
    wl.run_fp64_reference = not args.no_fp64_reference
    wl.setup(kpp, torch, rank)
    stream = torch.cuda.current_stream()
    flush = torch.empty(512 << 20, dtype=torch.uint8, device="cuda")

    _log(f"{args.workload}: set up")
    for _ in range(args.warmup):
        wl.step()
    torch.cuda.synchronize()
    _log(f"{args.workload}: {args.warmup} warm-up steps done")
    step_ms, steps = [], []
    with ClockSampler(local) as clk:
        if dist:
            dist.barrier()
        torch.cuda.synchronize()
        n0 = kpp.launch_count()
        for _ in range(args.steps):
            flush.zero_()
            e0 = torch.cuda.Event(enable_timing=True)
            e1 = torch.cuda.Event(enable_timing=True)
            e0.record(stream)
            st = wl.step()
            e1.record(stream)
            e1.synchronize()
            step_ms.append(e0.elapsed_time(e1))
            steps.append(st)
        torch.cuda.synchronize()
        launches = kpp.launch_count() - n0
        if dist:
            dist.barrier()
    assert all(st["ok"] for st in steps), steps
    total_ms, total_units = aggregate_ranks(sum(step_ms), sum(st["units"] for st in steps), dist)
    value = total_units / (total_ms / 1e3)
    peaks = _peaks()

    line = {"metric": wl.metric, "value": value, "unit": wl.unit, "n_gpus": world, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": total_ms / args.steps, "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": wl.dtype, "data": "synthetic",
            "config": {"workload": wl.desc, "parallelism": f"replicas x{world}",
                       "l2": "flushed between steps (512 MiB write, outside the step events)",
                       "step": "the whole request stream through the server" if isinstance(wl, Serving)
                       else "factor phase + solve to 1e-8 + FP64 residual confirmation"},
            "time_to_tol_ms": statistics.mean(step_ms), "gpu_launches": launches,
            "roofline": wl.roofline(steps, peaks), "clocks": clk.summary()}
    if "iters" in steps[-1]:
        line["iters_to_tol"] = statistics.mean(st["iters"] for st in steps)
    if "kernel_ms" in steps[-1]:
        line["solve_kernel_ms"] = statistics.mean(st["kernel_ms"] for st in steps)
    if "rel_res" in steps[-1]:
        line["rel_res_true"] = steps[-1]["rel_res"]
    line.update(wl.extra(steps))
    if rank == 0 and not args.no_e2e:
        e = wl.e2e()
        if e:
            line["e2e"] = e
    if rank == 0 and not args.no_cpu_baseline:
        cb = wl.cpu_baseline(args.cpu_budget)
        if cb:
            line["cpu_baseline"] = cb
    if rank == 0:
        print(json.dumps(line), flush=True)
    if dist:
        dist.destroy_process_group()


if __name__ == "__main__":
    main()
