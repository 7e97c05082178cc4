"""Benchmark of the FS-1 hot path on GB300.

Workload (one "step"): a batch of 256 independent 1D pairs, N = 2^20 grid points
each (h = 2^-20), eps = 1e-4, 3-component Gaussian-mixture histograms with a
1e-6 floor, stabilised FP32 iteration with FP64 reductions, run to a marginal
L1 error of 1e-6 or 5000 iterations.  Every step solves the whole batch through
the library's C ABI (fs1_solve_batch).

Metric: N*iterations per second (sum over pairs of N * iterations / wall time).

Arms
  default               the CUDA library, inputs resident in HBM (value), plus an
                        end-to-end pass from pinned host buffers (e2e).
  --impl reference      the CPU FP64 oracle (the paper's sequential FS-1
                        recurrences in plain C) on the host cores, on a bounded
                        sample of the same workload.

Multi-GPU (torchrun): pairs are independent, so every rank solves its own batch
of 256 pairs (weak scaling); the only collective is the barrier and max-reduce
of the timing.
"""
from __future__ import annotations

import argparse
import concurrent.futures as cf
import json
import math
import os
import signal
import statistics
import subprocess
import sys
import tempfile
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

from paper_2202_10042_gb300 import inputs  # noqa: E402

WORKLOAD = dict(name="fs1_1d_log_fp32_batch256_n2^20_eps1e-4", n=1 << 20, pairs=256, eps=1e-4,
                tol=1e-6, itr_max=5000)
METRIC = "N*iters/s"
BYTES_PER_NIT = 28.0  # algorithmic HBM bytes per N*iteration of a streaming realisation


# ---------------------------------------------------------------------------
# distributed helpers (host logic; covered by CPU gloo tests)
# ---------------------------------------------------------------------------

def dist_env():
    rank = int(os.environ.get("RANK", "0"))
    world = int(os.environ.get("WORLD_SIZE", "1"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return rank, world, local


def shard_pairs(pairs_per_rank: int, rank: int) -> list:
    """Weak scaling: rank r solves its own pairs r*P .. r*P + P - 1."""
    return list(range(rank * pairs_per_rank, (rank + 1) * pairs_per_rank))


def reduce_max(x: float, world: int, device=None) -> float:
    if world <= 1:
        return x
    import torch
    import torch.distributed as dist
    t = torch.tensor([x], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def reduce_sum(x: float, world: int, device=None) -> float:
    if world <= 1:
        return x
    import torch
    import torch.distributed as dist
    t = torch.tensor([x], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.SUM)
    return float(t.item())


def barrier(world: int) -> None:
    if world > 1:
        import torch.distributed as dist
        dist.barrier()


# ---------------------------------------------------------------------------
# clocks sampling during the timed region
# ---------------------------------------------------------------------------

class Clocks:
    QUERY = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
             "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
             "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_index: int):
        self.gpu = gpu_index
        self.proc = None
        self.path = None

    def __enter__(self):
        fd, self.path = tempfile.mkstemp(prefix="fs1_clocks_", suffix=".csv")
        os.close(fd)
        try:
            self.proc = subprocess.Popen(["nvidia-smi", f"--query-gpu={self.QUERY}", "--format=csv,noheader,nounits",
                                          "-i", str(self.gpu), "-lms", "200", "-f", self.path],
                                         stdout=subprocess.DEVNULL, stderr=subprocess.DEVNULL)
        except FileNotFoundError:
            self.proc = None
        return self

    def __exit__(self, *exc):
        if self.proc is not None:
            self.proc.send_signal(signal.SIGTERM)
            try:
                self.proc.wait(timeout=5)
            except subprocess.TimeoutExpired:
                self.proc.kill()

    def summary(self):
        rows = []
        if self.path and os.path.exists(self.path):
            for line in open(self.path):
                parts = [p.strip() for p in line.split(",")]
                if len(parts) < 9:
                    continue
                try:
                    rows.append((float(parts[1]), float(parts[2]), parts[5:9]))
                except ValueError:
                    continue
            os.unlink(self.path)
        if not rows:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["unsampled"], "samples": 0}
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        reasons = set()
        for _, _, flags in rows:
            for nm, fl in zip(names, flags):
                if fl.lower() == "active":
                    reasons.add(nm)
        return {"sm_mhz": statistics.median(r[0] for r in rows), "sm_max_mhz": max(r[1] for r in rows),
                "reasons": sorted(reasons), "samples": len(rows)}


# ---------------------------------------------------------------------------
# workload construction
# ---------------------------------------------------------------------------

def make_pairs(indices, n, eps, tol, itr_max, workers=16):
    def one(i):
        p = inputs.workload2(i, n=n, eps=eps, tol=tol, itr_max=itr_max)
        return p.a.astype(np.float32), p.b.astype(np.float32)
    with cf.ThreadPoolExecutor(max_workers=workers) as ex:
        return list(ex.map(one, indices))


def host_cores() -> int:
    try:
        return len(os.sched_getaffinity(0))
    except AttributeError:
        return os.cpu_count() or 1


# ---------------------------------------------------------------------------
# the oracle arm (CPU)
# ---------------------------------------------------------------------------

def oracle_sample(n, eps, pairs_idx, iters, workers):
    """Time the CPU FP64 oracle (stabilised sequential FS-1 in C) on a sample:
    len(pairs_idx) pairs x `iters` iterations, one pair per host thread."""
    from oracle import cref
    cref.build()
    data = [inputs.workload2(i, n=n, eps=eps) for i in pairs_idx]
    t0 = time.perf_counter()
    res = cref.solve_many([(p.a, p.b, p.h[0], p.eps, 0.0, iters) for p in data], workers=workers)
    dt = time.perf_counter() - t0
    nit = sum(p.a.size * r.iters for p, r in zip(data, res))
    return nit / dt, dt, nit


def run_reference(args):
    rank, world, _ = dist_env()
    if rank != 0:
        return 0
    cores = host_cores()
    npairs = max(1, min(8, cores))
    iters = 40
    W = WORKLOAD
    for _ in range(args.warmup):
        oracle_sample(W["n"], W["eps"], list(range(npairs)), 5, npairs)
    vals, t_tot, nit_tot = [], 0.0, 0
    for _ in range(args.steps):
        v, dt, nit = oracle_sample(W["n"], W["eps"], list(range(npairs)), iters, npairs)
        vals.append(v)
        t_tot += dt
        nit_tot += nit
    value = nit_tot / t_tot
    sample = f"{npairs} pairs of the workload x {iters} iterations per step (FP64, tol=0)"
    line = {"impl": "reference", "metric": METRIC, "value": value, "unit": "N*iters/s",
            "n_gpus": args.gpus, "steps": args.steps, "warmup": args.warmup,
            "ms_per_step": 1000.0 * t_tot / args.steps, "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
            "config": {"workload": W["name"], "n": W["n"], "pairs": W["pairs"], "eps": W["eps"],
                       "tol": W["tol"], "itr_max": W["itr_max"], "parallelism": "host threads"},
            "cpu_baseline": {"value": value, "unit": "N*iters/s", "cores": npairs, "kind": "oracle",
                             "sample": sample},
            "e2e": {"value": value, "unit": "N*iters/s", "h2d_bytes_per_step": 0,
                    "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)
    return 0


# ---------------------------------------------------------------------------
# the CUDA arm
# ---------------------------------------------------------------------------

def run_gpu(args):
    import torch
    rank, world, local = dist_env()
    if world > 1:
        import torch.distributed as dist
        torch.cuda.set_device(local)
        dist.init_process_group("nccl", device_id=torch.device("cuda", local))
    dev = torch.device("cuda", local if world > 1 else 0)
    torch.cuda.set_device(dev)

    import __graft_entry__
    __graft_entry__.build()
    from paper_2202_10042_gb300 import fs1

    W = dict(WORKLOAD)
    if args.pairs:
        W["pairs"] = args.pairs
    if args.itr_max is not None:
        W["itr_max"] = args.itr_max
    idx = shard_pairs(W["pairs"], rank)
    host = make_pairs(idx, W["n"], W["eps"], W["tol"], W["itr_max"])
    h = 1.0 / W["n"]
    stream = torch.cuda.current_stream(dev)
    solver = fs1.Solver("log", "fp32", stream=stream.cuda_stream, team_size=args.team_size,
                        autotune=not args.no_autotune, use_graph=not args.no_graph)

    # device-resident inputs
    dev_t = [(torch.from_numpy(a).to(dev), torch.from_numpy(b).to(dev)) for a, b in host]
    probs = [fs1.Solver.problem(a, b, h, W["eps"], W["tol"], W["itr_max"]) for a, b in dev_t]
    # pinned host inputs for the end-to-end pass
    pin_t = [(torch.from_numpy(a).pin_memory(), torch.from_numpy(b).pin_memory()) for a, b in host]
    probs_h = [fs1.Solver.problem(a, b, h, W["eps"], W["tol"], W["itr_max"]) for a, b in pin_t]
    torch.cuda.synchronize()

    def step(ps):
        st, w, infos = solver.solve(ps)
        bad = [fs1.STATUS_NAMES.get(i.status) for i in infos
               if i.status not in (fs1.FS1_OK, fs1.FS1_ENOTCONV)]
        if bad:
            raise RuntimeError(f"solve failed: {bad[:4]}")
        return w, infos

    for _ in range(args.warmup):
        step(probs)

    # ---- timed region: device-resident inputs
    barrier(world)
    torch.cuda.synchronize()
    l0 = fs1.fs1_launch_count()
    ev0, ev1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    nit = 0
    kern_ms = []
    with Clocks(dev.index if dev.index is not None else 0) as clk:
        ev0.record(stream)
        for _ in range(args.steps):
            w, infos = step(probs)
            nit += sum(int(p.n[0]) * int(i.iters) for p, i in zip(probs, infos))
            kern_ms.append(infos[0].ms)
        ev1.record(stream)
        torch.cuda.synchronize()
    launches = fs1.fs1_launch_count() - l0
    barrier(world)
    ms = ev0.elapsed_time(ev1)
    ms_max = reduce_max(ms, world, dev)
    nit_all = reduce_sum(float(nit), world, dev)
    value = nit_all / (ms_max / 1000.0)
    iters = [int(i.iters) for i in infos]
    errs = [float(i.marginal_err) for i in infos]
    kernel_ms = statistics.mean(kern_ms)
    nit_step = nit / args.steps

    # ---- end to end: pinned host buffers, H2D + solve + D2H each step
    barrier(world)
    torch.cuda.synchronize()
    e_steps = max(1, min(args.steps, args.e2e_steps))
    t0 = time.perf_counter()
    e_nit = 0
    for _ in range(e_steps):
        w, infos = step(probs_h)
        e_nit += sum(int(p.n[0]) * int(i.iters) for p, i in zip(probs_h, infos))
    torch.cuda.synchronize()
    e_s = reduce_max(time.perf_counter() - t0, world, dev)
    e_val = reduce_sum(float(e_nit), world, dev) / e_s
    h2d = sum(a.numel() * a.element_size() + b.numel() * b.element_size() for a, b in pin_t)
    d2h = len(probs_h) * (32 + 24)  # per-pair result record + mass-check record

    achieved = BYTES_PER_NIT * nit_step / (kernel_ms / 1000.0) / 1e9
    peaks = {}
    try:
        peaks = json.load(open(os.path.join(ROOT, "MEASURED_PEAKS.json")))
    except (OSError, ValueError):
        pass
    peak = peaks.get("hbm_gbs", 6800.0)
    peak_src = "measured" if "hbm_gbs" in peaks else "fallback"
    traffic = None
    tr_path = os.path.join(ROOT, "profiles", "traffic.json")
    if os.path.exists(tr_path):
        try:
            tr = json.load(open(tr_path))
            if tr.get("workload") == W["name"] and tr.get("kernel_rev") == kernel_revision():
                traffic = tr.get("bytes_per_launch")
        except (OSError, ValueError):
            pass

    cpu = None
    if rank == 0 and world == 1 and not args.no_cpu:
        cores = host_cores()
        npairs = max(1, min(8, cores))
        v, dt, onit = oracle_sample(W["n"], W["eps"], list(range(npairs)), args.cpu_iters, npairs)
        cpu = {"value": v, "unit": "N*iters/s", "cores": npairs, "kind": "oracle",
               "sample": f"{npairs} pairs of the workload x {args.cpu_iters} iterations "
                         f"(FP64 stabilised sequential FS-1, one pair per thread), {dt:.1f} s"}

    if rank == 0:
        line = {"metric": METRIC, "value": value, "unit": "N*iters/s", "n_gpus": world,
                "steps": args.steps, "warmup": args.warmup, "ms_per_step": ms_max / args.steps,
                "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f32",
                "data": "synthetic",
                "config": {"workload": W["name"], "n": W["n"], "pairs": len(idx), "eps": W["eps"],
                           "tol": W["tol"], "itr_max": W["itr_max"], "parallelism": f"dp{world} (pairs)",
                           "l2": "inputs larger than L2 (%.1f GB per step)" % (h2d / 1e9),
                           "team_size": int(infos[0].team_size),
                           "launch": "graph replay" if solver.stats()["graph_replays"] else "direct",
                           "iters_min": min(iters), "iters_max": max(iters),
                           "err_median": statistics.median(errs)},
                "roofline": {"bound": "hbm", "achieved": achieved, "peak": peak, "unit": "GB/s",
                             "frac": achieved / peak, "traffic": traffic,
                             "peak_source": peak_src,
                             "note": "achieved = 28 B per N*iteration (streaming-equivalent bytes) "
                                     "/ team-kernel time; the kernel keeps state on chip"},
                "e2e": {"value": e_val, "unit": "N*iters/s", "h2d_bytes_per_step": h2d,
                        "d2h_bytes_per_step": d2h},
                "gpu_launches": launches,
                "clocks": clk.summary(),
                "cpu_baseline": cpu}
        print(json.dumps(line), flush=True)
    solver.close()
    if world > 1:
        import torch.distributed as dist
        dist.destroy_process_group()
    return 0


def kernel_revision() -> str:
    import hashlib
    h = hashlib.sha256()
    for f in sorted(os.listdir(os.path.join(ROOT, "paper_2202_10042_gb300", "csrc"))):
        h.update(open(os.path.join(ROOT, "paper_2202_10042_gb300", "csrc", f), "rb").read())
    return h.hexdigest()[:16]


def main(argv=None):
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=3)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="fs1", choices=["fs1", "reference"])
    ap.add_argument("--pairs", type=int, default=0, help="override pairs per rank (testing)")
    ap.add_argument("--itr-max", type=int, default=None, help="override the cap (testing)")
    ap.add_argument("--e2e-steps", type=int, default=1)
    ap.add_argument("--cpu-iters", type=int, default=300)
    ap.add_argument("--no-cpu", action="store_true")
    ap.add_argument("--team-size", type=int, default=0, help="CTAs per pair (0: autotuned)")
    ap.add_argument("--no-autotune", action="store_true", help="fixed team-size heuristic")
    ap.add_argument("--no-graph", action="store_true", help="direct launches instead of graph replay")
    args = ap.parse_args(argv)
    if args.impl == "reference":
        return run_reference(args)
    return run_gpu(args)


if __name__ == "__main__":
    sys.exit(main())
