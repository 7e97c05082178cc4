"""Benchmark of the FS-1 hot path on GB300.

Workloads (one "step" solves the whole batch through the library's C ABI,
fs1_solve_batch; --workload picks one, 2 is the default and the headline):
  1  one 1D pair, N = 1000 (h = 1e-3), eps = 1e-2, 2-component Gaussian
     mixtures + 1e-4 floor, plain FS-1 (Algorithm 1 as written) in FP64,
     1000 iterations
  2  256 1D pairs, N = 2^20 (h = 2^-20), eps = 1e-4, 3-component Gaussian
     mixtures + 1e-6 floor, stabilised FP32 iteration with FP64 reductions,
     marginal L1 error 1e-6 or 5000 iterations
  3  4096 uneven 1D pairs, N log-uniform in [256, 65536], eps log-uniform in
     [1e-3, 1e-1], Dirichlet(1) weights smoothed by a width-5 box + 1e-6
     floor, stabilised FP32, one persistent launch
  4  64 2D pairs on a 512 x 512 grid (h = 1/512), eps = 1e-3, images of 1-5
     anisotropic Gaussian blobs + 1e-7 floor, stabilised FP32 (Algorithm 2)
  6  replay of the paper's Section 5.1 (Table 1): 100 pairs of U[0, 1]
     histograms on [-3, 3], N = 8000, eps = 1e-3, 1000 iterations
  7  replay of Section 5.2 (Table 2): the Ricker pair, N = 8000, eps = 1e-2,
     500 iterations, 100 repeats
  8  replay of Section 5.3 (Table 3): 64 pairs of 160 x 160 U[0, 1] images,
     h = 1, eps = 1e-2, 1000 iterations
  9  32 3D grids of 64^3 cells, eps = 2e-3, 1-3 Gaussian blobs + 1e-7 floor,
     stabilised FP32, marginal error 1e-6 or 2000 iterations
  10 the Remarks' tau-triggered stabilised form as written (FP64) on the
     Section 5.2 Ricker pair at N = 2000, eps = 5e-4 (where the plain FP64
     iteration overflows), 500 iterations, 100 repeats
For 6-8 vs_baseline is the ratio to the FS-1 rate the paper's tables imply on
its CPU (context: another machine).
The serving workload is measured by `python -m paper_2202_10042_gb300.serve`.

Metric: N*iterations per second (sum over pairs of grid points x iterations /
device time of the steps).

Arms
  default               the CUDA library, inputs resident in HBM (value), plus an
                        end-to-end pass from pinned host buffers (e2e), and the
                        same pairs solved one fs1_w1 call each on a sample
                        (one_pair_per_launch).
  --impl reference      the CPU FP64 oracle (the paper's sequential FS-1
                        recurrences in plain C) on the host cores, on a bounded
                        sample of the same workload.

Multi-GPU (torchrun): pairs are independent, so every rank solves its own batch
(weak scaling); the only collectives are the barrier and the max / sum reduce
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

METRIC = "N*iters/s"
L2_BYTES = 129 << 20

# Streaming-equivalent HBM bytes per N*iteration: what a realisation that
# streams the state through HBM would move.  FP32: the v-half reads u, b and
# the accepted v and writes v (16 B), the u-half reads v, a and writes u
# (12 B); FP64 doubles it.  2D counts the same 28 B per point (a two-pass
# realisation also writes and reads the fast-axis partial sums, 44 B).
WORKLOADS = {
    1: dict(name="fs1_1d_plain_fp64_n1000_eps1e-2_it1000", pairs=1, variant="plain", precision="fp64",
            dtype="f64", bytes_per_nit=56.0, kw={}, sample_iters=1000, solo=0),
    2: dict(name="fs1_1d_log_fp32_batch256_n2^20_eps1e-4", pairs=256, variant="log", precision="fp32",
            dtype="f32", bytes_per_nit=28.0, kw=dict(n=1 << 20, eps=1e-4, tol=1e-6, itr_max=5000),
            sample_iters=300, solo=8),
    3: dict(name="fs1_1d_log_fp32_uneven4096_n256-65536", pairs=4096, variant="log", precision="fp32",
            dtype="f32", bytes_per_nit=28.0, kw={}, sample_iters=200, solo=64),
    4: dict(name="fs1_2d_log_fp32_batch64_512x512_eps1e-3", pairs=64, variant="log", precision="fp32",
            dtype="f32", bytes_per_nit=28.0, kw={}, sample_iters=40, solo=4),
    # replays of the paper's Section 5 experiments; `paper` is the FS-1 rate its
    # tables imply on its CPU (grid points x iterations / printed time)
    6: dict(name="paper_e1_1d_random_n8000_eps1e-3_it1000", pairs=100, variant="log", precision="fp32",
            dtype="f32", bytes_per_nit=28.0, kw={}, sample_iters=1000, solo=8,
            paper=8000 * 1000 / 1.53e-1),
    7: dict(name="paper_e2_ricker_n8000_eps1e-2_it500", pairs=100, variant="log", precision="fp32",
            dtype="f32", bytes_per_nit=28.0, kw={}, sample_iters=500, solo=8,
            paper=8000 * 500 / 5.96e-2),
    8: dict(name="paper_e3_2d_random_160x160_h1_eps1e-2_it1000", pairs=64, variant="log", precision="fp32",
            dtype="f32", bytes_per_nit=28.0, kw={}, sample_iters=200, solo=4,
            paper=160 * 160 * 1000 / 1.08),
    9: dict(name="fs1_3d_log_fp32_batch32_64^3_eps2e-3", pairs=32, variant="log", precision="fp32",
            dtype="f32", bytes_per_nit=28.0, kw={}, sample_iters=20, solo=2),
    10: dict(name="paper_form_fp64_ricker_n2000_eps5e-4_it500", pairs=100, variant="paper", precision="fp64",
             dtype="f64", bytes_per_nit=56.0, kw=dict(n=2000, eps=5e-4, itr_max=500),
             sample_iters=500, solo=4),
    # pairs beyond the on-chip capacity: the state in device memory
    11: dict(name="fs1_1d_log_fp32_stream4_n2^23_eps1e-5_it500", pairs=4, variant="log", precision="fp32",
             dtype="f32", bytes_per_nit=28.0, kw=dict(n=1 << 23, eps=1e-5, tol=1e-6, itr_max=500),
             sample_iters=20, solo=0),
}

GENERATORS = {1: inputs.workload1, 2: inputs.workload2, 3: inputs.workload3, 4: inputs.workload4,
              6: inputs.paper_e1, 7: inputs.paper_e2, 8: inputs.paper_e3, 9: inputs.workload9,
              10: inputs.paper_e2, 11: inputs.workload2}


def gen_problem(workload: int, index: int, **over):
    W = WORKLOADS[workload]
    kw = dict(W["kw"])
    kw.update({k: v for k, v in over.items() if v is not None})
    return GENERATORS[workload](index, **kw)


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

def make_problems(workload, indices, itr_max=None, workers=16, **over):
    with cf.ThreadPoolExecutor(max_workers=workers) as ex:
        return list(ex.map(lambda i: gen_problem(workload, i, itr_max=itr_max, **over), indices))


def host_cores() -> int:
    try:
        return len(os.sched_getaffinity(0))
    except AttributeError:
        return os.cpu_count() or 1


# ---------------------------------------------------------------------------
# the oracle arm (CPU)
# ---------------------------------------------------------------------------

def solve_ms(problems, infos) -> float:
    """Solve-kernel time of one call (ms) from its per-problem infos: problems of
    one team or grid launch share that launch's time, and the 1D pairs streamed
    through device memory (team size 0) share the time of their solves, which
    run after the launches of the others."""
    streamed = [float(i.ms) for p, i in zip(problems, infos) if p.ndim == 1 and int(i.team_size) == 0]
    shared = [float(i.ms) for p, i in zip(problems, infos) if not (p.ndim == 1 and int(i.team_size) == 0)]
    return (max(shared) if shared else 0.0) + (max(streamed) if streamed else 0.0)


def oracle_sample(workload, pairs_idx, iters, workers):
    """Time the CPU FP64 oracle (sequential FS-1 in C: the plain form for the
    plain workload, the stabilised one otherwise) on a sample: the given pairs
    x `iters` iterations with tol = 0, one pair per host thread."""
    from oracle import cref
    cref.build()
    W = WORKLOADS[workload]
    data = [gen_problem(workload, i) for i in pairs_idx]
    tau = math.inf if W["variant"] == "plain" else 1e10
    t0 = time.perf_counter()
    res = cref.solve_many([(p.a, p.b, p.h if p.ndim >= 2 else p.h[0], p.eps, 0.0, iters) for p in data],
                          workers=workers, tau=tau)
    dt = time.perf_counter() - t0
    nit = sum(p.a.size * r.iters for p, r in zip(data, res))
    return nit / dt, dt, nit


def cpu_sample_threads(W, cores: int) -> int:
    """Host threads of the oracle sample: one pair per thread on every core the
    process may run on (os.sched_getaffinity), at most one per pair of the
    workload."""
    return max(1, min(W["pairs"], cores))


def cpu_sample_desc(W, npairs, iters, dt=None):
    what = f"{npairs} pair(s) of the workload x {iters} iterations (FP64 " + \
        ("plain" if W["variant"] == "plain" else "stabilised") + " sequential FS-1, one pair per thread, tol=0)"
    return what + (f", {dt:.1f} s" if dt is not None else "")


def run_reference(args):
    rank, world, _ = dist_env()
    if rank != 0:
        return 0
    W = WORKLOADS[args.workload]
    cores = host_cores()
    npairs = cpu_sample_threads(W, cores)
    iters = max(1, W["sample_iters"] // 4)
    for _ in range(args.warmup):
        oracle_sample(args.workload, list(range(npairs)), max(1, iters // 8), npairs)
    t_tot, nit_tot = 0.0, 0
    for _ in range(args.steps):
        v, dt, nit = oracle_sample(args.workload, list(range(npairs)), iters, npairs)
        t_tot += dt
        nit_tot += nit
    value = nit_tot / t_tot
    line = {"impl": "reference", "metric": METRIC, "value": value, "unit": "N*iters/s",
            "n_gpus": args.gpus, "steps": args.steps, "warmup": args.warmup,
            "ms_per_step": 1000.0 * t_tot / args.steps, "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
            "config": {"workload": W["name"], "pairs": W["pairs"], "parallelism": "host threads"},
            "cpu_baseline": {"value": value, "unit": "N*iters/s", "cores": npairs, "host_cores": cores,
                             "kind": "oracle",
                             "sample": cpu_sample_desc(W, npairs, iters) + " per step"},
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

    W = WORKLOADS[args.workload]
    npairs = args.pairs or W["pairs"]
    idx = shard_pairs(npairs, rank)
    over = {"side": args.side, "eps": args.eps} if args.workload == 4 else {}
    host = make_problems(args.workload, idx, itr_max=args.itr_max, **over)
    tdt = torch.float64 if W["precision"] == "fp64" else torch.float32
    stream = torch.cuda.current_stream(dev)
    solver = fs1.Solver(W["variant"], W["precision"], stream=stream.cuda_stream, team_size=args.team_size,
                        autotune=not args.no_autotune, use_graph=not args.no_graph, grid2d=args.grid2d)

    def hgrid(p):
        return tuple(p.h) if p.ndim >= 2 else p.h[0]

    # device-resident inputs
    dev_t = [(torch.from_numpy(p.a).to(dev, tdt), torch.from_numpy(p.b).to(dev, tdt)) for p in host]
    probs = [fs1.Solver.problem(a, b, hgrid(p), p.eps, p.tol, p.itr_max) for p, (a, b) in zip(host, dev_t)]
    # pinned host inputs for the end-to-end pass
    pin_t = [(torch.from_numpy(p.a).to(tdt).pin_memory(), torch.from_numpy(p.b).to(tdt).pin_memory())
             for p in host]
    probs_h = [fs1.Solver.problem(a, b, hgrid(p), p.eps, p.tol, p.itr_max) for p, (a, b) in zip(host, pin_t)]
    in_bytes = sum(a.numel() * a.element_size() + b.numel() * b.element_size() for a, b in dev_t)
    flush = torch.empty(2 * L2_BYTES // 4, dtype=torch.float32, device=dev) if in_bytes < 2 * L2_BYTES else None
    torch.cuda.synchronize()

    def check(infos):
        bad = [fs1.STATUS_NAMES.get(i.status) for i in infos if i.status not in (fs1.FS1_OK, fs1.FS1_ENOTCONV)]
        if bad:
            raise RuntimeError(f"solve failed: {bad[:4]}")

    def step(ps):
        st, w, infos = solver.solve(ps)
        check(infos)
        return w, infos

    def nit_of(infos):
        return sum(int(p.a.size) * int(i.iters) for p, i in zip(host, infos))

    for _ in range(args.warmup):
        step(probs)

    # ---- timed region: device-resident inputs; each step between its own
    # events on the launching stream, the L2 flush (small inputs) outside them
    barrier(world)
    torch.cuda.synchronize()
    l0 = fs1.fs1_launch_count()
    evs = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)) for _ in range(args.steps)]
    nit = 0
    kern_ms = []
    with Clocks(dev.index if dev.index is not None else 0) as clk:
        for e0, e1 in evs:
            if flush is not None:
                flush.fill_(1.0)
            e0.record(stream)
            w, infos = step(probs)
            e1.record(stream)
            nit += nit_of(infos)
            kern_ms.append(solve_ms(host, infos))
        torch.cuda.synchronize()
    launches = fs1.fs1_launch_count() - l0
    barrier(world)
    ms = sum(e0.elapsed_time(e1) for e0, e1 in evs)
    ms_max = reduce_max(ms, world, dev)
    nit_all = reduce_sum(float(nit), world, dev)
    value = nit_all / (ms_max / 1000.0)
    iters = [int(i.iters) for i in infos]
    errs = [float(i.marginal_err) for i in infos]
    teams = sorted({int(i.team_size) for i in infos})
    kernel_ms = statistics.mean(kern_ms)
    nit_step = nit / args.steps
    st_h = solver.stats()
    graph = st_h["graph_replays"] > 0
    # the team kernel's instantiation of the timed launches (1D): exact E, or generic
    kernel_inst = None
    if host[0].ndim == 1 and W["variant"] != "paper":
        if all(int(i.team_size) == 0 for i in infos):
            kernel_inst = "streaming (state in device memory)"
        elif st_h["last_exact_E"] > 0:
            kernel_inst = f"exact, {st_h['last_exact_E']} points per thread"
        else:
            kernel_inst = "generic"

    # ---- end to end: pinned host buffers, H2D + solve + D2H each step, over
    # as many steps as the device-timed region, after one untimed pass that
    # sizes the staging buffers
    step(probs_h)
    barrier(world)
    torch.cuda.synchronize()
    e_steps = args.e2e_steps if args.e2e_steps > 0 else args.steps
    t0 = time.perf_counter()
    e_nit = 0
    for _ in range(e_steps):
        w_h, infos_h = step(probs_h)
        e_nit += nit_of(infos_h)
    torch.cuda.synchronize()
    e_s = reduce_max(time.perf_counter() - t0, world, dev)
    e_val = reduce_sum(float(e_nit), world, dev) / e_s
    h2d = sum(a.numel() * a.element_size() + b.numel() * b.element_size() for a, b in pin_t)
    d2h = len(probs_h) * 32   # one result record per pair

    # ---- the same pairs one fs1_w1 call each (sample), for comparison
    solo = None
    if W["solo"] and not args.no_solo:
        k = min(W["solo"], len(probs))
        s_nit, t0 = 0, time.perf_counter()
        for p, q in zip(host[:k], probs[:k]):
            st, w1, info = fs1.fs1_w1(solver.h, q)
            s_nit += int(p.a.size) * int(info.iters)
        solo_s = time.perf_counter() - t0
        solo = {"value": s_nit / solo_s, "unit": METRIC, "pairs": k,
                "note": "the first pairs of the batch solved one fs1_w1 call (one launch) each, wall clock"}

    achieved = W["bytes_per_nit"] * nit_step / (kernel_ms / 1000.0) / 1e9
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
        n_s = cpu_sample_threads(W, cores)
        v, dt, onit = oracle_sample(args.workload, list(range(n_s)), W["sample_iters"], n_s)
        cpu = {"value": v, "unit": METRIC, "cores": n_s, "host_cores": cores, "kind": "oracle",
               "sample": cpu_sample_desc(W, n_s, W["sample_iters"], dt)}

    if rank == 0:
        p0 = host[0]
        cfg = {"workload": W["name"], "pairs": len(idx), "variant": W["variant"], "precision": W["precision"],
               "parallelism": f"dp{world} (pairs)",
               "l2": ("inputs larger than L2 (%.2f GB per step)" % (in_bytes / 1e9)) if flush is None
               else "L2 flushed between steps (%.0f MB write)" % (flush.numel() * 4 / 1e6),
               "team_size": teams[0] if len(teams) == 1 else teams,
               "launch": "graph replay" if graph else "direct",
               **({"team_kernel": kernel_inst} if kernel_inst else {}),
               **({"kernel_2d": "grid kernel (fs1_config.grid2d = 1)"} if args.grid2d else {}),
               "iters_min": min(iters), "iters_max": max(iters), "err_median": statistics.median(errs)}
        if args.workload in (2, 11):
            cfg.update({"n": p0.a.size, "eps": p0.eps, "tol": p0.tol, "itr_max": p0.itr_max})
        if over and (args.side or args.eps):
            cfg["workload"] += " (overridden: side %d, eps %g)" % (p0.a.shape[0], p0.eps)
        line = {"metric": METRIC, "value": value, "unit": "N*iters/s", "n_gpus": world,
                "steps": args.steps, "warmup": args.warmup, "ms_per_step": ms_max / args.steps,
                "higher_is_better": True, "scaling": "weak",
                "vs_baseline": value / W["paper"] if "paper" in W else None, "dtype": W["dtype"],
                "data": "synthetic", "config": cfg,
                "roofline": {"bound": "hbm", "achieved": achieved, "peak": peak, "unit": "GB/s",
                             "frac": achieved / peak, "traffic": traffic, "peak_source": peak_src,
                             "note": "achieved = %.0f B per N*iteration (streaming-equivalent bytes) "
                                     "/ solve-kernel time; the kernel keeps state on chip" % W["bytes_per_nit"]},
                "e2e": {"value": e_val, "unit": "N*iters/s", "h2d_bytes_per_step": h2d,
                        "d2h_bytes_per_step": d2h, "steps": e_steps},
                "one_pair_per_launch": solo,
                "gpu_launches": launches,
                "clocks": clk.summary(),
                "cpu_baseline": cpu}
        print(json.dumps(line), flush=True)
    solver.close()
    if world > 1:
        import torch.distributed as dist
        dist.destroy_process_group()
    return 0


TEAM_KERNEL_SOURCES = ("fs1_team.cuh", "fs1_solve1d.cu", "fs1_team_exact_*.cu", "fs1_device.cuh",
                       "fs1_internal.h")


def kernel_revision() -> str:
    """Hash of the sources the 1D team kernel is built from: the recorded ncu
    traffic applies while it matches."""
    import glob
    import hashlib
    h = hashlib.sha256()
    for pat in TEAM_KERNEL_SOURCES:
        for f in sorted(glob.glob(os.path.join(ROOT, "paper_2202_10042_gb300", "csrc", pat))):
            h.update(open(f, "rb").read())
    return h.hexdigest()[:16]


def main(argv=None):
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--workload", type=int, default=2, choices=sorted(WORKLOADS))
    ap.add_argument("--no-solo", action="store_true", help="skip the one-pair-per-launch sample")
    ap.add_argument("--steps", type=int, default=3)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="fs1", choices=["fs1", "reference"])
    ap.add_argument("--pairs", type=int, default=0, help="override pairs per rank (testing)")
    ap.add_argument("--itr-max", type=int, default=None, help="override the cap (testing)")
    ap.add_argument("--e2e-steps", type=int, default=0, help="end-to-end steps (0: as many as --steps)")
    ap.add_argument("--no-cpu", action="store_true")
    ap.add_argument("--team-size", type=int, default=0, help="CTAs per pair (0: autotuned)")
    ap.add_argument("--no-autotune", action="store_true", help="fixed team-size heuristic")
    ap.add_argument("--no-graph", action="store_true", help="direct launches instead of graph replay")
    ap.add_argument("--side", type=int, default=None, help="workload 4: image side (default 512)")
    ap.add_argument("--eps", type=float, default=None, help="workload 4: eps (default 1e-3)")
    ap.add_argument("--grid2d", action="store_true",
                    help="2D images on the grid kernel (state in device memory) instead of the cluster kernel")
    args = ap.parse_args(argv)
    if args.impl == "reference":
        return run_reference(args)
    return run_gpu(args)


if __name__ == "__main__":
    sys.exit(main())
