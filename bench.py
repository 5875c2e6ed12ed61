"""Benchmark: Metropolis attempts/s of the inhomogeneous NMC sweep on one GB300.

Workload (default): random 4-SAT, N = 50,000 variables, M = 480,000 clauses (alpha 9.6),
1,024 multi-spin-coded replicas, 5,000 sweeps, per-variable beta geometric 0.3 -> 6.0 with a
seeded 20% subset at 0.4x for the first half, then ramped. One step = one whole anneal of
that workload: initial states, energies, 5,000 colour-ordered sweeps with best-so-far
tracking, and the readback of states / energies / best states into device buffers. The
instance and its schedule are resident in HBM before the timed region (their upload is what
the end-to-end number adds).

Prints one JSON line (rank 0). `--impl reference` times the CPU oracle on the host cores
instead, on a bounded sample of the same workload.
"""
from __future__ import annotations

import argparse
import json
import os
import statistics
import subprocess
import sys
import tempfile
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

import nmc_inputs as W  # noqa: E402

METRIC = "Metropolis attempts/s (4-SAT N=50k, 1024 replicas, inhomogeneous beta)"
UNIT = "attempts/s"


def peaks():
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as f:
            p = json.load(f)
        return float(p["hbm_gbs"]), "measured"
    except Exception:
        return 6800.0, "fallback"


def algorithmic_bytes_per_sweep(lits: np.ndarray, n_vars: int, replicas: int) -> int:
    """Bytes one sweep must move: for every attempt the (k-1) neighbour literals of each
    clause of the variable, one bit per replica (replica-private state), the variable's own
    state read and written, the occurrence lists (k int32 per occurrence) and the beta row."""
    used = (lits != 0).sum(axis=1)
    occ = int(used.sum())                          # sum of degrees
    nbr_bits = int((used * (used - 1)).sum())      # sum over occurrences of (k-1)
    words = (replicas + 31) // 32
    state = nbr_bits * words * 4 + 2 * n_vars * words * 4
    shared = occ * int(lits.shape[1]) * 4 + n_vars * 4
    return state + shared


class Clocks:
    """Samples nvidia-smi clocks and throttle reasons while the timed region runs."""

    Q = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
         "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
         "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_index: int):
        self.gpu = gpu_index
        self.proc = None
        self.path = None

    def start(self):
        fd, self.path = tempfile.mkstemp(suffix=".csv")
        os.close(fd)
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", f"--id={self.gpu}", f"--query-gpu={self.Q}",
                 "--format=csv,noheader,nounits", "-lms", "200"],
                stdout=open(self.path, "w"), stderr=subprocess.DEVNULL)
        except Exception:
            self.proc = None

    def stop(self):
        if self.proc is None:
            return None
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except Exception:
            self.proc.kill()
        rows = []
        for line in open(self.path):
            parts = [p.strip() for p in line.split(",")]
            if len(parts) >= 9:
                rows.append(parts)
        os.unlink(self.path)
        if not rows:
            return None
        sm = [float(r[1]) for r in rows if r[1].replace(".", "").isdigit()]
        smax = [float(r[2]) for r in rows if r[2].replace(".", "").isdigit()]
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        reasons = sorted({names[i] for r in rows for i in range(4) if r[5 + i] == "Active"})
        loaded = [s for s in sm if smax and s > 0.5 * max(smax)] or sm
        return {"sm_mhz": statistics.median(loaded) if loaded else None,
                "sm_max_mhz": max(smax) if smax else None, "reasons": reasons,
                "samples": len(rows)}


def dist_setup():
    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("gloo")
    return world, rank, local


def dist_max(x: float, world: int) -> float:
    """Max over ranks of a host float (timing only; no data-path collective)."""
    if world == 1:
        return x
    import torch
    import torch.distributed as dist
    t = torch.tensor([x], dtype=torch.float64)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def dist_barrier(world: int):
    if world > 1:
        import torch.distributed as dist
        dist.barrier()


def workload(args):
    wl = W.workload_ksat_large(n_steps=args.sweeps, n_vars=args.n_vars)
    wl["replicas"] = args.replicas
    return wl


def run_ours(args, world, rank, local):
    import torch

    import paper_2111_13628_gb300 as nmc

    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)
    wl = workload(args)
    lits, n, beta, R, T = wl["lits"], wl["n_vars"], wl["beta"], wl["replicas"], wl["n_steps"]
    attempts_per_step = n * R * T
    stream = torch.cuda.Stream(device=dev)
    ctx = nmc.Context(local, stream=stream)
    inst = ctx.load_ksat(lits, n)
    ctx.set_schedule(inst, beta)
    rs = ctx.replicas_create(inst, R, seed=wl["seed"])
    out = dict(states=torch.empty((R, n), dtype=torch.uint8, device=dev),
               energies=torch.empty(R, dtype=torch.int64, device=dev),
               best_energies=torch.empty(R, dtype=torch.int64, device=dev),
               best_states=torch.empty((R, n), dtype=torch.uint8, device=dev))
    flush = torch.empty(512 * 1024 * 1024 // 4, dtype=torch.float32, device=dev)  # > L2

    seed_base = 1000 * rank

    def step(i, ev=None):
        ctx.replicas_reset(rs, seed_base + i)
        if ev is not None:
            ev[0].record(stream)
        if args.path == "batch":
            ctx.batch_run([rs], 0, T)
        else:
            ctx.replicas_run(rs, 0, T)  # "run": library's choice; "grid": NMC_RUN_PATH=grid
        if ev is not None:
            ev[1].record(stream)
        ctx.replicas_read_device(rs, **out)

    for i in range(args.warmup):
        step(i)
        with torch.cuda.stream(stream):
            flush.zero_()
    ctx.sync()
    torch.cuda.synchronize()
    dist_barrier(world)

    clocks = Clocks(local)
    clocks.start()
    sweep_events = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True))
                    for _ in range(args.steps)]
    t_start = torch.cuda.Event(enable_timing=True)
    t_stop = torch.cuda.Event(enable_timing=True)
    torch.cuda.synchronize()
    dist_barrier(world)
    t_start.record(stream)
    for i in range(args.steps):
        step(args.warmup + i, sweep_events[i])
        with torch.cuda.stream(stream):
            flush.zero_()  # L2 flush between steps (512 MB written)
    t_stop.record(stream)
    ctx.sync()
    torch.cuda.synchronize()
    dist_barrier(world)
    clk = clocks.stop()
    total_ms = t_start.elapsed_time(t_stop)
    sweep_ms = [a.elapsed_time(b) for a, b in sweep_events]
    total_ms = dist_max(total_ms, world)
    ms_per_step = total_ms / args.steps
    value = world * attempts_per_step * args.steps / (total_ms / 1e3)

    # roofline of the dominant kernel (the persistent sweep kernel, one launch per step)
    peak, peak_kind = peaks()
    bytes_launch = algorithmic_bytes_per_sweep(lits, n, R) * T
    sweep_avg_s = statistics.mean(sweep_ms) / 1e3
    achieved = bytes_launch / sweep_avg_s / 1e9
    _, n_colours = ctx.ksat_colouring(inst)

    # end to end through the C ABI with host buffers: instance + schedule upload, anneal,
    # readback of states / best states / energies to the host
    e2e = None
    if args.e2e_steps > 0:
        lits_h = torch.from_numpy(lits).pin_memory()
        beta_h = torch.from_numpy(beta).pin_memory()
        host = dict(states=torch.empty((R, n), dtype=torch.uint8).pin_memory(),
                    energies=torch.empty(R, dtype=torch.int64).pin_memory(),
                    best_energies=torch.empty(R, dtype=torch.int64).pin_memory(),
                    best_states=torch.empty((R, n), dtype=torch.uint8).pin_memory())
        times = []
        for i in range(args.e2e_steps + 1):
            dist_barrier(world)
            t0 = time.perf_counter()
            ei = ctx.load_ksat(lits_h.numpy(), n)
            ctx.set_schedule(ei, beta_h.numpy())
            ctx.anneal(ei, R, 0, T, seed_base + 7 + i, out={k: v.numpy() for k, v in host.items()})
            ctx.unload(ei)
            dt = time.perf_counter() - t0
            if i > 0:  # the first pass warms the host allocator and pinned paths
                times.append(dist_max(dt, world))
        e2e_s = statistics.mean(times)
        h2d = lits.nbytes + beta.nbytes
        d2h = 2 * R * n + 2 * R * 8
        e2e = {"value": world * attempts_per_step / e2e_s, "unit": UNIT,
               "h2d_bytes_per_step": int(h2d), "d2h_bytes_per_step": int(d2h),
               "s_per_step": e2e_s, "steps": len(times),
               "path": "nmc_load_ksat + nmc_set_schedule (pinned host) + nmc_anneal (host outputs)"}

    cpu = None
    if rank == 0 and world == 1 and args.cpu_baseline:
        cpu = cpu_baseline(wl, args.cpu_sweeps, args.cpu_replicas)

    ctx.replicas_destroy(rs)
    ctx.close()
    if rank != 0:
        return None
    res = {
        "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": ms_per_step, "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None, "dtype": "u32 (bit-sliced 32 replicas/word)",
        "data": "synthetic (seeded random 4-SAT; the paper's instances are not available)",
        "config": {"workload": wl["name"] + f"_t{T}", "n_vars": n, "n_clauses": int(lits.shape[0]),
                   "k": int(lits.shape[1]), "replicas": R, "sweeps": T, "n_colours": n_colours,
                   "attempts_per_step": attempts_per_step,
                   "parallelism": "replicas only" if world == 1 else f"replicas x{world} GPUs",
                   "l2": "flushed between steps (512 MB write); beta schedule 1 GB > L2"},
        "roofline": {"bound": "hbm", "achieved": achieved, "peak": peak, "unit": "GB/s",
                     "frac": achieved / peak, "traffic": None,
                     "kernel": "ksat_sweep_kernel (one persistent launch per step)",
                     "peak_source": peak_kind,
                     "algorithmic_bytes_per_launch": bytes_launch,
                     "launch_ms_mean": statistics.mean(sweep_ms)},
        "e2e": e2e,
        "gpu_launches": 4 * args.steps,
        "clocks": clk,
        "cpu_baseline": cpu,
    }
    return res


def cpu_baseline(wl, sweeps, replicas):
    import oracle as O
    O.build()
    n = wl["n_vars"]
    beta = np.ascontiguousarray(wl["beta"][:, :sweeps])
    threads = min(os.cpu_count() or 1, replicas)
    t0 = time.perf_counter()
    O.ksat_anneal(wl["lits"], n, beta, 0, sweeps, wl["seed"], replicas=replicas, n_threads=threads)
    dt = time.perf_counter() - t0
    att = n * replicas * sweeps
    return {"value": att / dt, "unit": UNIT, "cores": threads, "kind": "oracle",
            "sample": f"{replicas} replicas x {sweeps} sweeps of the same instance "
                      f"({att:.3g} attempts, {dt:.1f} s wall, includes the oracle's colouring)"}


def run_reference(args, world, rank):
    if rank != 0:
        return None
    wl = workload(args)
    n, R, T = wl["n_vars"], wl["replicas"], wl["n_steps"]
    for _ in range(args.warmup):
        pass  # the oracle has no warm-up state; each step is independent
    vals, secs = [], []
    cb = None
    for i in range(args.steps):
        cb = cpu_baseline(wl, args.cpu_sweeps, args.cpu_replicas)
        vals.append(cb["value"])
        secs.append(n * args.cpu_replicas * args.cpu_sweeps / cb["value"])
    value = statistics.mean(vals)
    return {"impl": "reference", "metric": METRIC, "value": value, "unit": UNIT,
            "n_gpus": world, "steps": args.steps, "warmup": args.warmup,
            "ms_per_step": 1e3 * statistics.mean(secs), "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "u8 (oracle, one replica per chain)",
            "data": "synthetic (seeded random 4-SAT)",
            "config": {"workload": wl["name"] + f"_t{T}", "n_vars": n, "replicas": R,
                       "sweeps": T, "parallelism": "host threads over replicas"},
            "cpu_baseline": {"value": value, "unit": UNIT, "cores": cb["cores"],
                             "kind": "oracle", "sample": cb["sample"]},
            "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0,
                    "d2h_bytes_per_step": 0}}


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=5)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--sweeps", type=int, default=5000)
    ap.add_argument("--n-vars", type=int, default=50_000)
    ap.add_argument("--replicas", type=int, default=1024)
    ap.add_argument("--e2e-steps", type=int, default=2)
    ap.add_argument("--cpu-sweeps", type=int, default=8)
    ap.add_argument("--cpu-replicas", type=int, default=64)
    ap.add_argument("--no-cpu-baseline", dest="cpu_baseline", action="store_false")
    ap.add_argument("--path", default="run", choices=["run", "batch", "grid"],
                    help="run: nmc_replicas_run (the library picks the kernel); batch: "
                         "nmc_batch_run; grid: nmc_replicas_run on the grid-barrier kernel")
    args = ap.parse_args()
    if args.path == "grid":
        os.environ["NMC_RUN_PATH"] = "grid"
    world, rank, local = dist_setup()
    if args.impl == "reference":
        res = run_reference(args, world, rank)
    else:
        res = run_ours(args, world, rank, local)
    if rank == 0 and res is not None:
        print(json.dumps(res))
    if world > 1:
        import torch.distributed as dist
        dist.destroy_process_group()


if __name__ == "__main__":
    main()
