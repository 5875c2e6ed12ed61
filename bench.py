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


TRAFFIC_FILE = "ksat_batch_4sat_n50000_r1024_traffic.json"  # under profiles/


def captured_traffic(kernel: str, workload: str):
    """DRAM bytes per launch from the committed ncu capture, or None if the kernel source has
    changed since the counters were taken (or the workload differs)."""
    import hashlib
    try:
        with open(os.path.join(ROOT, "profiles", TRAFFIC_FILE)) as f:
            rec = json.load(f)[kernel]
        with open(os.path.join(ROOT, rec["source"]), "rb") as f:
            h = hashlib.sha256(f.read()).hexdigest()[:16]
        if h != rec["source_sha256_16"] or rec["workload"] != workload:
            return None
        return int(rec["dram_bytes_read"]) + int(rec["dram_bytes_write"])
    except Exception:
        return None


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
                     "frac": achieved / peak,
                     "traffic": (captured_traffic("ksat_batch_kernel", wl["name"] + f"_t{T}")
                                 if args.path != "grid" else None),
                     "kernel": ("ksat_batch_kernel (clusters of CTAs per replica word)"
                                if args.path != "grid" else "ksat_sweep_fast_kernel (grid barrier)"),
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
    """The oracle on the host cores, as it stands, on a bounded sample of the workload: the same
    replicas over the first `sweeps` sweeps and over the first `short` sweeps. The rate is the
    difference in attempts over the difference in wall time, so the one-off work of each call
    (the oracle's own colouring and incidence lists) is left out of it."""
    import oracle as O
    O.build()
    n = wl["n_vars"]
    short = max(1, sweeps // 6)
    threads = min(os.cpu_count() or 1, replicas)
    secs = []
    for sw in (short, sweeps):
        beta = np.ascontiguousarray(wl["beta"][:, :sw])
        t0 = time.perf_counter()
        O.ksat_anneal(wl["lits"], n, beta, 0, sw, wl["seed"], replicas=replicas, n_threads=threads)
        secs.append(time.perf_counter() - t0)
    att = n * replicas * (sweeps - short)
    dt = max(secs[1] - secs[0], 1e-9)
    return {"value": att / dt, "unit": UNIT, "cores": threads, "kind": "oracle",
            "seconds": secs[0] + secs[1],
            "sample": f"{replicas} replicas of the same instance over {short} and over {sweeps} "
                      f"sweeps ({secs[0]:.1f} s and {secs[1]:.1f} s wall); the rate is the "
                      f"{att:.3g} attempts of the extra {sweeps - short} sweeps over the time "
                      f"difference, so the oracle's one-off colouring and list building are "
                      f"excluded"}


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
        secs.append(cb["seconds"])
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


# ---------------------------------------------------------------------------------------------
# Secondary workloads (one JSON line each; the default line above is the headline)
# ---------------------------------------------------------------------------------------------

def _ctx_stream():
    import torch

    import paper_2111_13628_gb300 as nmc
    torch.cuda.set_device(0)
    stream = torch.cuda.Stream()
    return nmc.Context(0, stream=stream), stream


def _roofline(bytes_total, seconds, note):
    peak, src = peaks()
    a = bytes_total / seconds / 1e9
    return {"bound": "hbm", "achieved": a, "peak": peak, "unit": "GB/s", "frac": a / peak,
            "traffic": None, "peak_source": src, "note": note}


def _oracle_ksat_sample(jobs, threads=None):
    """Oracle rate over k-SAT jobs (lits, n, beta, seed, replicas, sweeps): each job runs over
    its first `sweeps` sweeps and over a sixth of them; the rate is the attempts of the extra
    sweeps over the extra wall time (the oracle's one-off colouring and lists left out)."""
    import oracle as O
    O.build()
    att, dt, wall, cores = 0, 0.0, 0.0, 1
    for lits, n, beta, seed, R, sw in jobs:
        short = max(1, sw // 6)
        th = min(os.cpu_count() or 1, R) if threads is None else threads
        cores = max(cores, th)
        secs = []
        for t in (short, sw):
            b = np.ascontiguousarray(beta[:, :t])
            t0 = time.perf_counter()
            O.ksat_anneal(lits, n, b, 0, t, seed, replicas=R, n_threads=th)
            secs.append(time.perf_counter() - t0)
        att += n * R * (sw - short)
        dt += max(secs[1] - secs[0], 1e-9)
        wall += secs[0] + secs[1]
    return att / dt, cores, wall, att


def run_ksat_small(args):
    """4-SAT N=200, M=1920, 64 replicas, 1000 sweeps: one step = one whole anneal."""
    import torch
    ctx, stream = _ctx_stream()
    wl = W.workload_ksat_small(1000)
    lits, n, beta, R, T = wl["lits"], wl["n_vars"], wl["beta"], wl["replicas"], wl["n_steps"]
    inst = ctx.load_ksat(lits, n)
    ctx.set_schedule(inst, beta)
    rs = ctx.replicas_create(inst, R, seed=wl["seed"])
    steps = max(args.steps, 10)
    for i in range(max(args.warmup, 3)):
        ctx.replicas_reset(rs, i)
        ctx.replicas_run(rs, 0, T)
    ctx.sync()
    clocks = Clocks(0)
    clocks.start()
    a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    a.record(stream)
    for i in range(steps):
        ctx.replicas_reset(rs, 100 + i)
        ctx.replicas_run(rs, 0, T)
    b.record(stream)
    ctx.sync()
    ck = clocks.stop()
    ms = a.elapsed_time(b) / steps
    _, n_colours = ctx.ksat_colouring(inst)
    ctx.close()
    rate, cores, wall, att = _oracle_ksat_sample([(lits, n, beta, wl["seed"], R, T)])
    bytes_step = algorithmic_bytes_per_sweep(lits, n, R) * T
    return {"metric": "Metropolis attempts/s", "value": n * R * T / (ms / 1e3), "unit": UNIT,
            "ms_per_step": ms, "steps": steps, "warmup": max(args.warmup, 3),
            "higher_is_better": True, "dtype": "u32 (bit-sliced 32 replicas/word)",
            "data": "synthetic (seeded random 4-SAT)",
            "config": {"workload": wl["name"] + "_t1000", "n_colours": n_colours,
                       "l2": "working set (100 KB) stays in L2: a latency-bound size"},
            "roofline": _roofline(bytes_step, ms / 1e3, "sweep byte model; the whole step "
                                  "(init, energies, 1000 sweeps) in the denominator"),
            "clocks": ck,
            "cpu_baseline": {"value": rate, "unit": UNIT, "cores": cores, "kind": "oracle",
                             "sample": f"the whole workload ({R} replicas) over 166 and 1000 "
                                       f"sweeps, rate from the difference ({wall:.1f} s wall)"}}


def run_ksat_batch(args, wide=False):
    """Uneven batch in one persistent launch per step: 256 instances of random 3-SAT (alpha 4.2)
    or 4-SAT (alpha 9.6), N in [1000, 20000], 32..256 replicas, 2000 sweeps, factored schedules.
    With wide: 64 instances of 3-SAT (alpha 4.2) or 6-SAT (alpha 12, two int4 list entries per
    occurrence), 1000 sweeps, the same otherwise. Beside it: the plain per-instance form (one
    nmc_replicas_run per set) on a sample of the sets."""
    import torch
    ctx, stream = _ctx_stream()
    if wide:
        n_inst, T, mix, seed = 64, 1000, [(3, 4.2), (6, 12.0)], 1006
    else:
        n_inst, T, mix, seed = args.batch_instances, 2000, [(3, 4.2), (4, 9.6)], 1003
    specs = W.workload_ksat_mix(n_inst, T, mix, seed)
    sets, attempts, per, bytes_step = [], 0, [], 0
    for sp in specs:
        inst = ctx.load_ksat(sp["lits"], sp["n"])
        ctx.set_schedule_factored(inst, sp["base"], sp["factor"])
        rs = ctx.replicas_create(inst, sp["R"], seed=sp["seed"])
        sets.append(rs)
        attempts += sp["n"] * sp["R"] * T
        bytes_step += algorithmic_bytes_per_sweep(sp["lits"], sp["n"], sp["R"]) * T
        per.append((rs, sp["n"] * sp["R"] * T))
    # launch shapes tuned on 8 sweeps of this batch (outside the timed region; states restored)
    shapes = ctx.batch_autotune(sets, 0, 8).tolist()
    flush = torch.empty(512 * 2 ** 20 // 4, dtype=torch.float32, device="cuda")
    clocks = Clocks(0)
    tot = 0.0
    for i in range(max(args.warmup, 3) + args.steps):
        if i == max(args.warmup, 3):
            clocks.start()
        with torch.cuda.stream(stream):
            flush.fill_(float(i))  # L2 flush between steps (outside the events)
        a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        a.record(stream)
        for j, rs in enumerate(sets):
            ctx.replicas_reset(rs, 10_000 + j + 1000 * i)
        ctx.batch_run(sets, 0, T)
        b.record(stream)
        ctx.sync()
        if i >= max(args.warmup, 3):
            tot += a.elapsed_time(b)
    ck = clocks.stop()
    ms = tot / args.steps
    # plain per-instance form on a sample of the sets: one nmc_replicas_run per set, in turn
    sample = per[:: max(1, len(per) // 16)]
    c, d = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    c.record(stream)
    for rs, _ in sample:
        ctx.replicas_run(rs, 0, T)
    d.record(stream)
    ctx.sync()
    plain = sum(x for _, x in sample) / (c.elapsed_time(d) / 1e3)
    ctx.close()
    jobs = []
    for sp in specs[:: max(1, n_inst // 4)][:4]:
        beta = (sp["factor"][:, None] * sp["base"][None, :24]).astype(np.float32)
        jobs.append((sp["lits"], sp["n"], beta, sp["seed"], min(sp["R"], 32), 24))
    rate, cores, wall, att = _oracle_ksat_sample(jobs)
    name = (f"ksat_batch_{n_inst}x_3sat_6sat_N1k-20k_R32-256_t{T}" if wide
            else f"ksat_batch_{n_inst}x_N1k-20k_R32-256_t{T}")
    return {"metric": "Metropolis attempts/s (batched, one launch)", "value": attempts / (ms / 1e3),
            "unit": UNIT, "ms_per_step": ms, "steps": args.steps, "warmup": max(args.warmup, 3),
            "higher_is_better": True, "dtype": "u32 (bit-sliced 32 replicas/word)",
            "data": "synthetic (seeded random k-SAT)",
            "config": {"workload": name, "attempts_per_step": attempts,
                       "mix": [f"{k}-SAT alpha {a}" for k, a in mix],
                       "l2": "flushed between steps (512 MB write)",
                       "tuned_shapes": {"k<=4": shapes[0], "k<=8": shapes[1],
                                        "fields": "CTAs per item, lanes, us per sweep"}},
            "roofline": _roofline(bytes_step, ms / 1e3, "sweep byte model summed over the "
                                  "instances; the step includes the initial states and energies"),
            "plain_per_instance": {"value": plain, "unit": UNIT,
                                   "sample": f"{len(sample)} of the {n_inst} sets, one launch each"},
            "clocks": ck,
            "cpu_baseline": {"value": rate, "unit": UNIT, "cores": cores, "kind": "oracle",
                             "sample": f"{len(jobs)} of the instances, up to 32 replicas each, "
                                       f"over 4 and 24 sweeps; rate from the difference "
                                       f"({att:.3g} attempts, {wall:.1f} s wall)"}}


def run_qap_batch(args):
    """64 QAP instances, n in [32, 256], 4096 replicas each, all 10^4 steps of the schedule (one
    step of the bench = the whole anneal, one batched launch per launch shape)."""
    import torch
    ctx, stream = _ctx_stream()
    specs = W.workload_qap_batch()
    T = specs[0]["n_steps"]
    sets, attempts, bytes_step = [], 0, 0
    for sp in specs:
        inst = ctx.load_qap(sp["F"], sp["D"])
        ctx.set_schedule(inst, sp["beta"])
        sets.append(ctx.replicas_create(inst, sp["replicas"], seed=sp["seed"]))
        attempts += sp["n"] * sp["replicas"] * T
        bytes_step += 2 * sp["n"] * sp["n"] * sp["replicas"] * T  # 2n B per swap attempt
    clocks = Clocks(0)
    tot = 0.0
    for i in range(args.warmup + args.steps):
        if i == args.warmup:
            clocks.start()
        a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        a.record(stream)
        for j, rs in enumerate(sets):
            ctx.replicas_reset(rs, specs[j]["seed"] + 1000 * i)
        ctx.qap_batch_run(sets, 0, T)
        b.record(stream)
        ctx.sync()
        if i >= args.warmup:
            tot += a.elapsed_time(b)
    ck = clocks.stop()
    ms = tot / args.steps
    ctx.close()
    import oracle as O
    O.build()
    R, steps = 64, 200
    t0 = time.perf_counter()
    att = 0
    for sp in specs:
        O.qap_anneal(sp["F"], sp["D"], np.ascontiguousarray(sp["beta"][:, :steps]), 0, steps,
                     sp["seed"], replicas=R)
        att += sp["n"] * R * steps
    cpu_s = time.perf_counter() - t0
    return {"metric": "swap attempts/s", "value": attempts / (ms / 1e3), "unit": "swap attempts/s",
            "ms_per_step": ms, "steps": args.steps, "warmup": args.warmup,
            "higher_is_better": True, "dtype": "i16 permutations, i32/i64 costs",
            "data": "synthetic (seeded random QAP)",
            "config": {"workload": f"qap_64x_n32-256_R4096_t{T}", "attempts_per_step": attempts,
                       "l2": "F, D and the permutations (75 MB) stay L2-resident; the 369 MB "
                             "schedule streams"},
            "roofline": _roofline(bytes_step, ms / 1e3, "2n bytes of permutation state per "
                                  "swap attempt; F and D come from shared memory"),
            "clocks": ck,
            "cpu_baseline": {"value": att / cpu_s, "unit": "swap attempts/s",
                             "cores": min(os.cpu_count() or 1, R), "kind": "oracle",
                             "sample": f"all 64 instances, {R} replicas each, the first {steps} "
                                       f"steps ({att:.3g} attempts, {cpu_s:.1f} s wall)"}}


def run_pt(args):
    """Replica exchange on random 4-SAT N=5,000, alpha=9.884 (M=49,420, the paper's 4-SAT
    size): 32 ladders x 32 temperatures (1,024 replicas), geometric ladder beta 0.5 -> 5.0 over
    a homogeneous schedule, an exchange round every 10 sweeps, 2,000 sweeps per step. Beside
    it: the same sweeps without exchanges, and the adaptive ladder's construction time."""
    import torch
    ctx, stream = _ctx_stream()
    n, alpha, T, L, G, per = 5000, 9.884, 2000, 32, 32, 10
    lits = W.random_ksat(n, alpha, 4, 2111)
    inst = ctx.load_ksat(lits, n)
    ctx.set_schedule_factored(inst, np.ones(T, np.float32), np.ones(n, np.float32))
    R = G * L
    rs = ctx.replicas_create(inst, R, seed=1)
    ladder = W.geometric_profile(0.5, 5.0, L).astype(np.float32)
    ctx.set_ladder(rs, ladder)
    flush = torch.empty(512 * 2 ** 20 // 4, dtype=torch.float32, device="cuda")

    def timed(fn, steps):
        tot = 0.0
        for i in range(args.warmup + steps):
            with torch.cuda.stream(stream):
                flush.fill_(float(i))  # L2 flush between steps (outside the events)
            a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            a.record(stream)
            fn(i)
            b.record(stream)
            ctx.sync()
            if i >= args.warmup:
                tot += a.elapsed_time(b)
        return tot / steps

    def pt_step(i):
        ctx.replicas_reset(rs, 100 + i)
        ctx.run_pt(rs, 0, T, per)

    def plain_step(i):  # the same ladder temperatures, no exchange round (one launch)
        ctx.replicas_reset(rs, 100 + i)
        ctx.run_pt(rs, 0, T, T + 1)

    clocks = Clocks(0)
    clocks.start()
    ms = timed(pt_step, args.steps)
    ck = clocks.stop()
    ms_plain = timed(plain_step, max(2, args.steps // 2))
    t = time.time()
    betas, sigmas = ctx.adaptive_ladder(inst, 256, 3, 0.3, 1.1, 1.0, 48, 50, 100)
    ladder_s = time.time() - t
    ctx.close()
    import oracle as O
    t = time.time()
    O.ksat_pt_anneal(lits, n, np.ones((n, 20), np.float32), ladder, 0, 20, per, 1, replicas=L)
    cpu_s = time.time() - t
    cpu = {"value": n * L * 20 / cpu_s, "unit": UNIT, "cores": 1, "kind": "oracle",
           "sample": f"one ladder of {L} replicas x 20 sweeps, exchange every {per} "
                     f"({cpu_s:.1f} s, single-threaded: the rounds couple the replicas)"}
    attempts = n * R * T
    bps = algorithmic_bytes_per_sweep(lits, n, R)
    peak, src = peaks()
    achieved = bps * T / (ms / 1e3) / 1e9
    return {"metric": "Metropolis attempts/s (replica exchange)", "value": attempts / (ms / 1e3),
            "unit": UNIT, "ms_per_step": ms, "steps": args.steps, "warmup": args.warmup,
            "higher_is_better": True, "dtype": "u32 (bit-sliced 32 replicas/word)",
            "data": "synthetic (seeded random 4-SAT)",
            "config": {"workload": f"pt_4sat_n{n}_m{lits.shape[0]}_{G}x{L}temps_t{T}_round{per}",
                       "attempts_per_step": attempts, "exchange_rounds": T // per,
                       "l2": "flushed between steps (512 MB write)"},
            "roofline": {"bound": "hbm", "achieved": achieved, "peak": peak, "unit": "GB/s",
                         "frac": achieved / peak, "traffic": None, "peak_source": src,
                         "note": "whole step (sweep launches + exchange rounds) against the "
                                 "sweep byte model"},
            "no_exchange": {"value": attempts / (ms_plain / 1e3), "unit": UNIT,
                            "ms_per_step": ms_plain},
            "adaptive_ladder": {"s": ladder_s, "temps": int(len(betas)),
                                "beta_last": float(betas[-1]), "sigma_last": float(sigmas[-1]),
                                "config": "256 replicas, beta0 0.3, alpha 1.1, sigma_min 1.0, "
                                          "50 + 100 sweeps per level"},
            "clocks": ck, "cpu_baseline": cpu}


def _timed_events(stream, fn, warmup, steps, flush=None):
    """Mean CUDA-event time of fn(i) over `steps` calls after `warmup` calls; an optional L2
    flush runs between calls, outside the events."""
    import torch
    tot = 0.0
    for i in range(warmup + steps):
        if flush is not None:
            with torch.cuda.stream(stream):
                flush.fill_(float(i))
        a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        a.record(stream)
        fn(i)
        b.record(stream)
        torch.cuda.synchronize()
        if i >= warmup:
            tot += a.elapsed_time(b)
    return tot / steps


def run_learning(args):
    """Learning stage on random 4-SAT N=5,000, alpha=9.884 (M=49,420): loopy BP on the surrogate
    Hamiltonians of 64 seeds at once (seeds = best states of a 200-sweep anneal at beta 3), lambda
    continuation 0.4 -> 0.025, beta 1, tol 1e-8, at most 100 iterations per lambda; then backbone
    growth from the correlations. Metric: message updates (edge x seed x iteration) per second."""
    import torch
    ctx, stream = _ctx_stream()
    n, S = 5000, 64
    lits = W.random_ksat(n, 9.884, 4, 2111)
    inst = ctx.load_ksat(lits, n)
    ctx.set_schedule(inst, W.beta_constant(n, 200, 3.0))
    seeds = ctx.anneal(inst, S, 0, 200, 5)["best_states"]
    lams = [0.4, 0.2, 0.1, 0.05, 0.025]
    flush = torch.empty(512 * 2 ** 20 // 4, dtype=torch.float32, device="cuda")
    out = {}

    def lbp(i):
        out["r"] = ctx.cnf_lbp(inst, seeds, 1.0, lams, 1e-8, 100)

    ms = _timed_events(stream, lbp, args.warmup, args.steps, flush)
    r = out["r"]
    edges = int((lits != 0).sum())
    updates = edges * int(r["iters"].sum())
    t_bb = _timed_events(stream, lambda i: ctx.cnf_backbone(inst, r["corr"], 1.0, 2.5, 2.0),
                         1, 3)
    lab, nc = ctx.cnf_backbone(inst, r["corr"], 1.0, 2.5, 2.0)
    ctx.close()
    import oracle as O
    t = time.time()
    ro = O.cnf_lbp(lits, n, seeds[0], 1.0, lams, 1e-8, 100)
    cpu_s = time.time() - t
    cpu = {"value": edges * int(ro["iters"].sum()) / cpu_s, "unit": "edge-seed updates/s",
           "cores": 1, "kind": "oracle",
           "sample": f"seed 0 alone, same lambdas ({int(ro['iters'].sum())} iterations, "
                     f"{cpu_s:.1f} s)"}
    bytes_per_update = 40  # u read + h write (variable pass), h read + u read/write (clause pass)
    peak, src = peaks()
    achieved = bytes_per_update * updates / (ms / 1e3) / 1e9
    return {"metric": "LBP message updates/s", "value": updates / (ms / 1e3),
            "unit": "edge-seed updates/s", "ms_per_step": ms, "steps": args.steps,
            "warmup": args.warmup, "higher_is_better": True, "dtype": "f64",
            "data": "synthetic (seeded random 4-SAT; seeds from the engine's anneal)",
            "config": {"workload": f"lbp_4sat_n{n}_m{lits.shape[0]}_S{S}_lambda5",
                       "edges": edges, "iterations_total": int(r["iters"].sum()),
                       "lambdas_converged_mean": float(r["n_done"].mean()),
                       "l2": "flushed between steps (512 MB write); messages 4 x 101 MB > L2"},
            "roofline": {"bound": "hbm", "achieved": achieved, "peak": peak, "unit": "GB/s",
                         "frac": achieved / peak, "traffic": None, "peak_source": src,
                         "note": "40 B per edge-seed update (8 B u + 8 B h, then 8 B h + 16 B u); "
                                 "includes one 4-byte readback per iteration"},
            "backbone": {"ms": t_bb, "clusters_seed0": int(nc[0]),
                         "backbone_vars_seed0": int((lab[0] >= 0).sum()),
                         "thresholds": "seed 2.5, cutoff 2.0"},
            "cpu_baseline": cpu}


def run_moves(args):
    """Held-unit (two-chain) sampling, the collective move and whitening on the bench instance
    (4-SAT N=50,000, M=480,000, 1,024 replicas). Two-chain schedule: a seeded 20% backbone,
    10 cycles of 20 hot (base 3.0 / heat 4) + 20 cold + 10 unlearning sweeps (500 sweeps). Metric:
    attempts on the unheld variables per second; beside it the same 500 sweeps with nothing held,
    one collective flip of the backbone (ms), and whitening of all replicas (ms)."""
    import torch
    ctx, stream = _ctx_stream()
    wl = W.workload_ksat_large(n_steps=2)
    lits, n, R = wl["lits"], wl["n_vars"], 1024
    inst = ctx.load_ksat(lits, n)
    bb = W.seeded_subset(n, 0.2, 77)
    labels = np.where(bb, 0, -1).astype(np.int32)
    cycles, th, tc, tu = 10, 20, 20, 10
    T = cycles * (th + tc + tu)
    ctx.set_schedule_backbone(inst, labels, cycles, th, tc, tu, 3.0, 4.0)
    rs = ctx.replicas_create(inst, R, seed=1)
    flush = torch.empty(512 * 2 ** 20 // 4, dtype=torch.float32, device="cuda")

    def held(i):
        ctx.replicas_reset(rs, 10 + i)
        ctx.replicas_run(rs, 0, T)

    clocks = Clocks(0)
    clocks.start()
    ms = _timed_events(stream, held, args.warmup, args.steps, flush)
    ck = clocks.stop()
    nb = int(bb.sum())
    attempts = R * cycles * (th * nb + tc * (n - nb) + tu * n)
    # byte model restricted to the attempted variables: per variable and sweep its clauses' other
    # literals (k-1 words each), its own word read and written, its entries (k int32 each) and
    # its beta (the same terms as algorithmic_bytes_per_sweep)
    used = lits != 0
    deg = np.bincount(np.abs(lits[used]) - 1, minlength=n).astype(np.int64)
    kk = used.sum(axis=1)
    nbr = np.zeros(n, np.int64)
    np.add.at(nbr, np.abs(lits[used]) - 1, np.repeat(kk - 1, kk))
    Wd = (R + 31) // 32
    per_var = nbr * 4 * Wd + 2 * 4 * Wd + deg * lits.shape[1] * 4 + 4
    bytes_step = cycles * (th * int(per_var[bb].sum()) + tc * int(per_var[~bb].sum()) +
                           tu * int(per_var.sum()))
    ctx.set_schedule_factored(inst, np.full(T, 3.0, np.float32), np.ones(n, np.float32))
    ms_plain = _timed_events(stream, held, 1, max(2, args.steps // 2), flush)
    mask = bb.astype(np.uint8)
    beta = np.full(R, 0.75, np.float32)
    ms_flip = _timed_events(stream, lambda i: ctx.cluster_flip(rs, mask, beta, 1000 + i),
                            2, 5, flush)
    ms_white = _timed_events(stream, lambda i: ctx.whitening(rs), 1, 3, flush)
    frozen = ctx.whitening(rs)
    st = ctx.replicas_read(rs)
    ctx.close()
    import oracle as O
    sched = O.backbone_schedule(labels, 3.0, 4.0, 1, th, tc, tu)[:, :th]
    t = time.time()
    O.ksat_anneal(lits, n, sched, 0, th, 1, replicas=16)
    cpu_s = time.time() - t
    t = time.time()
    for r in range(4):
        O.ksat_whitening(lits, n, st["states"][r])
    cpu_w = (time.time() - t) / 4
    cpu = {"value": 16 * th * nb / cpu_s, "unit": UNIT, "cores": min(16, os.cpu_count() or 1),
           "kind": "oracle",
           "sample": f"16 replicas x the {th} hot sweeps of the first cycle ({cpu_s:.1f} s, "
                     f"includes the oracle's colouring); whitening {cpu_w * 1e3:.0f} ms per "
                     f"replica single-threaded"}
    return {"metric": "Metropolis attempts/s (two-chain held sampling)",
            "value": attempts / (ms / 1e3), "unit": UNIT, "ms_per_step": ms,
            "steps": args.steps, "warmup": args.warmup, "higher_is_better": True,
            "dtype": "u32 (bit-sliced 32 replicas/word)", "data": "synthetic (seeded random 4-SAT)",
            "config": {"workload": f"twochain_4sat_n{n}_r{R}_bb20pct_{cycles}x({th}+{tc}+{tu})",
                       "attempts_per_step": attempts, "sweeps": T,
                       "l2": "flushed between steps (512 MB write)"},
            "nothing_held": {"ms_per_step": ms_plain, "value": n * R * T / (ms_plain / 1e3)},
            "cluster_flip": {"ms_per_move": ms_flip, "mask_vars": nb, "replicas": R},
            "whitening": {"ms": ms_white, "frozen_mean": float(frozen.mean())},
            "roofline": {"bound": "hbm", "achieved": bytes_step / (ms / 1e3) / 1e9,
                         "peak": peaks()[0], "unit": "GB/s",
                         "frac": bytes_step / (ms / 1e3) / 1e9 / peaks()[0], "traffic": None,
                         "peak_source": peaks()[1],
                         "note": "sweep byte model over the attempted (unheld) variables"},
            "clocks": ck, "cpu_baseline": cpu}


def _serving_stream(args):
    """Config 5's request stream: Poisson arrivals at args.rate for args.duration seconds; each
    request random 4-SAT (N log-uniform in [500, 50000], alpha uniform in [9.0, 9.8], 32
    replicas, beta linear 0.5 -> 4.0 with a seeded 30% at 0.5x) or QAP (n uniform in [32, 192],
    F, D as the QAP batch, 256 replicas, beta linear 0.01 -> 1.0 times a seeded per-facility
    factor in [0.5, 1.5]), with probability 1/2 each, of 1000..5000 sweeps. The formulas and
    matrices are drawn from a pool generated before the run (args.pool 4-SAT formulas and
    args.pool / 4 QAP instances, each request picking one), so that generating synthetic data
    does not delay the arrivals; every request's instance is still built by the engine inside
    its submit call (colouring, lists), and that is part of its measured latency."""
    rate, dur = args.rate, args.duration
    s = W.Stream(1005)
    pool_k, pool_q = [], []
    for i in range(args.pool):
        n = int(round(float(np.exp(np.log(500) + (np.log(50000) - np.log(500)) * s.unit(1)[0]))))
        alpha = 9.0 + 0.8 * s.unit(1)[0]
        pool_k.append((W.random_ksat(n, alpha, 4, 1005 * 1000 + i), n))
    for i in range(max(2, args.pool // 4)):
        n = 32 + int(s.below(161, 1)[0])
        F, D = W.random_qap(n, 1005 * 3000 + i)
        pool_q.append((F, D, n))
    t_arr = np.cumsum(-np.log(1.0 - s.unit(int(rate * dur * 1.5) + 10)) / rate)
    t_arr = t_arr[t_arr < dur]
    nreq = len(t_arr)
    is_q = s.below(2, nreq)
    which = s.below(1 << 30, nreq)
    sweeps = 1000 + s.below(4001, nreq)
    reqs = []
    for i in range(nreq):
        T = int(sweeps[i])
        if is_q[i]:
            F, D, n = pool_q[int(which[i]) % len(pool_q)]
            base = W.linear_profile(0.01, 1.0, T).astype(np.float32)
            factor = (0.5 + W.Stream(7000 + i).unit(n)).astype(np.float32)
            reqs.append(("qap", (F, D, n), base, factor, 256, T))
        else:
            lits, n = pool_k[int(which[i]) % len(pool_k)]
            base = W.linear_profile(0.5, 4.0, T).astype(np.float32)
            factor = np.where(W.seeded_subset(n, 0.3, 8000 + i), 0.5, 1.0).astype(np.float32)
            reqs.append(("ksat", (lits, n), base, factor, 32, T))
    return t_arr, reqs


def run_serving(args):
    """Serving loop under config 5's load: p50 / p99 latency (from the start of each submit call
    to completion) and achieved attempts/s, beside the plain path measured on the same arrival
    stream: one request at a time in arrival order through nmc_load_* + nmc_set_schedule_factored
    + nmc_anneal (FIFO), run for a bounded time and reported on the requests it completed."""
    import paper_2111_13628_gb300 as nmc
    t_arr, reqs = _serving_stream(args)
    nreq = len(reqs)
    work = [r[1][-1] * r[4] * r[5] for r in reqs]
    srv = nmc.Server(0, max_active=args.max_active, slice_log2=args.slice_log2,
                     memory_budget=int(args.memory_budget_gb * (1 << 30)))
    ids = [None] * nreq
    t0 = time.perf_counter()

    def submit_one(i):
        kind, inst, base, factor, R, T = reqs[i]
        wait = t0 + t_arr[i] - time.perf_counter()
        if wait > 0:
            time.sleep(wait)
        if kind == "ksat":
            ids[i] = srv.submit_ksat(inst[0], inst[1], base=base, factor=factor, replicas=R, seed=i)
        else:
            ids[i] = srv.submit_qap(inst[0], inst[1], base=base, factor=factor, replicas=R, seed=i)

    from concurrent.futures import ThreadPoolExecutor
    # submissions run on a pool: a k-SAT submit builds the instance on the host (colouring,
    # lists) on the calling thread, so arrivals are not serialised behind one another
    with ThreadPoolExecutor(max_workers=16) as pool:
        list(pool.map(submit_one, range(nreq)))
    late = time.perf_counter() - t0 - float(t_arr[-1])
    print(f"serving: {nreq} requests submitted (last {late:.2f} s after its arrival time); "
          f"stats {srv.stats()}", file=sys.stderr, flush=True)
    lat, failed = np.full(nreq, np.nan), 0
    for j, i in enumerate(ids):
        while srv.poll(i, wait_ms=500) in (0, 1):
            pass
        try:
            _, lat[j] = srv.result(i)
        except nmc.NmcError:
            failed += 1
    wall = time.perf_counter() - t0
    st = srv.stats()
    print(f"serving: all done after {wall:.1f} s; stats {st}", file=sys.stderr, flush=True)
    srv.close()
    # plain single-instance path, measured: a worker takes the requests in arrival order (waiting
    # for each arrival time) and runs each alone; latency = completion - arrival
    ctx = nmc.Context(0)
    plat, pwork, busy = [], 0, 0.0
    p0 = time.perf_counter()
    for i in range(nreq):
        now = time.perf_counter() - p0
        if now > args.plain_seconds:
            break
        if now < t_arr[i]:
            time.sleep(t_arr[i] - now)
        kind, inst, base, factor, R, T = reqs[i]
        tt = time.perf_counter()
        h = ctx.load_ksat(inst[0], inst[1]) if kind == "ksat" else ctx.load_qap(inst[0], inst[1])
        ctx.set_schedule_factored(h, base, factor)
        ctx.anneal(h, R, 0, T, seed=i)
        ctx.unload(h)
        done = time.perf_counter()
        busy += done - tt
        plat.append(done - p0 - t_arr[i])
        pwork += work[i]
    ctx.close()
    k = len(plat)
    srv_k = lat[:k][~np.isnan(lat[:k])]
    return {"metric": "serving latency and throughput", "unit": "s",
            "p50_s": float(np.nanpercentile(lat, 50)), "p99_s": float(np.nanpercentile(lat, 99)),
            "requests": nreq, "failed": failed, "offered_attempts_per_s": sum(work) / args.duration,
            "achieved_attempts_per_s": sum(work) / wall, "wall_s": wall,
            "server": st,
            "config": {"workload": f"serving_poisson{args.rate:g}rps_{args.duration:g}s",
                       "pool": f"{args.pool} 4-SAT formulas, {max(2, args.pool // 4)} QAP "
                               f"instances (generated before the run)",
                       "max_active": args.max_active, "slice_log2": args.slice_log2},
            "plain_fifo": {"attempts_per_s": pwork / busy if busy > 0 else None,
                           "requests": k, "p50_s": float(np.percentile(plat, 50)),
                           "p99_s": float(np.percentile(plat, 99)),
                           "served_same_requests": {"p50_s": float(np.percentile(srv_k, 50)),
                                                    "p99_s": float(np.percentile(srv_k, 99))},
                           "sample": f"the first {k} requests of the same stream, queued in "
                                     f"arrival order through nmc_anneal alone for "
                                     f"{args.plain_seconds:g} s (measured, not modelled)"}}


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
    ap.add_argument("--cpu-sweeps", type=int, default=12)
    ap.add_argument("--cpu-replicas", type=int, default=64)
    ap.add_argument("--no-cpu-baseline", dest="cpu_baseline", action="store_false")
    ap.add_argument("--workload", default="ksat_large",
                    choices=["ksat_large", "ksat_small", "ksat_batch", "ksat_wide", "qap_batch",
                             "serving", "pt", "learning", "moves"])
    ap.add_argument("--batch-instances", type=int, default=256)
    ap.add_argument("--rate", type=float, default=200.0)
    ap.add_argument("--duration", type=float, default=60.0)
    ap.add_argument("--pool", type=int, default=256)
    ap.add_argument("--max-active", type=int, default=4096)
    ap.add_argument("--slice-log2", type=int, default=30)
    ap.add_argument("--memory-budget-gb", type=float, default=200.0)
    ap.add_argument("--plain-seconds", type=float, default=90.0)
    ap.add_argument("--path", default="run", choices=["run", "batch", "grid"],
                    help="run: nmc_replicas_run (the library picks the kernel); batch: "
                         "nmc_batch_run; grid: nmc_replicas_run on the grid-barrier kernel")
    args = ap.parse_args()
    if args.path == "grid":
        os.environ["NMC_RUN_PATH"] = "grid"
    world, rank, local = dist_setup()
    if args.impl == "reference":
        res = run_reference(args, world, rank)
    elif args.workload != "ksat_large":
        fn = {"ksat_small": run_ksat_small, "ksat_batch": run_ksat_batch,
              "ksat_wide": lambda a: run_ksat_batch(a, wide=True),
              "qap_batch": run_qap_batch, "serving": run_serving, "pt": run_pt,
              "learning": run_learning, "moves": run_moves}[args.workload]
        res = fn(args) if rank == 0 else None
    else:
        res = run_ours(args, world, rank, local)
    if rank == 0 and res is not None:
        print(json.dumps(res))
    if world > 1:
        import torch.distributed as dist
        dist.destroy_process_group()


if __name__ == "__main__":
    main()
