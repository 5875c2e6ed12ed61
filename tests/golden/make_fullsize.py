"""Writes the full-length expected outputs of the two benchmark workloads, from the oracle only.

The trajectories pinned here are the ones the benchmark times: the single-variable Metropolis
sweep with a per-variable inverse temperature (Sec. "Nonequilibrium inhomogeneous sampling over
subgraphs"; the sampling steps of Algorithm 1) on the 4-SAT energy of Sec. "4-SAT Problems Near
Computational Phase Transitions", and the swap Metropolis chain on the Koopmans-Beckmann cost of
Sec. "Quadratic Assignment Problems". Every value is computed by `oracle/` on the seeded inputs of
`nmc_inputs`; nothing here comes from the CUDA path.

  python tests/golden/make_fullsize.py ksat    # ~20 min per replica per core (64 replicas)
  python tests/golden/make_fullsize.py qap     # ~1 min on 8 cores
  python tests/golden/make_fullsize.py batch   # ~8 min on 3 cores
  python tests/golden/make_fullsize.py wide    # ~10 min on 3 cores
  python tests/golden/make_fullsize.py pt      # ~30 min on one core (the rounds couple a ladder)
  python tests/golden/make_fullsize.py moves   # ~5 min on 3 cores

Outputs (JSON, next to this script):
  fullsize_ksat_n50000_r1024_t5000.json   4-SAT N=50,000, M=480,000, 1,024 replicas, 5,000 sweeps
  fullsize_qap_64x_r4096_t10000.json      64 QAP instances, n in [32, 256], 4,096 replicas, 10^4 steps
  fullsize_ksat_batch_256x_t2000.json     256 uneven 3-/4-SAT instances, N in [1000, 20000],
                                          32..256 replicas, 2,000 sweeps, factored schedules
  fullsize_ksat_wide_64x_t1000.json       64 uneven 3-SAT / 6-SAT instances, 1,000 sweeps
  fullsize_pt_4sat_n5000_32x32_t2000.json replica exchange, 32 ladders x 32 temperatures, 2,000 sweeps
  fullsize_moves_4sat_n50000_r1024_t500.json  two-chain held sampling (500 sweeps), collective
                                          flip of the backbone, whitening
Per sampled replica: final and best energies and SHA-256 digests of the final and best states
(uint8 [N] assignments in the original variable order; int16 [n] little-endian permutations).
"""
from __future__ import annotations

import hashlib
import json
import os
import sys
import time

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(os.path.dirname(HERE))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

import nmc_inputs as W  # noqa: E402
import oracle as O  # noqa: E402

KSAT_FILE = os.path.join(HERE, "fullsize_ksat_n50000_r1024_t5000.json")
QAP_FILE = os.path.join(HERE, "fullsize_qap_64x_r4096_t10000.json")
BATCH_FILE = os.path.join(HERE, "fullsize_ksat_batch_256x_t2000.json")
WIDE_FILE = os.path.join(HERE, "fullsize_ksat_wide_64x_t1000.json")
PT_FILE = os.path.join(HERE, "fullsize_pt_4sat_n5000_32x32_t2000.json")
MOVES_FILE = os.path.join(HERE, "fullsize_moves_4sat_n50000_r1024_t500.json")

# 64 replicas, two in each of the 32 words of 32 replicas: the first and last lanes of the first
# and last words, the rest drawn once with numpy's default_rng(64)
KSAT_IDS = [0, 31, 32, 53, 75, 93, 98, 99, 128, 158, 172, 189, 203, 221, 239, 255, 271, 276, 307,
            317, 330, 334, 374, 381, 404, 409, 419, 444, 459, 470, 491, 496, 517, 539, 545, 552, 578,
            584, 623, 625, 640, 652, 684, 698, 726, 735, 738, 743, 769, 777, 806, 824, 854, 858, 867,
            878, 919, 920, 943, 944, 970, 990, 1013, 1023]
# instances of the 64-instance QAP batch: the first, the smallest and largest n, and others
QAP_IDS = [0, 4095, 2047]


def digest(a: np.ndarray) -> str:
    return hashlib.sha256(np.ascontiguousarray(a).tobytes()).hexdigest()


KSAT_WORKLOAD = ("workload_ksat_large(n_steps=5000): 4-SAT N=50000, M=480000, beta geometric "
                 "0.3->6.0, 20% at 0.4x for the first half then ramped; 1024 replicas")
KSAT_FIELDS = ("energies", "best_energies", "states_sha256", "best_states_sha256")


def ksat():
    """Oracle outputs of the KSAT_IDS replicas. Replicas already in the file for the same workload
    and seed are kept (each replica's trajectory is independent of which others are computed with
    it), so the set can grow in several runs."""
    wl = W.workload_ksat_large(n_steps=5000)
    have = {}
    if os.path.exists(KSAT_FILE):
        with open(KSAT_FILE) as f:
            old = json.load(f)
        if old.get("workload") == KSAT_WORKLOAD and old.get("seed") == wl["seed"]:
            for j, r in enumerate(old["replica_ids"]):
                have[r] = {k: old[k][j] for k in KSAT_FIELDS}
    todo = [r for r in KSAT_IDS if r not in have]
    t = time.time()
    if todo:
        out = O.ksat_anneal(wl["lits"], wl["n_vars"], wl["beta"], 0, wl["n_steps"], wl["seed"],
                            replica_ids=todo, n_threads=min(len(todo), os.cpu_count() or 1))
        for j, r in enumerate(todo):
            have[r] = {"energies": int(out["energies"][j]),
                       "best_energies": int(out["best_energies"][j]),
                       "states_sha256": digest(out["states"][j]),
                       "best_states_sha256": digest(out["best_states"][j])}
    rec = {
        "workload": KSAT_WORKLOAD,
        "seed": wl["seed"], "t0": 0, "t1": wl["n_steps"], "replicas": wl["replicas"],
        "replica_ids": KSAT_IDS,
        **{k: [have[r][k] for r in KSAT_IDS] for k in KSAT_FIELDS},
        "oracle_seconds_last_run": round(time.time() - t, 1),
        "oracle_replicas_last_run": len(todo),
    }
    with open(KSAT_FILE, "w") as f:
        json.dump(rec, f, indent=1)
        f.write("\n")
    print(KSAT_FILE, rec["energies"], rec["best_energies"], rec["oracle_seconds_last_run"], "s")


def qap_instances(sets):
    ns = [s["n"] for s in sets]
    pick = [0, int(np.argmin(ns)), int(np.argmax(ns)), 17, 33, 63]
    seen = []
    for i in pick:
        if i not in seen:
            seen.append(i)
    return seen


def qap():
    sets = W.workload_qap_batch()  # 64 instances, 10^4 steps, 4096 replicas each
    t = time.time()
    recs = []
    for i in qap_instances(sets):
        s = sets[i]
        out = O.qap_anneal(s["F"], s["D"], s["beta"], 0, s["n_steps"], s["seed"],
                           replica_ids=QAP_IDS)
        recs.append({"instance": i, "n": s["n"], "seed": s["seed"], "replica_ids": QAP_IDS,
                     "energies": [int(x) for x in out["energies"]],
                     "best_energies": [int(x) for x in out["best_energies"]],
                     "perms_sha256": [digest(p.astype("<i2")) for p in out["perms"]],
                     "best_perms_sha256": [digest(p.astype("<i2")) for p in out["best_perms"]]})
        print("qap instance", i, "n", s["n"], recs[-1]["energies"], flush=True)
    rec = {"workload": "workload_qap_batch(): 64 instances, n uniform in [32, 256], F, D symmetric "
                       "uniform [0, 99] (F half zeros), beta linear 0.01->1.0 x per-facility "
                       "factor in [0.5, 1.5], 4096 replicas, 10^4 steps",
           "t0": 0, "t1": sets[0]["n_steps"], "replicas": sets[0]["replicas"],
           "instances": recs, "oracle_seconds": round(time.time() - t, 1)}
    with open(QAP_FILE, "w") as f:
        json.dump(rec, f, indent=1)
        f.write("\n")
    print(QAP_FILE, rec["oracle_seconds"], "s")


# Batched workloads: (instances, sweeps, mix of (k, alpha), seed, output file, checked instances).
# "batch": the first two (4-SAT, 3-SAT), the smallest N, the largest N (also the most replicas),
# the fewest replicas, the last. "wide": the first 3-SAT and 6-SAT, the largest 6-SAT, the
# smallest and largest N, the fewest (a 6-SAT) and most replicas, the last.
BATCHES = {
    "batch": (256, 2000, ((3, 4.2), (4, 9.6)), 1003, BATCH_FILE, [0, 1, 6, 35, 121, 255]),
    "wide": (64, 1000, ((3, 4.2), (6, 12.0)), 1006, WIDE_FILE, [0, 4, 17, 47, 19, 52, 12, 63]),
}


def batch(which="batch"):
    """A batched benchmark's instances as the batch launch runs them once from their initial
    states: sweeps 0..T-1 of each set, beta[u][t] = float32(factor[u] * base[t])."""
    n_inst, T, mix, seed, path, pick = BATCHES[which]
    specs = W.workload_ksat_mix(n_inst, T, mix, seed)
    t = time.time()
    recs = []
    for i in pick:
        s = specs[i]
        beta = (s["factor"][:, None] * s["base"][None, :]).astype(np.float32)
        ids = [0, s["R"] // 2, s["R"] - 1]
        out = O.ksat_anneal(s["lits"], s["n"], beta, 0, T, s["seed"], replica_ids=ids,
                            n_threads=len(ids))
        recs.append({"instance": i, "n": s["n"], "k": s["k"], "replicas": s["R"],
                     "seed": s["seed"], "replica_ids": ids,
                     "energies": [int(x) for x in out["energies"]],
                     "best_energies": [int(x) for x in out["best_energies"]],
                     "states_sha256": [digest(r) for r in out["states"]],
                     "best_states_sha256": [digest(r) for r in out["best_states"]]})
        print(which, "instance", i, "n", s["n"], "k", s["k"], recs[-1]["energies"], flush=True)
    kinds = " or ".join(f"{k}-SAT alpha {a}" for k, a in mix)
    rec = {"workload": f"workload_ksat_mix({n_inst}, {T}, {mix}, {seed}): {kinds}, N uniform in "
                       "[1000, 20000], 32..256 replicas, beta = factor x base (linear 0.5->4.0, "
                       f"30% at 0.5x), {T} sweeps",
           "t0": 0, "t1": T, "instances": recs, "oracle_seconds": round(time.time() - t, 1)}
    with open(path, "w") as f:
        json.dump(rec, f, indent=1)
        f.write("\n")
    print(path, rec["oracle_seconds"], "s")


def pt():
    """Replica exchange as the benchmark runs it (Sec. "Nonequilibrium inhomogeneous sampling
    over subgraphs"; App. "Adaptive Parallel Tempering"): 4-SAT N=5,000, alpha 9.884, 32 ladders
    of 32 temperatures (geometric 0.5 -> 5.0) over a homogeneous schedule, an exchange round every
    10 sweeps, 2,000 sweeps, Philox seed 1. Ladder 0 (replicas 0..31) evolves independently of the
    other ladders, so the oracle runs it alone (single-threaded: the rounds couple its replicas)."""
    n, alpha, T, L, per = 5000, 9.884, 2000, 32, 10
    lits = W.random_ksat(n, alpha, 4, 2111)
    ladder = W.geometric_profile(0.5, 5.0, L).astype(np.float32)
    t = time.time()
    out = O.ksat_pt_anneal(lits, n, np.ones((n, T), np.float32), ladder, 0, T, per, 1,
                           replicas=L)
    rec = {"workload": "4-SAT N=5000 alpha 9.884 (random_ksat seed 2111), ladder geometric "
                       "0.5->5.0 x 32, 32 ladders (1024 replicas), beta 1, 2000 sweeps, "
                       "exchange every 10, Philox seed 1; ladder 0",
           "t0": 0, "t1": T, "per": per, "replica_ids": list(range(L)),
           "energies": [int(x) for x in out["energies"]],
           "best_energies": [int(x) for x in out["best_energies"]],
           "states_sha256": [digest(r) for r in out["states"]],
           "best_states_sha256": [digest(r) for r in out["best_states"]],
           "slots": [int(x) for x in out["slots"]],
           "oracle_seconds": round(time.time() - t, 1)}
    with open(PT_FILE, "w") as f:
        json.dump(rec, f, indent=1)
        f.write("\n")
    print(PT_FILE, rec["energies"][:4], rec["oracle_seconds"], "s")


MOVES_IDS = [0, 517, 1023]


def moves():
    """Two-chain held sampling, then the collective move and whitening, as the benchmark runs
    them on the 50,000-variable instance (Algorithm 1's cycle; Sec. "Nonequilibrium inhomogeneous
    sampling over subgraphs"): a seeded 20% backbone, 10 cycles of 20 hot (base 3.0, heat 4) + 20
    cold + 10 unlearning sweeps, Philox seed 1, then one flip of the backbone at beta 0.75 (move
    1000) and generalized whitening of the best states."""
    wl = W.workload_ksat_large(n_steps=2)
    lits, n = wl["lits"], wl["n_vars"]
    labels = np.where(W.seeded_subset(n, 0.2, 77), 0, -1).astype(np.int32)
    cycles, th, tc, tu = 10, 20, 20, 10
    T = cycles * (th + tc + tu)
    beta = O.backbone_schedule(labels, 3.0, 4.0, cycles, th, tc, tu)
    t = time.time()
    ids = np.array(MOVES_IDS)
    ch = O.ksat_anneal(lits, n, beta, 0, T, 1, replica_ids=ids, n_threads=len(ids))
    mask = (labels >= 0).astype(np.uint8)
    mv = O.ksat_cluster_flip(lits, n, ch, mask, np.full(len(ids), 0.75, np.float32), 1000, 1,
                             replica_ids=ids)
    frozen = [int(O.ksat_whitening(lits, n, mv["best_states"][j])[1]) for j in range(len(ids))]
    rec = {"workload": "workload_ksat_large (4-SAT N=50000, M=480000), 1024 replicas, backbone "
                       "seeded_subset(n, 0.2, 77), 10 x (20 hot + 20 cold + 10 unlearning), base "
                       "3.0, heat 4.0, Philox seed 1; flip of the backbone at beta 0.75, move "
                       "1000; whitening of the best states",
           "t0": 0, "t1": T, "replica_ids": MOVES_IDS,
           "chain": {"energies": [int(x) for x in ch["energies"]],
                     "best_energies": [int(x) for x in ch["best_energies"]],
                     "states_sha256": [digest(r) for r in ch["states"]],
                     "best_states_sha256": [digest(r) for r in ch["best_states"]]},
           "accepted": [int(x) for x in mv["accepted"]],
           "energies": [int(x) for x in mv["energies"]],
           "best_energies": [int(x) for x in mv["best_energies"]],
           "states_sha256": [digest(r) for r in mv["states"]],
           "best_states_sha256": [digest(r) for r in mv["best_states"]],
           "frozen": frozen, "oracle_seconds": round(time.time() - t, 1)}
    with open(MOVES_FILE, "w") as f:
        json.dump(rec, f, indent=1)
        f.write("\n")
    print(MOVES_FILE, rec["energies"], rec["accepted"], rec["frozen"], rec["oracle_seconds"], "s")


if __name__ == "__main__":
    which = sys.argv[1:] or ["ksat", "qap", "batch", "wide", "pt", "moves"]
    if "qap" in which:
        qap()
    if "moves" in which:
        moves()
    if "pt" in which:
        pt()
    for b in ("batch", "wide"):
        if b in which:
            batch(b)
    if "ksat" in which:
        ksat()
