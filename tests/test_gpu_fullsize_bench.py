"""The benchmark's own workloads at full length, on the GPU, against stored oracle outputs.

`bench.py` times a 5,000-sweep anneal of 1,024 replicas of a 50,000-variable 4-SAT formula (the
sampling stage of Algorithm 1 with a per-variable inverse temperature, Sec. "Nonequilibrium
inhomogeneous sampling over subgraphs"), the same sweep over batches of uneven formulas (256
3-/4-SAT sets for 2,000 sweeps, 64 3-/6-SAT sets for 1,000) in one launch, and a 10^4-step swap
anneal of 64 QAP instances with 4,096 replicas each (Sec. "Quadratic Assignment Problems"). These
tests run exactly those launches and compare sampled replicas with `tests/golden/fullsize_*.json`,
which `tests/golden/make_fullsize.py` wrote from the oracle alone (the oracle needs about twenty
minutes per replica of the 50,000-variable run, so the expected values are stored rather than
recomputed here). Final and best energies must be equal and the final
and best states equal byte for byte (SHA-256 of each row): tolerance zero, all outputs are integers.
Every replica is also checked for the invariants best <= final, and a spread of them for energies
that match a recount of their states.
"""
import hashlib
import json
import os

import numpy as np
import pytest

import nmc_inputs as W
import oracle as O

pytestmark = pytest.mark.gpu

GOLDEN = os.path.join(os.path.dirname(os.path.abspath(__file__)), "golden")


def _digest(a):
    return hashlib.sha256(np.ascontiguousarray(a).tobytes()).hexdigest()


def _golden(name):
    with open(os.path.join(GOLDEN, name)) as f:
        return json.load(f)


@pytest.fixture(scope="module")
def ctx():
    import paper_2111_13628_gb300 as nmc
    c = nmc.Context(0)
    yield c
    c.close()


def test_ksat_bench_workload_full_length(ctx):
    g = _golden("fullsize_ksat_n50000_r1024_t5000.json")
    wl = W.workload_ksat_large(n_steps=g["t1"])
    lits, n, beta, R = wl["lits"], wl["n_vars"], wl["beta"], wl["replicas"]
    assert R == g["replicas"] and wl["seed"] == g["seed"]
    inst = ctx.load_ksat(lits, n)
    ctx.set_schedule(inst, beta)
    del beta
    rs = ctx.replicas_create(inst, R, seed=g["seed"])
    ctx.replicas_run(rs, g["t0"], g["t1"])  # the bench's launch: the library's default path
    got = ctx.replicas_read(rs)
    ctx.replicas_destroy(rs)
    ctx.unload(inst)
    for j, r in enumerate(g["replica_ids"]):
        assert int(got["energies"][r]) == g["energies"][j], r
        assert int(got["best_energies"][r]) == g["best_energies"][j], r
        assert _digest(got["states"][r]) == g["states_sha256"][j], r
        assert _digest(got["best_states"][r]) == g["best_states_sha256"][j], r
    assert np.all(got["best_energies"] <= got["energies"])
    assert np.all(got["best_energies"] >= 0)
    rows = np.arange(0, R, 61)
    assert np.array_equal(O.ksat_energies(lits, n, got["states"][rows]), got["energies"][rows])
    assert np.array_equal(O.ksat_energies(lits, n, got["best_states"][rows]),
                          got["best_energies"][rows])


@pytest.mark.parametrize("name,n_inst,T,mix,seed", [
    ("fullsize_ksat_batch_256x_t2000.json", 256, 2000, ((3, 4.2), (4, 9.6)), 1003),
    ("fullsize_ksat_wide_64x_t1000.json", 64, 1000, ((3, 4.2), (6, 12.0)), 1006),
])
def test_ksat_batch_workload_full_length(ctx, name, n_inst, T, mix, seed):
    """The batched benchmarks' launch: 256 uneven 3-/4-SAT sets (or 64 3-/6-SAT sets, two list
    entries per occurrence for k = 6), launch shapes tuned on 8 sweeps (states restored), then
    every sweep of every set in one batched launch."""
    g = _golden(name)
    assert g["t1"] == T
    specs = W.workload_ksat_mix(n_inst, T, mix, seed)
    insts, sets = [], []
    for s in specs:
        inst = ctx.load_ksat(s["lits"], s["n"])
        ctx.set_schedule_factored(inst, s["base"], s["factor"])
        insts.append(inst)
        sets.append(ctx.replicas_create(inst, s["R"], seed=s["seed"]))
    ctx.batch_autotune(sets, 0, 8)
    ctx.batch_run(sets, g["t0"], g["t1"])
    checked = {rec["instance"]: rec for rec in g["instances"]}
    for i, (s, rs) in enumerate(zip(specs, sets)):
        if i in checked or i % 16 == 0:
            got = ctx.replicas_read(rs)
            assert np.all(got["best_energies"] <= got["energies"])
            rows = np.arange(0, s["R"], 37)
            assert np.array_equal(O.ksat_energies(s["lits"], s["n"], got["states"][rows]),
                                  got["energies"][rows])
            rec = checked.get(i)
            if rec is not None:
                assert rec["n"] == s["n"] and rec["seed"] == s["seed"] and rec["replicas"] == s["R"]
                for j, r in enumerate(rec["replica_ids"]):
                    assert int(got["energies"][r]) == rec["energies"][j], (i, r)
                    assert int(got["best_energies"][r]) == rec["best_energies"][j], (i, r)
                    assert _digest(got["states"][r]) == rec["states_sha256"][j], (i, r)
                    assert _digest(got["best_states"][r]) == rec["best_states_sha256"][j], (i, r)
        ctx.replicas_destroy(rs)
    for inst in insts:
        ctx.unload(inst)


def test_qap_bench_workload_full_length(ctx):
    g = _golden("fullsize_qap_64x_r4096_t10000.json")
    specs = W.workload_qap_batch()
    sets, insts = [], []
    for s in specs:
        inst = ctx.load_qap(s["F"], s["D"])
        ctx.set_schedule(inst, s["beta"])
        insts.append(inst)
        sets.append(ctx.replicas_create(inst, s["replicas"], seed=s["seed"]))
    ctx.qap_batch_run(sets, g["t0"], g["t1"])  # the bench's launch: all 64 sets at once
    checked = {rec["instance"]: rec for rec in g["instances"]}
    for i, (s, rs) in enumerate(zip(specs, sets)):
        if i in checked or i % 16 == 0:
            got = ctx.replicas_read(rs)
            assert np.all(got["best_energies"] <= got["energies"])
            for r in range(0, s["replicas"], 1021):
                assert int(got["energies"][r]) == O.qap_cost(s["F"], s["D"], got["states"][r])
            rec = checked.get(i)
            if rec is not None:
                assert rec["n"] == s["n"] and rec["seed"] == s["seed"]
                for j, r in enumerate(rec["replica_ids"]):
                    assert int(got["energies"][r]) == rec["energies"][j], (i, r)
                    assert int(got["best_energies"][r]) == rec["best_energies"][j], (i, r)
                    assert _digest(got["states"][r].astype("<i2")) == rec["perms_sha256"][j]
                    assert _digest(got["best_states"][r].astype("<i2")) == rec["best_perms_sha256"][j]
        ctx.replicas_destroy(rs)
    for inst in insts:
        ctx.unload(inst)
