"""The next-step paths at the sizes and launch configurations `bench.py` times, against the
oracle on outputs it can reproduce one by one (or one ladder / one seed at a time).

* replica exchange: 4-SAT N = 5,000, alpha 9.884, 32 ladders x 32 temperatures, exchange every 10
  sweeps; ladder 0 (replicas 0..31) evolves independently of the other ladders, so the oracle
  runs it alone and must match bit for bit;
* LBP: 64 seeds of the same instance at once; seeds 0 and 63 are recomputed by the oracle
  (tolerance 1e-9, derived in test_gpu_lbp.py);
* two-chain sampling, collective move and whitening on the 50,000-variable instance with 1,024
  replicas: sampled replicas bit for bit.

The replica-exchange and two-chain runs are checked twice: on short schedules against the oracle
run here, and at the benchmark's full length (2,000 sweeps with 200 exchange rounds; 500 held-
sampling sweeps) against oracle outputs stored by `tests/golden/make_fullsize.py`.
"""
import numpy as np
import pytest

import nmc_inputs as W
import oracle as O

pytestmark = pytest.mark.gpu
KEYS = ("states", "energies", "best_energies", "best_states")


@pytest.fixture(scope="module")
def ctx():
    import paper_2111_13628_gb300 as nmc
    c = nmc.Context(0)
    yield c
    c.close()


def test_replica_exchange_bench_configuration(ctx):
    n, T, L, G, per = 5000, 60, 32, 32, 10
    lits = W.random_ksat(n, 9.884, 4, 2111)
    ladder = W.geometric_profile(0.5, 5.0, L).astype(np.float32)
    beta = np.ones((n, T), np.float32)
    inst = ctx.load_ksat(lits, n)
    ctx.set_schedule_factored(inst, np.ones(T, np.float32), np.ones(n, np.float32))
    rs = ctx.replicas_create(inst, G * L, 1)
    ctx.set_ladder(rs, ladder)
    ctx.run_pt(rs, 0, T, per)
    got = ctx.replicas_read(rs)
    slots = ctx.read_slots(rs)
    ctx.replicas_destroy(rs)
    ctx.unload(inst)
    want = O.ksat_pt_anneal(lits, n, beta, ladder, 0, T, per, 1, replicas=L)
    for k in KEYS:
        assert np.array_equal(got[k][:L], want[k]), k
    assert np.array_equal(slots[:L], want["slots"])
    for g in range(G):
        assert sorted(slots[g * L:(g + 1) * L].tolist()) == list(range(L))


def test_lbp_bench_configuration(ctx):
    n, S = 5000, 64
    lits = W.random_ksat(n, 9.884, 4, 2111)
    inst = ctx.load_ksat(lits, n)
    ctx.set_schedule(inst, W.beta_constant(n, 200, 3.0))
    seeds = ctx.anneal(inst, S, 0, 200, 5)["best_states"]
    lams = [0.4, 0.2, 0.1, 0.05, 0.025]
    got = ctx.cnf_lbp(inst, seeds, 1.0, lams, 1e-8, 100)
    ctx.unload(inst)
    for s in (0, S - 1):
        want = O.cnf_lbp(lits, n, seeds[s], 1.0, lams, 1e-8, 100)
        assert got["n_done"][s] == want["n_done"]
        assert np.array_equal(got["iters"][s], want["iters"])
        assert np.allclose(got["marg"][s], want["marg"], atol=1e-9, rtol=0)
        assert np.allclose(got["corr"][s], want["corr"], atol=1e-9, rtol=0)


def test_two_chain_flip_and_whitening_bench_instance(ctx):
    wl = W.workload_ksat_large(n_steps=2)
    lits, n, R = wl["lits"], wl["n_vars"], 1024
    labels = np.where(W.seeded_subset(n, 0.2, 77), 0, -1).astype(np.int32)
    cycles, th, tc, tu = 1, 12, 12, 6
    inst = ctx.load_ksat(lits, n)
    ctx.set_schedule_backbone(inst, labels, cycles, th, tc, tu, 3.0, 4.0)
    rs = ctx.replicas_create(inst, R, 1)
    ctx.replicas_run(rs, 0, th + tc + tu)
    mask = (labels >= 0).astype(np.uint8)
    acc = ctx.cluster_flip(rs, mask, np.full(R, 0.75, np.float32), 1000, accepted=True)
    got = ctx.replicas_read(rs)
    frozen = ctx.whitening(rs, use_best=True)
    ctx.replicas_destroy(rs)
    ctx.unload(inst)
    beta = O.backbone_schedule(labels, 3.0, 4.0, cycles, th, tc, tu)
    ids = np.array([0, 517, 1023])
    ch = O.ksat_anneal(lits, n, beta, 0, th + tc + tu, 1, replica_ids=ids)
    mv = O.ksat_cluster_flip(lits, n, ch, mask, np.full(3, 0.75, np.float32), 1000, 1,
                             replica_ids=ids)
    for j, r in enumerate(ids):
        assert acc[r] == mv["accepted"][j]
        for k in KEYS:
            assert np.array_equal(got[k][r], mv[k][j]), (r, k)
        wf, wc = O.ksat_whitening(lits, n, mv["best_states"][j])
        assert frozen[r] == wc


def _golden(name):
    import json
    import os
    with open(os.path.join(os.path.dirname(os.path.abspath(__file__)), "golden", name)) as f:
        return json.load(f)


def _digest(a):
    import hashlib
    return hashlib.sha256(np.ascontiguousarray(a).tobytes()).hexdigest()


def _same_as_golden(got, g, r, j):
    assert int(got["energies"][r]) == g["energies"][j], r
    assert int(got["best_energies"][r]) == g["best_energies"][j], r
    assert _digest(got["states"][r]) == g["states_sha256"][j], r
    assert _digest(got["best_states"][r]) == g["best_states_sha256"][j], r


def test_replica_exchange_bench_configuration_full_length(ctx):
    """All 2,000 sweeps and 200 exchange rounds of the benchmark's replica-exchange run against
    the oracle's stored outputs for ladder 0 (tests/golden/make_fullsize.py pt)."""
    g = _golden("fullsize_pt_4sat_n5000_32x32_t2000.json")
    n, T, L, G, per = 5000, g["t1"], 32, 32, g["per"]
    lits = W.random_ksat(n, 9.884, 4, 2111)
    ladder = W.geometric_profile(0.5, 5.0, L).astype(np.float32)
    inst = ctx.load_ksat(lits, n)
    ctx.set_schedule_factored(inst, np.ones(T, np.float32), np.ones(n, np.float32))
    rs = ctx.replicas_create(inst, G * L, 1)
    ctx.set_ladder(rs, ladder)
    ctx.run_pt(rs, 0, T, per)
    got = ctx.replicas_read(rs)
    slots = ctx.read_slots(rs)
    ctx.replicas_destroy(rs)
    ctx.unload(inst)
    for j, r in enumerate(g["replica_ids"]):
        _same_as_golden(got, g, r, j)
    assert slots[:L].tolist() == g["slots"]
    for lg in range(G):
        assert sorted(slots[lg * L:(lg + 1) * L].tolist()) == list(range(L))
    assert np.all(got["best_energies"] <= got["energies"])
    rows = np.arange(0, G * L, 53)
    assert np.array_equal(O.ksat_energies(lits, n, got["states"][rows]), got["energies"][rows])


def test_two_chain_flip_and_whitening_full_length(ctx):
    """The benchmark's 500 held-sampling sweeps (10 cycles), then the collective flip of the
    backbone and whitening, against the oracle's stored outputs (make_fullsize.py moves)."""
    g = _golden("fullsize_moves_4sat_n50000_r1024_t500.json")
    wl = W.workload_ksat_large(n_steps=2)
    lits, n, R = wl["lits"], wl["n_vars"], 1024
    labels = np.where(W.seeded_subset(n, 0.2, 77), 0, -1).astype(np.int32)
    inst = ctx.load_ksat(lits, n)
    ctx.set_schedule_backbone(inst, labels, 10, 20, 20, 10, 3.0, 4.0)
    rs = ctx.replicas_create(inst, R, 1)
    ctx.replicas_run(rs, g["t0"], g["t1"])
    chain = ctx.replicas_read(rs)
    mask = (labels >= 0).astype(np.uint8)
    acc = ctx.cluster_flip(rs, mask, np.full(R, 0.75, np.float32), 1000, accepted=True)
    got = ctx.replicas_read(rs)
    frozen = ctx.whitening(rs, use_best=True)
    ctx.replicas_destroy(rs)
    ctx.unload(inst)
    for j, r in enumerate(g["replica_ids"]):
        _same_as_golden(chain, g["chain"], r, j)
        _same_as_golden(got, g, r, j)
        assert int(acc[r]) == g["accepted"][j]
        assert int(frozen[r]) == g["frozen"][j]
    assert np.all(got["best_energies"] <= got["energies"])
