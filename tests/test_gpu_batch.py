"""Batched sweep (many uneven k-SAT replica sets in one launch) against the oracle and
against the single-set path: bit for bit."""
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


@pytest.mark.parametrize("lanes", [1, 4, 8])
def test_uneven_batch_matches_oracle(ctx, monkeypatch, lanes):
    monkeypatch.setenv("NMC_BATCH_LANES", str(lanes))
    specs = [(120, 4.2, 3, 32, 30), (333, 9.6, 4, 70, 30), (57, 9.6, 4, 1, 30),
             (900, 4.2, 3, 96, 30), (64, 2.0, 6, 40, 30), (1500, 9.6, 4, 33, 30)]
    sets, inputs = [], []
    for i, (n, alpha, k, R, T) in enumerate(specs):
        lits = W.random_ksat(n, alpha, k, 50 + i)
        beta = W.beta_inhomogeneous_linear(n, T, 0.5, 4.0, 0.3, 0.5, 60 + i)
        inst = ctx.load_ksat(lits, n)
        ctx.set_schedule(inst, beta)
        rs = ctx.replicas_create(inst, R, seed=70 + i)
        sets.append((inst, rs))
        inputs.append((lits, n, beta, R, T, 70 + i))
    rs_ids = [rs for _, rs in sets]
    # two segments: [0, 12) for all, then [12, T) — segments compose in the batch too
    ctx.batch_run(rs_ids, 0, 12)
    ctx.batch_run(rs_ids, 12, [s[4] for s in specs])
    for (inst, rs), (lits, n, beta, R, T, seed) in zip(sets, inputs):
        got = ctx.replicas_read(rs)
        want = O.ksat_anneal(lits, n, beta, 0, T, seed, replicas=R)
        for key in KEYS:
            assert np.array_equal(got[key], want[key]), (n, key)
        ctx.replicas_destroy(rs)
        ctx.unload(inst)


def test_batch_equals_single_set_path(ctx):
    wl = W.workload_ksat_batch(n_instances=6, n_steps=20, n_min=1000, n_max=6000, seed=77)
    outs_b, outs_s = [], []
    sets = []
    for w in wl:
        inst = ctx.load_ksat(w["lits"], w["n_vars"])
        ctx.set_schedule(inst, w["beta"])
        a = ctx.replicas_create(inst, w["replicas"], seed=w["seed"])
        b = ctx.replicas_create(inst, w["replicas"], seed=w["seed"])
        sets.append((inst, a, b))
    ctx.batch_run([a for _, a, _ in sets], 0, 20)
    for inst, a, b in sets:
        ctx.replicas_run(b, 0, 20)
        ga, gb = ctx.replicas_read(a), ctx.replicas_read(b)
        for key in KEYS:
            assert np.array_equal(ga[key], gb[key]), key
        ctx.replicas_destroy(a)
        ctx.replicas_destroy(b)
        ctx.unload(inst)


def test_batch_rejects(ctx):
    import paper_2111_13628_gb300 as nmc
    lits = W.random_ksat(50, 4.2, 3, 1)
    inst = ctx.load_ksat(lits, 50)
    ctx.set_schedule(inst, W.beta_constant(50, 5, 1.0))
    rs = ctx.replicas_create(inst, 32, seed=1)
    with pytest.raises(nmc.NmcError):
        ctx.batch_run([rs, rs], 0, 2)        # repeated set
    with pytest.raises(nmc.NmcError):
        ctx.batch_run([rs], 0, 6)            # schedule too short
    with pytest.raises(nmc.NmcError):
        ctx.batch_run([rs + 100], 0, 1)      # unknown set
    assert ctx.batch_max_vars() > 40_000
    ctx.replicas_destroy(rs)
    ctx.unload(inst)


@pytest.mark.parametrize("lanes", [1, 4, 8])
@pytest.mark.parametrize("ctas", [1, 2, 4, 8])
def test_cluster_shapes_agree(ctx, monkeypatch, ctas, lanes):
    """One large instance spread over clusters of 1, 2, 4 or 8 CTAs per 32-replica word, with 1,
    4 or 8 lanes per variable, gives the oracle's trajectories (sampled replicas) and the
    grid-kernel path's results."""
    monkeypatch.setenv("NMC_BATCH_CTAS", str(ctas))
    monkeypatch.setenv("NMC_BATCH_LANES", str(lanes))
    n, T, R = 3000, 6, 1024
    lits = W.random_ksat(n, 9.6, 4, 91)
    beta = W.beta_frozen_ramp(n, T, 0.3, 6.0, 0.2, 0.4, 92)
    inst = ctx.load_ksat(lits, n)
    ctx.set_schedule(inst, beta)
    a = ctx.replicas_create(inst, R, seed=93)
    b = ctx.replicas_create(inst, R, seed=93)
    ctx.batch_run([a], 0, T)
    monkeypatch.setenv("NMC_RUN_PATH", "grid")
    ctx.replicas_run(b, 0, T)
    monkeypatch.delenv("NMC_RUN_PATH")
    ga, gb = ctx.replicas_read(a), ctx.replicas_read(b)
    for key in KEYS:
        assert np.array_equal(ga[key], gb[key]), key
    ids = np.array([0, 63, 64, 511, 1000], dtype=np.int32)
    want = O.ksat_anneal(lits, n, beta, 0, T, 93, replica_ids=ids)
    for key in KEYS:
        assert np.array_equal(ga[key][ids], want[key]), key
    ctx.replicas_destroy(a)
    ctx.replicas_destroy(b)
    ctx.unload(inst)


def test_batch_mixes_occurrence_widths_and_segments(ctx):
    """Sets with k <= 4 and k > 4 in one call (two launches), each with its own sweep range."""
    specs = [(200, 9.6, 4, 64, 7, 19), (150, 2.0, 6, 40, 0, 12), (300, 4.2, 3, 33, 3, 3),
             (90, 1.2, 8, 96, 5, 30)]
    sets, data = [], []
    for i, (n, alpha, k, R, t0, t1) in enumerate(specs):
        lits = W.random_ksat(n, alpha, k, 60 + i)
        beta = W.beta_inhomogeneous_linear(n, 30, 0.5, 4.0, 0.3, 0.5, 70 + i)
        inst = ctx.load_ksat(lits, n)
        ctx.set_schedule(inst, beta)
        rs = ctx.replicas_create(inst, R, seed=80 + i)
        sets.append((inst, rs))
        data.append((lits, n, beta, R, t0, t1, 80 + i))
    ctx.batch_run([rs for _, rs in sets], [d[4] for d in data], [d[5] for d in data])
    for (inst, rs), (lits, n, beta, R, t0, t1, seed) in zip(sets, data):
        got = ctx.replicas_read(rs)
        init = O.ksat_anneal(lits, n, beta, 0, 0, seed, replicas=R)
        want = O.ksat_anneal(lits, n, beta, t0, t1, seed, replicas=R, init=init["states"],
                             init_best=init["best_states"], init_best_energy=init["best_energies"])
        for key in KEYS:
            assert np.array_equal(got[key], want[key]), (n, key)
        ctx.replicas_destroy(rs)
        ctx.unload(inst)
