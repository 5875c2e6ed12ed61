"""Held (frozen) units and the collective move on the GPU, through the C ABI, against the CPU
oracle: bit for bit.

Held units (beta = +inf in the schedule) run through every k-SAT kernel shape (one thread per
variable, teams of 4 and 8 lanes, the grid-barrier kernels with 1 and 2 warps per variable) and
the QAP kernels; the collective move runs with shared and per-replica masks, with ragged replica
words, interleaved with sweeps, in replica-exchange runs, and through its argument checks.
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


def _same(got, want, ids=None):
    for k in KEYS:
        g = got[k] if ids is None else got[k][ids]
        assert np.array_equal(g, want[k]), k


def _held_schedule(n, T, seed, frac=0.3):
    """Inhomogeneous profile with a seeded subset held for the first half, another subset held
    for the second half (the alternation of the two-chain scheme)."""
    beta = W.beta_inhomogeneous_linear(n, T, 0.3, 3.0, 0.3, 0.5, seed)
    a = W.seeded_subset(n, frac, seed + 1)
    beta[a, : T // 2] = np.inf
    beta[~a, T // 2:] = np.where(W.seeded_subset(n, 0.5, seed + 2)[~a, None], np.inf,
                                 beta[~a, T // 2:])
    return beta


@pytest.mark.parametrize("shape", ["lanes1", "lanes4", "lanes8", "grid"])
def test_held_variables_every_kernel(ctx, monkeypatch, shape):
    if shape == "grid":
        monkeypatch.setenv("NMC_RUN_PATH", "grid")
    else:
        monkeypatch.setenv("NMC_BATCH_LANES", shape[5:])
    n, T, R = 700, 24, 70
    lits = W.random_ksat(n, 9.6, 4, 41)
    beta = _held_schedule(n, T, 5)
    inst = ctx.load_ksat(lits, n)
    ctx.set_schedule(inst, beta)
    got = ctx.anneal(inst, R, 0, T, 13)
    ctx.unload(inst)
    want = O.ksat_anneal(lits, n, beta, 0, T, 13, replicas=R)
    _same(got, want)


@pytest.mark.parametrize("warps", [1, 2])
def test_held_variables_fast_grid_kernel(ctx, monkeypatch, warps):
    monkeypatch.setenv("NMC_RUN_PATH", "grid")
    monkeypatch.setenv("NMC_SWEEP_WARPS", str(warps))
    n, T, R = 400, 10, 1024
    lits = W.random_ksat(n, 9.6, 4, 42)
    beta = _held_schedule(n, T, 6)
    inst = ctx.load_ksat(lits, n)
    ctx.set_schedule(inst, beta)
    got = ctx.anneal(inst, R, 0, T, 17)
    ctx.unload(inst)
    ids = np.array([0, 1, 31, 32, 500, 1023])
    want = O.ksat_anneal(lits, n, beta, 0, T, 17, replica_ids=ids)
    _same(got, want, ids)


def test_held_factored_schedule(ctx):
    n, T = 300, 16
    lits = W.random_ksat(n, 4.2, 3, 43)
    base = W.linear_profile(0.5, 2.0, T).astype(np.float32)
    factor = np.where(W.seeded_subset(n, 0.25, 3), np.inf, 1.0).astype(np.float32)
    inst = ctx.load_ksat(lits, n)
    ctx.set_schedule_factored(inst, base, factor)
    got = ctx.anneal(inst, 64, 0, T, 2)
    ctx.unload(inst)
    beta = (base[None, :] * factor[:, None]).astype(np.float32)
    _same(got, O.ksat_anneal(lits, n, beta, 0, T, 2, replicas=64))


@pytest.mark.parametrize("n", [7, 40, 200])
def test_held_qap_facilities(ctx, n):
    F, D = W.random_qap(n, 300 + n)
    T, R = 12, 64
    beta = W.beta_scaled_linear(n, T, 0.01, 1.0, 0.5, 1.5, 9)
    beta[W.seeded_subset(n, 0.3, 4), : T // 2] = np.inf
    inst = ctx.load_qap(F, D)
    ctx.set_schedule(inst, beta)
    got = ctx.anneal(inst, R, 0, T, 3)
    ctx.unload(inst)
    want = O.qap_anneal(F, D, beta, 0, T, 3, replicas=R)
    for k in ("perms", "energies", "best_energies", "best_perms"):
        g = got["states" if k == "perms" else "best_states" if k == "best_perms" else k]
        assert np.array_equal(g, want[k]), k


def _oracle_chain(lits, n, beta, R, seed, plan):
    """Applies plan = [("sweep", t0, t1) | ("flip", mask, beta_r, move_id)] with the oracle."""
    ch = None
    for step in plan:
        if step[0] == "sweep":
            _, t0, t1 = step
            if ch is None:
                ch = O.ksat_anneal(lits, n, beta, t0, t1, seed, replicas=R)
            else:
                ch = O.ksat_anneal(lits, n, beta, t0, t1, seed, replicas=R, init=ch["states"],
                                   init_best=ch["best_states"],
                                   init_best_energy=ch["best_energies"])
        else:
            _, mask, b, mid = step
            if ch is None:
                ch = O.ksat_anneal(lits, n, beta, 0, 0, seed, replicas=R)
            ch = O.ksat_cluster_flip(lits, n, ch, mask, b, mid, seed)
    return ch


def test_cluster_moves_interleaved_with_sweeps(ctx):
    n, T, R = 500, 20, 70
    lits = W.random_ksat(n, 9.6, 4, 51)
    beta = W.beta_inhomogeneous_linear(n, T, 0.5, 3.0, 0.3, 0.5, 7)
    rng = np.random.default_rng(8)
    shared = (rng.random(n) < 0.2).astype(np.uint8)
    per = (rng.random((R, n)) < 0.1).astype(np.uint8)
    betas = np.linspace(0.2, 3.0, R).astype(np.float32)
    plan = [("flip", shared, betas, 0), ("sweep", 0, 7), ("flip", per, betas, 1),
            ("flip", shared, np.float32(0.7), 2), ("sweep", 7, 20), ("flip", per, betas, 3)]
    want = _oracle_chain(lits, n, beta, R, 19, plan)
    inst = ctx.load_ksat(lits, n)
    ctx.set_schedule(inst, beta)
    rs = ctx.replicas_create(inst, R, 19)
    accs = []
    for step in plan:
        if step[0] == "sweep":
            ctx.replicas_run(rs, step[1], step[2])
        else:
            accs.append(ctx.cluster_flip(rs, step[1], step[2], step[3], accepted=True))
    got = ctx.replicas_read(rs)
    ctx.replicas_destroy(rs)
    ctx.unload(inst)
    _same(got, want)
    assert any(a.any() for a in accs) and not all(a.all() for a in accs)


def test_cluster_move_accepts_like_the_oracle(ctx):
    n, R = 300, 4096
    lits = W.random_ksat(n, 4.2, 3, 52)
    mask = (np.random.default_rng(2).random(n) < 0.05).astype(np.uint8)
    inst = ctx.load_ksat(lits, n)
    rs = ctx.replicas_create(inst, R, 23)
    ch = None
    for mid, b in enumerate([0.0, 0.4, 2.0, 65535.0]):
        acc = ctx.cluster_flip(rs, mask, b, 100 + mid, accepted=True)
        if ch is None:
            ch = O.ksat_anneal(lits, n, W.beta_constant(n, 1, 1.0), 0, 0, 23, replicas=R)
        ch = O.ksat_cluster_flip(lits, n, ch, mask, b, 100 + mid, 23)
        assert np.array_equal(acc, ch["accepted"]), b
    got = ctx.replicas_read(rs)
    ctx.replicas_destroy(rs)
    ctx.unload(inst)
    _same(got, ch)


def test_cluster_move_inside_replica_exchange(ctx):
    wl = W.workload_ksat_small(30)
    lits, n, beta = wl["lits"], wl["n_vars"], wl["beta"]
    L, G = 16, 4
    ladder = W.geometric_profile(0.4, 2.5, L).astype(np.float32)
    mask = W.seeded_subset(n, 0.15, 3).astype(np.uint8)
    inst = ctx.load_ksat(lits, n)
    ctx.set_schedule(inst, beta)
    rs = ctx.replicas_create(inst, G * L, wl["seed"])
    ctx.set_ladder(rs, ladder)
    ctx.run_pt(rs, 0, 12, 4)
    slots = ctx.read_slots(rs)
    ctx.cluster_flip(rs, mask, ladder[slots], 5)
    ctx.run_pt(rs, 12, 30, 4)
    got = ctx.replicas_read(rs)
    got["slots"] = ctx.read_slots(rs)
    ctx.replicas_destroy(rs)
    ctx.unload(inst)
    a = O.ksat_pt_anneal(lits, n, beta, ladder, 0, 12, 4, wl["seed"], replicas=G * L)
    f = O.ksat_cluster_flip(lits, n, a, mask, ladder[a["slots"]], 5, wl["seed"])
    b = O.ksat_pt_anneal(lits, n, beta, ladder, 12, 30, 4, wl["seed"], replicas=G * L,
                         slots=a["slots"], init=f["states"], init_best=f["best_states"],
                         init_best_energy=f["best_energies"])
    _same(got, b)
    assert np.array_equal(got["slots"], b["slots"])


def test_cluster_move_argument_checks(ctx):
    import paper_2111_13628_gb300 as nmc
    n = 50
    inst = ctx.load_ksat(W.random_ksat(n, 4.2, 3, 1), n)
    rs = ctx.replicas_create(inst, 40, 1)
    for mask, b in [(np.zeros((3, n), np.uint8), 1.0),      # 3 rows: neither 1 nor R
                    (np.full((1, n), 2, np.uint8), 1.0),    # not 0/1
                    (np.zeros((1, n), np.uint8), np.inf),   # beta not finite
                    (np.zeros((1, n), np.uint8), -0.5)]:
        with pytest.raises(nmc.NmcError) as e:
            ctx.cluster_flip(rs, mask, b, 0)
        assert e.value.code == nmc.NMC_EINVAL
    ctx.replicas_destroy(rs)
    F, D = W.random_qap(6, 1)
    q = ctx.load_qap(F, D)
    qs = ctx.replicas_create(q, 8, 1)
    with pytest.raises(nmc.NmcError) as e:
        ctx._check(ctx._lib.nmc_replicas_cluster_flip(ctx._h, qs, 1, np.zeros(6, np.uint8).ctypes.data,
                                                      np.ones(8, np.float32).ctypes.data, 0, None))
    assert e.value.code == nmc.NMC_EINVAL
    ctx.replicas_destroy(qs)
    ctx.unload(q)
    ctx.unload(inst)
