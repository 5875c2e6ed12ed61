"""Replica exchange and the adaptive ladder on the GPU, through the C ABI, against the CPU
oracle: bit for bit (states, energies, best-so-far, slots; the ladders' doubles exactly, k-SAT
and QAP).

Cases span several colour classes, several replica words with a ragged last word, both
occurrence widths (k <= 4 and k <= 8), exchange rounds that straddle run boundaries, and the
argument checks of the entry points.
"""
import numpy as np
import pytest

import nmc_inputs as W
import oracle as O

pytestmark = pytest.mark.gpu

KEYS = ("states", "energies", "best_energies", "best_states", "slots")


@pytest.fixture(scope="module")
def ctx():
    import paper_2111_13628_gb300 as nmc
    c = nmc.Context(0)
    yield c
    c.close()


def _gpu_pt(ctx, lits, n, beta, ladder, R, seed, runs, per, slots=None):
    inst = ctx.load_ksat(lits, n)
    ctx.set_schedule(inst, beta)
    rs = ctx.replicas_create(inst, R, seed)
    ctx.set_ladder(rs, ladder, slots)
    for t0, t1 in runs:
        ctx.run_pt(rs, t0, t1, per)
    out = ctx.replicas_read(rs)
    out["slots"] = ctx.read_slots(rs)
    ctx.replicas_destroy(rs)
    ctx.unload(inst)
    return out


def _same(got, want):
    for k in KEYS:
        assert np.array_equal(got[k], want[k]), k


@pytest.mark.parametrize("L,G,per,T", [(16, 4, 3, 40), (20, 4, 1, 25), (12, 1, 5, 33)])
def test_pt_parity_inhomogeneous_profile(ctx, L, G, per, T):
    wl = W.workload_ksat_small(T)
    ladder = W.geometric_profile(0.4, 2.5, L).astype(np.float32)
    got = _gpu_pt(ctx, wl["lits"], wl["n_vars"], wl["beta"], ladder, G * L, wl["seed"],
                  [(0, T)], per)
    want = O.ksat_pt_anneal(wl["lits"], wl["n_vars"], wl["beta"], ladder, 0, T, per,
                            wl["seed"], replicas=G * L)
    _same(got, want)
    assert not np.array_equal(got["slots"], np.arange(G * L) % L)


def test_pt_segments_and_given_slots(ctx):
    n = 500
    lits = W.random_ksat(n, 9.6, 4, 17)
    T = 30
    beta = W.beta_inhomogeneous_linear(n, T, 0.5, 3.0, 0.3, 0.5, seed=4)
    L, G = 10, 7  # R = 70: three words, the last one ragged
    ladder = W.geometric_profile(0.3, 3.0, L).astype(np.float32)
    rng = np.random.default_rng(2)
    slots = np.concatenate([rng.permutation(L) for _ in range(G)]).astype(np.int32)
    got = _gpu_pt(ctx, lits, n, beta, ladder, G * L, 11, [(0, 7), (7, 8), (8, 19), (19, 30)], 4,
                  slots=slots)
    want = O.ksat_pt_anneal(lits, n, beta, ladder, 0, T, 4, 11, replicas=G * L, slots=slots)
    _same(got, want)


def test_pt_wide_clauses(ctx):
    """Clauses of up to 6 literals use the two-word occurrence layout."""
    n = 300
    lits = W.random_ksat(n, 3.0, 6, 5)
    T = 20
    beta = W.beta_constant(n, T, 1.0)
    ladder = np.linspace(0.5, 4.0, 8).astype(np.float32)
    got = _gpu_pt(ctx, lits, n, beta, ladder, 64, 3, [(0, T)], 2)
    want = O.ksat_pt_anneal(lits, n, beta, ladder, 0, T, 2, 3, replicas=64)
    _same(got, want)


def test_pt_equal_ladder_matches_plain_run(ctx):
    wl = W.workload_ksat_small(20)
    R = 64
    got = _gpu_pt(ctx, wl["lits"], wl["n_vars"], wl["beta"], np.ones(16, np.float32), R,
                  wl["seed"], [(0, 20)], 2)
    inst = ctx.load_ksat(wl["lits"], wl["n_vars"])
    ctx.set_schedule(inst, wl["beta"])
    plain = ctx.anneal(inst, R, 0, 20, wl["seed"])
    ctx.unload(inst)
    for k in ("states", "energies", "best_energies", "best_states"):
        assert np.array_equal(got[k], plain[k]), k


def test_adaptive_ladder_parity(ctx):
    n = 400
    lits = W.random_ksat(n, 9.6, 4, 23)
    inst = ctx.load_ksat(lits, n)
    args = (96, 7, 0.05, 1.1, 2.0, 10, 6, 10)
    betas, sigmas = ctx.adaptive_ladder(inst, *args)
    ctx.unload(inst)
    ob, osg = O.adaptive_ladder(lits, n, *args)
    assert len(betas) >= 3
    assert np.array_equal(betas, ob) and np.array_equal(sigmas, osg)


@pytest.mark.parametrize("n,R", [(24, 70), (100, 40)])
def test_qap_adaptive_ladder_parity(ctx, n, R):
    """QAP ladder: per-replica double cost sums in the kernel (a ragged last 32-replica block),
    the one-thread sequential sum over replicas; betas and sigmas equal to the last bit."""
    F, D = W.random_qap(n, 900 + n)
    inst = ctx.load_qap(F, D)
    args = (R, 13, 0.0005, 0.9, 1.0, 6, 5, 9)
    betas, sigmas = ctx.adaptive_ladder(inst, *args)
    ctx.unload(inst)
    ob, osg = O.qap_adaptive_ladder(F, D, *args)
    assert len(betas) >= 3
    assert np.array_equal(betas, ob) and np.array_equal(sigmas, osg)


def test_pt_argument_checks(ctx):
    import paper_2111_13628_gb300 as nmc
    wl = W.workload_ksat_small(10)
    inst = ctx.load_ksat(wl["lits"], wl["n_vars"])
    ctx.set_schedule(inst, wl["beta"])
    rs = ctx.replicas_create(inst, 48, 1)
    with pytest.raises(nmc.NmcError) as e:
        ctx.run_pt(rs, 0, 5, 1)  # no ladder yet
    assert e.value.code == nmc.NMC_ESTATE
    with pytest.raises(nmc.NmcError) as e:
        ctx.set_ladder(rs, np.ones(10, np.float32))  # 48 % 10 != 0
    assert e.value.code == nmc.NMC_EINVAL
    with pytest.raises(nmc.NmcError) as e:
        ctx.set_ladder(rs, np.array([1.0, np.nan, 2.0], np.float32))
    assert e.value.code == nmc.NMC_EINVAL
    bad = np.zeros(48, np.int32)  # not a permutation per ladder
    with pytest.raises(nmc.NmcError) as e:
        ctx.set_ladder(rs, np.ones(12, np.float32), bad)
    assert e.value.code == nmc.NMC_EINVAL
    ctx.set_ladder(rs, np.ones(12, np.float32))
    with pytest.raises(nmc.NmcError) as e:
        ctx.run_pt(rs, 0, 5, 0)
    assert e.value.code == nmc.NMC_EINVAL
    with pytest.raises(nmc.NmcError) as e:
        ctx.run_pt(rs, 0, 11, 1)  # schedule has 10 steps
    assert e.value.code == nmc.NMC_ESTATE
    with pytest.raises(nmc.NmcError) as e:
        ctx.adaptive_ladder(inst, 32, 1, 0.1, 1.1, -1.0, 4, 2, 2)
    assert e.value.code == nmc.NMC_EINVAL
    ctx.replicas_destroy(rs)
    ctx.unload(inst)


@pytest.mark.parametrize("n,L,G,per", [(24, 8, 4, 2), (100, 16, 2, 3), (200, 12, 3, 1)])
def test_qap_pt_parity(ctx, n, L, G, per):
    """QAP replica exchange: launch shapes of 2 and 7 facilities per lane on 16 lanes and of 7 on
    32 lanes, several ladders, exchange rounds between and across run boundaries."""
    F, D = W.random_qap(n, 700 + n)
    T = 14
    beta = W.beta_scaled_linear(n, T, 0.01, 1.0, 0.5, 1.5, 9)
    ladder = W.geometric_profile(0.1, 3.0, L).astype(np.float32)
    R = G * L
    inst = ctx.load_qap(F, D)
    ctx.set_schedule(inst, beta)
    rs = ctx.replicas_create(inst, R, 21)
    ctx.set_ladder(rs, ladder)
    ctx.run_pt(rs, 0, 5, per)
    ctx.run_pt(rs, 5, T, per)
    got = ctx.replicas_read(rs)
    slots = ctx.read_slots(rs)
    ctx.replicas_destroy(rs)
    ctx.unload(inst)
    want = O.qap_pt_anneal(F, D, beta, ladder, 0, T, per, 21, replicas=R)
    for a, b in (("states", "perms"), ("energies", "energies"), ("best_energies", "best_energies"),
                 ("best_states", "best_perms")):
        assert np.array_equal(got[a], want[b]), a
    assert np.array_equal(slots, want["slots"])


def test_pt_checkpoint_resume(ctx):
    """A replica-exchange run read back after [0, 13) (states, best states, slots) and restored
    into a fresh set of the same instance and seed continues exactly: [13, 30) there equals the
    uninterrupted [0, 30)."""
    wl = W.workload_ksat_small(30)
    lits, n, beta = wl["lits"], wl["n_vars"], wl["beta"]
    L, G, per = 16, 4, 3
    ladder = W.geometric_profile(0.4, 2.5, L).astype(np.float32)
    inst = ctx.load_ksat(lits, n)
    ctx.set_schedule(inst, beta)
    a = ctx.replicas_create(inst, G * L, 8)
    ctx.set_ladder(a, ladder)
    ctx.run_pt(a, 0, 13, per)
    ck = ctx.replicas_read(a)
    ck_slots = ctx.read_slots(a)
    ctx.run_pt(a, 13, 30, per)
    full = ctx.replicas_read(a)
    full["slots"] = ctx.read_slots(a)
    b = ctx.replicas_create(inst, G * L, 8)
    ctx.replicas_restore(b, ck)
    ctx.set_ladder(b, ladder, ck_slots)
    ctx.run_pt(b, 13, 30, per)
    got = ctx.replicas_read(b)
    got["slots"] = ctx.read_slots(b)
    ctx.replicas_destroy(a)
    ctx.replicas_destroy(b)
    ctx.unload(inst)
    _same(got, full)
