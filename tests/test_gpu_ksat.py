"""k-SAT sweep on the GPU, through the C ABI, against the CPU oracle: bit for bit.

Every output is integer (0/1 states, energies), so the tolerance is zero. Sizes span several
colour classes, several replica words and a ragged last word; the full-size case runs the
launch configuration the bench times and compares sampled replicas, whose trajectories the
oracle reproduces one by one.
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


def _run(ctx, lits, n, beta, R, t0, t1, seed, init=None):
    inst = ctx.load_ksat(lits, n)
    ctx.set_schedule(inst, beta)
    out = ctx.anneal(inst, R, t0, t1, seed, init=init)
    ctx.unload(inst)
    return out


def _same(got, want, ids=None):
    for k in KEYS:
        g = got[k] if ids is None else got[k][ids]
        assert np.array_equal(g, want[k]), k


def test_colouring_matches_oracle(ctx):
    for n, alpha, k, seed in [(200, 9.6, 4, 1), (1000, 4.2, 3, 2), (300, 3.0, 6, 3)]:
        lits = W.random_ksat(n, alpha, k, seed)
        inst = ctx.load_ksat(lits, n)
        col, nc = ctx.ksat_colouring(inst)
        ocol, onc = O.ksat_colour(lits, n)
        assert nc == onc and np.array_equal(col, ocol)
        ctx.unload(inst)


def test_small_workload_full_parity(ctx):
    wl = W.workload_ksat_small(1000)
    got = _run(ctx, wl["lits"], wl["n_vars"], wl["beta"], wl["replicas"], 0, 1000, wl["seed"])
    want = O.ksat_anneal(wl["lits"], wl["n_vars"], wl["beta"], 0, 1000, wl["seed"],
                         replicas=wl["replicas"])
    _same(got, want)


@pytest.fixture(params=["auto", "grid"])
def run_path(request, monkeypatch):
    """Runs a test through the default kernel choice and through the grid-barrier kernel."""
    if request.param == "grid":
        monkeypatch.setenv("NMC_RUN_PATH", "grid")
    return request.param


@pytest.mark.parametrize("n,alpha,k,R,T", [
    (1, 0.0, 1, 5, 7),          # one variable, no clauses
    (2, 1.0, 2, 1, 9),          # single replica
    (37, 4.2, 3, 33, 25),       # ragged second word
    (150, 9.6, 4, 95, 30),      # three words, ragged
    (400, 9.6, 4, 256, 12),     # eight words
    (120, 2.0, 6, 40, 15),      # k > 4: two int4 per occurrence
    (90, 1.2, 8, 64, 10),       # k = 8
])
def test_parity_shapes(ctx, run_path, n, alpha, k, R, T):
    lits = W.random_ksat(n, alpha, k, 100 + n) if alpha > 0 else np.zeros((0, k), np.int32)
    beta = W.beta_inhomogeneous_linear(n, T, 0.2, 3.0, 0.3, 0.5, 200 + n)
    got = _run(ctx, lits, n, beta, R, 0, T, seed=5 + n)
    want = O.ksat_anneal(lits, n, beta, 0, T, 5 + n, replicas=R)
    _same(got, want)


def test_padded_clauses_and_high_degree(ctx, run_path):
    rng = np.random.default_rng(4)
    n, m, kmax = 60, 900, 5
    rows = np.zeros((m, kmax), np.int32)
    for a in range(m):
        kk = int(rng.integers(1, kmax + 1))
        v = rng.choice(n, size=kk, replace=False) + 1
        if a % 4 != 3 and 0 not in (v - 1):
            v[0] = 1  # variable 0 occurs in most clauses: degree > 511 -> 10-bit counters
        rows[a, :kk] = v * rng.choice([-1, 1], size=kk)
    deg0 = int((np.abs(rows) == 1).sum())
    assert deg0 > 511
    beta = W.beta_inhomogeneous_linear(n, 20, 0.1, 2.0, 0.3, 0.5, 9)
    got = _run(ctx, rows, n, beta, 50, 0, 20, seed=3)
    want = O.ksat_anneal(rows, n, beta, 0, 20, 3, replicas=50)
    _same(got, want)


def test_segments_resident_state_and_given_init(ctx, run_path):
    wl = W.workload_ksat_small(80)
    lits, n, beta = wl["lits"], wl["n_vars"], wl["beta"]
    inst = ctx.load_ksat(lits, n)
    ctx.set_schedule(inst, beta)
    rs = ctx.replicas_create(inst, 70, seed=9)
    for t0, t1 in [(0, 13), (13, 13), (13, 50), (50, 80)]:
        ctx.replicas_run(rs, t0, t1)
    got = ctx.replicas_read(rs)
    ctx.replicas_destroy(rs)
    want = O.ksat_anneal(lits, n, beta, 0, 80, 9, replicas=70)
    _same(got, want)
    init = np.random.default_rng(1).integers(0, 2, size=(70, n), dtype=np.uint8)
    got = ctx.anneal(inst, 70, 20, 80, seed=9, init=init)
    want = O.ksat_anneal(lits, n, beta, 20, 80, 9, replicas=70, init=init)
    _same(got, want)
    ctx.unload(inst)


def test_beta_zero_and_infinite(ctx, run_path):
    n = 300
    lits = W.random_ksat(n, 9.6, 4, 77)
    for val in (0.0, 65535.0):
        beta = W.beta_constant(n, 6, val)
        got = _run(ctx, lits, n, beta, 64, 0, 6, seed=1)
        want = O.ksat_anneal(lits, n, beta, 0, 6, 1, replicas=64)
        _same(got, want)


def test_device_outputs_and_device_schedule(ctx):
    import torch
    wl = W.workload_ksat_small(50)
    lits, n, beta = wl["lits"], wl["n_vars"], wl["beta"]
    inst = ctx.load_ksat(lits, n)
    ctx.set_schedule(inst, torch.from_numpy(beta).cuda())
    rs = ctx.replicas_create(inst, 64, seed=1)
    ctx.replicas_run(rs, 0, 50)
    dev = dict(states=torch.zeros((64, n), dtype=torch.uint8, device="cuda"),
               energies=torch.zeros(64, dtype=torch.int64, device="cuda"),
               best_energies=torch.zeros(64, dtype=torch.int64, device="cuda"),
               best_states=torch.zeros((64, n), dtype=torch.uint8, device="cuda"))
    ctx.replicas_read_device(rs, **dev)
    ctx.sync()
    want = O.ksat_anneal(lits, n, beta, 0, 50, 1, replicas=64)
    _same({k: v.cpu().numpy() for k, v in dev.items()}, want)
    ctx.replicas_destroy(rs)
    ctx.unload(inst)


def test_rejects_bad_input(ctx):
    import paper_2111_13628_gb300 as nmc
    bad = [np.array([[1, -1, 2]], np.int32),       # variable twice
           np.array([[0, 0, 0]], np.int32),        # empty clause
           np.array([[1, 2, 9]], np.int32)]        # out of range
    for lits in bad:
        with pytest.raises(nmc.NmcError) as e:
            ctx.load_ksat(lits, 5)
        assert e.value.code == nmc.NMC_EINVAL
    lits = W.random_ksat(20, 4.2, 3, 1)
    inst = ctx.load_ksat(lits, 20)
    for v in (np.nan, -1.0, 70000.0, -np.inf):  # +inf is valid: the variable is held
        beta = W.beta_constant(20, 4, 1.0)
        beta[3, 2] = v
        with pytest.raises(nmc.NmcError) as e:
            ctx.set_schedule(inst, beta)
        assert e.value.code == nmc.NMC_EINVAL
    rs = ctx.replicas_create(inst, 8, seed=1)
    with pytest.raises(nmc.NmcError) as e:
        ctx.replicas_run(rs, 0, 3)           # no schedule yet
    assert e.value.code == nmc.NMC_ESTATE
    ctx.set_schedule(inst, W.beta_constant(20, 4, 1.0))
    with pytest.raises(nmc.NmcError) as e:
        ctx.replicas_run(rs, 0, 5)           # schedule too short
    assert e.value.code == nmc.NMC_ESTATE
    with pytest.raises(nmc.NmcError):
        ctx.unload(inst)                     # replica set still alive
    ctx.replicas_destroy(rs)
    with pytest.raises(nmc.NmcError):
        ctx.replicas_create(inst, 4097, seed=1)
    ctx.unload(inst)


def test_bounded_wait_expires_and_context_survives(ctx):
    import paper_2111_13628_gb300 as nmc
    assert ctx.selftest_wait_timeout(300) == nmc.NMC_ETIMEOUT
    lits = W.random_ksat(50, 4.2, 3, 2)
    beta = W.beta_constant(50, 3, 1.0)
    got = _run(ctx, lits, 50, beta, 32, 0, 3, seed=2)
    want = O.ksat_anneal(lits, 50, beta, 0, 3, 2, replicas=32)
    _same(got, want)


def test_full_size_sampled_replicas(ctx, run_path):
    """The N=50,000 / 1024-replica workload in the bench's launch configuration: every replica
    is checked for energy consistency, and sampled replicas bit for bit (short schedule)."""
    T = 40
    wl = W.workload_ksat_large(n_steps=T)
    lits, n, beta, R = wl["lits"], wl["n_vars"], wl["beta"], wl["replicas"]
    inst = ctx.load_ksat(lits, n)
    ctx.set_schedule(inst, beta)
    rs = ctx.replicas_create(inst, R, seed=wl["seed"])
    ctx.replicas_run(rs, 0, T)
    got = ctx.replicas_read(rs)
    ctx.replicas_destroy(rs)
    ctx.unload(inst)
    ids = np.array([0, 31, 32, 517, 1023], dtype=np.int32)
    want = O.ksat_anneal(lits, n, beta, 0, T, wl["seed"], replica_ids=ids)
    _same(got, want, ids)
    for r in range(0, R, 97):
        assert got["energies"][r] == O.ksat_energy(lits, n, got["states"][r])
        assert got["best_energies"][r] == O.ksat_energy(lits, n, got["best_states"][r])
    assert np.all(got["best_energies"] <= got["energies"])


@pytest.mark.parametrize("extra", [0, 1])
def test_largest_shared_memory_instance(ctx, extra):
    """The largest formula whose word vector fits one CTA's shared memory (next to the acceptance
    table) runs on the cluster kernel; one variable more goes to the grid-barrier kernel. Both
    give the oracle's trajectories on sampled replicas, and every replica's energy matches a
    recount of its state."""
    n = ctx.batch_max_vars() + extra
    assert 40_000 < n < 60_000
    T, R = 8, 64
    lits = W.random_ksat(n, 9.6, 4, 900 + extra)
    beta = W.beta_inhomogeneous_linear(n, T, 0.5, 4.0, 0.3, 0.5, 901 + extra)
    inst = ctx.load_ksat(lits, n)
    ctx.set_schedule(inst, beta)
    rs = ctx.replicas_create(inst, R, seed=11)
    ctx.replicas_run(rs, 0, T)
    got = ctx.replicas_read(rs)
    ctx.replicas_destroy(rs)
    ctx.unload(inst)
    ids = np.array([0, 31, 32, 63], dtype=np.int32)
    want = O.ksat_anneal(lits, n, beta, 0, T, 11, replica_ids=ids)
    _same(got, want, ids)
    assert np.array_equal(O.ksat_energies(lits, n, got["states"]), got["energies"])
    assert np.array_equal(O.ksat_energies(lits, n, got["best_states"]), got["best_energies"])


@pytest.mark.parametrize("warps", [0, 1, 2, 4])
@pytest.mark.parametrize("n,alpha,k,R,T", [
    (500, 9.6, 4, 1024, 20),    # one 32-word group
    (300, 3.0, 6, 2048, 6),     # two word groups, two int4 per occurrence
    (2000, 4.2, 3, 1024, 8),    # low degree: 5-bit counters
])
def test_sweep_shapes_agree(ctx, monkeypatch, warps, n, alpha, k, R, T):
    """Every grid-kernel shape (general kernel, teams of 1, 2 or 4 warps per variable) gives
    the oracle's trajectories."""
    monkeypatch.setenv("NMC_RUN_PATH", "grid")
    monkeypatch.setenv("NMC_SWEEP_WARPS", str(warps))
    lits = W.random_ksat(n, alpha, k, 700 + n)
    beta = W.beta_inhomogeneous_linear(n, T, 0.3, 4.0, 0.3, 0.5, 800 + n)
    got = _run(ctx, lits, n, beta, R, 0, T, seed=n)
    want = O.ksat_anneal(lits, n, beta, 0, T, n, replicas=R)
    _same(got, want)


def test_factored_schedule_equals_expanded(ctx):
    """beta[u][t] = float32(base[t] * factor[u]) on the device equals the expanded array."""
    n, T, R = 500, 30, 64
    lits = W.random_ksat(n, 9.6, 4, 31)
    base = W.geometric_profile(0.3, 6.0, T).astype(np.float32)
    factor = np.where(W.seeded_subset(n, 0.2, 32), 0.4, 1.0).astype(np.float32)
    beta = (factor[:, None] * base[None, :]).astype(np.float32)  # IEEE float32 products
    inst = ctx.load_ksat(lits, n)
    ctx.set_schedule_factored(inst, base, factor)
    got = ctx.anneal(inst, R, 0, T, seed=33)
    ctx.unload(inst)
    _same(got, O.ksat_anneal(lits, n, beta, 0, T, 33, replicas=R))


def test_checkpoint_restore_continues_exactly(ctx):
    wl = W.workload_ksat_small(50)
    lits, n, beta = wl["lits"], wl["n_vars"], wl["beta"]
    inst = ctx.load_ksat(lits, n)
    ctx.set_schedule(inst, beta)
    a = ctx.replicas_create(inst, 70, seed=5)
    ctx.replicas_run(a, 0, 20)
    ckpt = ctx.replicas_read(a)
    ctx.replicas_destroy(a)
    b = ctx.replicas_create(inst, 70, seed=5)
    ctx.replicas_restore(b, ckpt)
    mid = ctx.replicas_read(b)
    for key in KEYS:
        assert np.array_equal(mid[key], ckpt[key]), key
    ctx.replicas_run(b, 20, 50)
    got = ctx.replicas_read(b)
    ctx.replicas_destroy(b)
    ctx.unload(inst)
    _same(got, O.ksat_anneal(lits, n, beta, 0, 50, 5, replicas=70))
