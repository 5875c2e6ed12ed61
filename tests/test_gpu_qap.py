"""QAP swap chain on the GPU, through the C ABI, against the CPU oracle: bit for bit."""
import numpy as np
import pytest

import nmc_inputs as W
import oracle as O

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def ctx():
    import paper_2111_13628_gb300 as nmc
    c = nmc.Context(0)
    yield c
    c.close()


def _same(got, want, ids=None):
    for a, b in (("states", "perms"), ("energies", "energies"),
                 ("best_energies", "best_energies"), ("best_states", "best_perms")):
        g = got[a] if ids is None else got[a][ids]
        assert np.array_equal(g, want[b]), a


# n picks the launch shape: 16 lanes per replica and n / 16 facilities per lane up to n = 128,
# 32 lanes and n / 32 per lane beyond; the cases cover all twelve shapes and their edges
@pytest.mark.parametrize("n,R,T", [(1, 3, 4), (2, 5, 6), (3, 33, 10), (31, 40, 8), (32, 32, 8),
                                   (33, 17, 8), (64, 9, 6), (72, 19, 4), (90, 33, 3),
                                   (100, 35, 4), (128, 64, 3), (129, 8, 3), (170, 10, 2),
                                   (192, 7, 2), (224, 5, 2), (256, 6, 2)])
def test_parity_shapes(ctx, n, R, T):
    F, D = W.random_qap(n, 300 + n)
    beta = W.beta_scaled_linear(n, T, 0.01, 1.0, 0.5, 1.5, 400 + n)
    inst = ctx.load_qap(F, D)
    ctx.set_schedule(inst, beta)
    got = ctx.anneal(inst, R, 0, T, seed=7 + n)
    ctx.unload(inst)
    want = O.qap_anneal(F, D, beta, 0, T, 7 + n, replicas=R)
    _same(got, want)


def test_segments_and_given_init(ctx):
    n, R, T = 57, 45, 30
    F, D = W.random_qap(n, 1)
    beta = W.beta_scaled_linear(n, T, 0.01, 1.0, 0.5, 1.5, 2)
    inst = ctx.load_qap(F, D)
    ctx.set_schedule(inst, beta)
    rs = ctx.replicas_create(inst, R, seed=3)
    for t0, t1 in [(0, 7), (7, 7), (7, 30)]:
        ctx.replicas_run(rs, t0, t1)
    got = ctx.replicas_read(rs)
    ctx.replicas_destroy(rs)
    _same(got, O.qap_anneal(F, D, beta, 0, T, 3, replicas=R))
    init = np.stack([np.random.default_rng(i).permutation(n) for i in range(R)]).astype(np.int16)
    got = ctx.anneal(inst, R, 5, T, seed=3, init=init)
    _same(got, O.qap_anneal(F, D, beta, 5, T, 3, replicas=R, init=init))
    ctx.unload(inst)


def test_rejects_bad_input(ctx):
    import paper_2111_13628_gb300 as nmc
    F, D = W.random_qap(6, 1)
    A = F.copy()
    A[0, 1] += 1                      # not symmetric
    B = F.copy()
    B[2, 2] = 1                       # non-zero diagonal
    C2 = F.copy()
    C2[0, 1] = C2[1, 0] = 300         # entry above 255
    for bad in (A, B, C2):
        with pytest.raises(nmc.NmcError):
            ctx.load_qap(bad, D)
    inst = ctx.load_qap(F, D)
    with pytest.raises(nmc.NmcError):
        ctx.replicas_create(inst, 2, 1, init=np.zeros((2, 6), np.int16))  # not permutations
    ctx.unload(inst)


def test_full_size_sampled_replicas(ctx):
    """A 256-facility instance with 4096 replicas (the largest of the QAP batch): sampled
    replicas bit for bit, all replicas for cost consistency."""
    n, R, T = 256, 4096, 3
    F, D = W.random_qap(n, 1004 * 1000)
    beta = W.beta_scaled_linear(n, T, 0.01, 1.0, 0.5, 1.5, 1004 * 2000)
    inst = ctx.load_qap(F, D)
    ctx.set_schedule(inst, beta)
    got = ctx.anneal(inst, R, 0, T, seed=20_000)
    ctx.unload(inst)
    ids = np.array([0, 31, 32, 2049, 4095], dtype=np.int32)
    _same(got, O.qap_anneal(F, D, beta, 0, T, 20_000, replica_ids=ids), ids)
    for r in range(0, R, 411):
        assert got["energies"][r] == O.qap_cost(F, D, got["states"][r])


def test_batched_qap_matches_single_sets_and_oracle(ctx):
    specs = [(20, 40, 9), (33, 70, 6), (64, 33, 5), (100, 64, 4), (200, 40, 3), (256, 35, 2)]
    sets, data = [], []
    for i, (n, R, T) in enumerate(specs):
        F, D = W.random_qap(n, 900 + i)
        beta = W.beta_scaled_linear(n, T, 0.01, 1.0, 0.5, 1.5, 910 + i)
        inst = ctx.load_qap(F, D)
        ctx.set_schedule(inst, beta)
        a = ctx.replicas_create(inst, R, seed=920 + i)
        b = ctx.replicas_create(inst, R, seed=920 + i)
        sets.append((inst, a, b))
        data.append((F, D, beta, R, T, 920 + i))
    ctx.qap_batch_run([a for _, a, _ in sets], 0, [d[4] for d in data])
    for (inst, a, b), (F, D, beta, R, T, seed) in zip(sets, data):
        ctx.replicas_run(b, 0, T)
        ga, gb = ctx.replicas_read(a), ctx.replicas_read(b)
        for key in ("states", "energies", "best_energies", "best_states"):
            assert np.array_equal(ga[key], gb[key]), key
        ids = np.array([0, R - 1], dtype=np.int32)
        _same(ga, O.qap_anneal(F, D, beta, 0, T, seed, replica_ids=ids), ids)
        ctx.replicas_destroy(a)
        ctx.replicas_destroy(b)
        ctx.unload(inst)


def test_checkpoint_restore_continues_exactly(ctx):
    n, R, T = 45, 40, 20
    F, D = W.random_qap(n, 77)
    beta = W.beta_scaled_linear(n, T, 0.01, 1.0, 0.5, 1.5, 78)
    inst = ctx.load_qap(F, D)
    ctx.set_schedule(inst, beta)
    a = ctx.replicas_create(inst, R, seed=79)
    ctx.replicas_run(a, 0, 8)
    ckpt = ctx.replicas_read(a)
    ctx.replicas_destroy(a)
    b = ctx.replicas_create(inst, R, seed=79)
    ctx.replicas_restore(b, ckpt)
    ctx.replicas_run(b, 8, T)
    got = ctx.replicas_read(b)
    ctx.replicas_destroy(b)
    ctx.unload(inst)
    _same(got, O.qap_anneal(F, D, beta, 0, T, 79, replicas=R))
