"""Whitening on the GPU (32 replicas per word, parallel rounds) against the CPU oracle (one
variable at a time): the fixed point is unique, so frozen flags and counts match bit for bit."""
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


@pytest.mark.parametrize("n,alpha,k,R,T,b", [(600, 4.2, 3, 70, 80, 4.0),
                                               (2000, 9.6, 4, 96, 60, 3.0),
                                               (300, 2.0, 6, 33, 40, 3.0)])
def test_whitening_parity(ctx, n, alpha, k, R, T, b):
    lits = W.random_ksat(n, alpha, k, 500 + n)
    inst = ctx.load_ksat(lits, n)
    ctx.set_schedule(inst, W.beta_constant(n, T, b))
    rs = ctx.replicas_create(inst, R, 3)
    ctx.replicas_run(rs, 0, T)
    st = ctx.replicas_read(rs)
    for use_best in (False, True):
        for gen in (True, False):
            cnt, fr, rounds = ctx.whitening(rs, use_best=use_best, generalized=gen, masks=True)
            X = st["best_states" if use_best else "states"]
            for r in range(R):
                wf, wc = O.ksat_whitening(lits, n, X[r], gen)
                assert cnt[r] == wc, (use_best, gen, r)
                assert np.array_equal(fr[r], wf), (use_best, gen, r)
            assert rounds >= 1
    ctx.replicas_destroy(rs)
    ctx.unload(inst)


def test_whitening_of_planted_solutions(ctx):
    """Assignments that satisfy every clause (a planted formula): the standard and generalized
    forms agree, and some variables are frozen."""
    n, m = 500, 3000  # clause density 6: the planted solution has a frozen core (414)
    rng = np.random.default_rng(8)
    x0 = rng.integers(0, 2, n).astype(np.uint8)
    rows = []
    while len(rows) < m:
        v = rng.choice(n, size=3, replace=False)
        s = rng.choice([-1, 1], size=3)
        if any((x0[v[j]] == 1) == (s[j] > 0) for j in range(3)):
            rows.append((v + 1) * s)
    lits = np.array(rows, np.int32)
    inst = ctx.load_ksat(lits, n)
    rs = ctx.replicas_create(inst, 40, 1, init=np.repeat(x0[None], 40, axis=0))
    g = ctx.whitening(rs, generalized=True)
    s = ctx.whitening(rs, generalized=False)
    want, wc = O.ksat_whitening(lits, n, x0)
    assert np.all(g == wc) and np.all(s == wc) and wc > 0
    ctx.replicas_destroy(rs)
    ctx.unload(inst)
