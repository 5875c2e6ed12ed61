"""Learning stage on the GPU (CNF loopy BP, backbone growth, the two-chain schedule) against
the CPU oracle, through the C ABI.

LBP runs in double precision on both sides. The GPU forms each cavity field by subtracting the
edge's own message from the variable's total field and uses CUDA's exp / log1p (the clause
pass forms (1 - tanh h)/2 as 1/(1 + e^{2h})), the oracle
sums the other clauses directly with the host libm: each step differs by a few units in the
last place (about 1e-16 relative), and in the contracting regime the fixed-point map shrinks
such differences instead of growing them, so 1e-9 absolute on marginals, correlations and
overlaps is a wide margin; iteration counts and converged-lambda counts must match exactly.
Backbone labels and the schedule are integer results and must match bit for bit (the backbone
kernels take the same correlation array as the oracle).
"""
import numpy as np
import pytest

import nmc_inputs as W
import oracle as O

pytestmark = pytest.mark.gpu
TOL = 1e-9


@pytest.fixture(scope="module")
def ctx():
    import paper_2111_13628_gb300 as nmc
    c = nmc.Context(0)
    yield c
    c.close()


def _tree_cnf(seed):
    rng = np.random.default_rng(seed)
    groups = [[0, 1, 2], [2, 3, 4], [2, 5], [4, 6, 7], [7, 8, 9, 10], [1, 11], [11, 12]]
    lits = np.zeros((len(groups), 4), np.int32)
    for a, g in enumerate(groups):
        lits[a, :len(g)] = (np.array(g) + 1) * rng.choice([-1, 1], size=len(g))
    return lits, 13


def _compare(got, lits, n, X, beta, lams, tol, max_iter, eps=None):
    for s in range(X.shape[0]):
        want = O.cnf_lbp(lits, n, X[s], beta, lams, tol, max_iter, eps=eps)
        assert got["n_done"][s] == want["n_done"], s
        assert np.array_equal(got["iters"][s], want["iters"]), (s, got["iters"][s], want["iters"])
        assert np.allclose(got["marg"][s], want["marg"], atol=TOL, rtol=0), s
        assert np.allclose(got["corr"][s], want["corr"], atol=TOL, rtol=0), s
        assert abs(got["p"][s] - want["p"]) < TOL and abs(got["q1"][s] - want["q1"]) < TOL


@pytest.mark.parametrize("beta,lams", [(0.7, [0.3]), (2.0, [0.4, 0.1, 0.02]), (1.2, [0.0])])
def test_lbp_tree_parity(ctx, beta, lams):
    lits, n = _tree_cnf(3)
    X = np.random.default_rng(1).integers(0, 2, size=(3, n)).astype(np.uint8)
    inst = ctx.load_ksat(lits, n)
    got = ctx.cnf_lbp(inst, X, beta, lams, 1e-13, 300)
    ctx.unload(inst)
    _compare(got, lits, n, X, beta, lams, 1e-13, 300)


@pytest.mark.parametrize("k,alpha,S", [(4, 9.6, 5), (3, 4.2, 33), (6, 2.5, 2)])
def test_lbp_random_formula_parity(ctx, k, alpha, S):
    n = 500
    lits = W.random_ksat(n, alpha, k, 90 + k)
    X = np.random.default_rng(k).integers(0, 2, size=(S, n)).astype(np.uint8)
    lams = [0.3, 0.15, 0.08, 0.04, 0.02]
    inst = ctx.load_ksat(lits, n)
    got = ctx.cnf_lbp(inst, X, 1.0, lams, 1e-9, 150)
    ctx.unload(inst)
    _compare(got, lits, n, X, 1.0, lams, 1e-9, 150)


def test_lbp_fallback_and_given_eps(ctx):
    n = 300
    lits = W.random_ksat(n, 9.6, 4, 6)
    X = np.random.default_rng(4).integers(0, 2, size=(4, n)).astype(np.uint8)
    lams = [0.5, 0.2, 0.1, 0.05, 0.02, 0.01, 0.005]
    eps = np.linspace(0.5, 2.0, n)
    inst = ctx.load_ksat(lits, n)
    got = ctx.cnf_lbp(inst, X, 1.0, lams, 1e-9, 15)
    gote = ctx.cnf_lbp(inst, X, 1.3, lams, 1e-9, 40, eps=eps)
    ctx.unload(inst)
    assert np.all(got["n_done"] < len(lams))
    _compare(got, lits, n, X, 1.0, lams, 1e-9, 15)
    _compare(gote, lits, n, X, 1.3, lams, 1e-9, 40, eps=eps)


def test_backbone_parity(ctx):
    n = 2000
    lits = W.random_ksat(n, 4.2, 3, 77)
    rng = np.random.default_rng(5)
    m = lits.shape[0]
    corr = np.tanh(rng.exponential(0.6, (3, m))) * rng.choice([-1, 1], (3, m))
    corr[0, :5] = 1.0  # infinite couplings
    inst = ctx.load_ksat(lits, n)
    for seed_thr, cutoff in [(1.5, 1.2), (2.0, 0.9), (0.8, 1.0), (9.0, 9.0)]:
        lab, nc = ctx.cnf_backbone(inst, corr, 1.0, seed_thr, cutoff)
        for s in range(3):
            want, wn = O.cnf_backbone(lits, n, corr[s], 1.0, seed_thr, cutoff)
            assert np.array_equal(lab[s], want), (seed_thr, cutoff, s)
            assert nc[s] == wn
    ctx.unload(inst)


def test_learning_pipeline_parity(ctx):
    """Seeds from a GPU anneal, LBP with continuation, backbones, the two-chain schedule, and
    the inhomogeneous sampling it drives: each stage against the oracle on the same input."""
    n, T = 800, 60
    lits = W.random_ksat(n, 9.6, 4, 31)
    inst = ctx.load_ksat(lits, n)
    ctx.set_schedule(inst, W.beta_constant(n, T, 2.0))
    seeds = ctx.anneal(inst, 4, 0, T, 3)["best_states"]
    lams = [0.4, 0.2, 0.1, 0.05]
    got = ctx.cnf_lbp(inst, seeds, 1.0, lams, 1e-10, 200)
    _compare(got, lits, n, seeds, 1.0, lams, 1e-10, 200)
    lab, nc = ctx.cnf_backbone(inst, got["corr"], 1.0, 2.5, 2.0)
    want, wn = O.cnf_backbone(lits, n, got["corr"][0], 1.0, 2.5, 2.0)
    assert np.array_equal(lab[0], want) and nc[0] == wn
    ctx.set_schedule_backbone(inst, lab[0], 3, 4, 3, 2, 3.0, 4.0)
    out = ctx.anneal(inst, 64, 0, 27, 9)
    ctx.unload(inst)
    beta = O.backbone_schedule(lab[0], 3.0, 4.0, 3, 4, 3, 2)
    ref = O.ksat_anneal(lits, n, beta, 0, 27, 9, replicas=64)
    for key in ("states", "energies", "best_energies", "best_states"):
        assert np.array_equal(out[key], ref[key]), key


def test_learning_stage_argument_checks(ctx):
    import paper_2111_13628_gb300 as nmc
    n = 40
    lits = W.random_ksat(n, 4.2, 3, 2)
    inst = ctx.load_ksat(lits, n)
    x = np.zeros(n, np.uint8)
    bad_calls = [
        lambda: ctx.cnf_lbp(inst, np.full(n, 2, np.uint8), 1.0, [0.1], 1e-9, 10),
        lambda: ctx.cnf_lbp(inst, x, np.nan, [0.1], 1e-9, 10),
        lambda: ctx.cnf_lbp(inst, x, 1.0, [np.inf], 1e-9, 10),
        lambda: ctx.cnf_lbp(inst, x, 1.0, [0.1], 1e-9, 0),
        lambda: ctx.cnf_backbone(inst, np.full(lits.shape[0], 1.5), 1.0, 1.0, 1.0),
        lambda: ctx.cnf_backbone(inst, np.zeros(lits.shape[0]), 0.0, 1.0, 1.0),
        lambda: ctx.set_schedule_backbone(inst, np.zeros(n, np.int32), 0, 1, 1, 1, 1.0, 2.0),
        lambda: ctx.set_schedule_backbone(inst, np.zeros(n, np.int32), 1, 1, 1, 1, 1.0, 0.0),
        lambda: ctx.set_schedule_backbone(inst, np.zeros(n, np.int32), 1, 1, 1, 1, 60000.0, 1e-4),
    ]
    for call in bad_calls:
        with pytest.raises(nmc.NmcError) as e:
            call()
        assert e.value.code == nmc.NMC_EINVAL
    ctx.unload(inst)
