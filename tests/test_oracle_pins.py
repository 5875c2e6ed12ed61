"""Pins the CPU oracle to facts other than itself (CPU only, no GPU).

Each check is chosen so that a plausible mistake in the oracle fails it: brute-force
enumeration of every assignment / permutation, recomputation of every energy change, the exact
Boltzmann law as the stationary distribution of the homogeneous chain (chi-square), closed
forms at beta = 0 and beta -> infinity, the Philox4x32-10 definition as implemented by an
independent library (triton's interpreter), and the threshold table against 60-digit
arithmetic (mpmath).
"""
import itertools
import json
import math
import os
import subprocess
import sys
from fractions import Fraction

import numpy as np
import pytest

import nmc_inputs as W
import oracle as O

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


# ---------------------------------------------------------------- independent evaluators
def energies_numpy(lits, X):
    """#violated clauses for every row of X (S x N uint8), written independently of the
    oracle: a clause is satisfied when any of its literals matches."""
    lits = np.asarray(lits)
    X = np.asarray(X, dtype=np.uint8)
    used = lits != 0
    var = np.abs(lits) - 1
    want = (lits > 0).astype(np.uint8)
    vals = X[:, np.where(used, var, 0)]  # S x M x k
    sat = ((vals == want[None]) & used[None]).any(axis=2)
    return (~sat).sum(axis=1).astype(np.int64)


def all_states(n):
    return ((np.arange(2 ** n)[:, None] >> np.arange(n)[None, :]) & 1).astype(np.uint8)


def small_cnf(n, m, k, seed, pad_some=False):
    rng = np.random.default_rng(seed)
    rows = []
    for _ in range(m):
        kk = k if not pad_some else int(rng.integers(1, k + 1))
        v = rng.choice(n, size=kk, replace=False) + 1
        s = rng.choice([-1, 1], size=kk)
        row = np.zeros(k, dtype=np.int32)
        row[:kk] = v * s
        rows.append(row)
    return np.array(rows, dtype=np.int32)


# ---------------------------------------------------------------- paper-printed sizes
def test_paper_clause_count_convention():
    path = os.path.join(ROOT, "tests", "golden", "paper_sizes.txt")
    rows = [l.split() for l in open(path) if l.strip() and not l.startswith("#")]
    for k, n, alpha, m, viol in rows:
        assert W.n_clauses(int(n), float(alpha)) == int(m)
        assert W.random_ksat(int(n), float(alpha), int(k), 7).shape == (int(m), int(k))
        # ratio 1e-4 of the clauses, rounded to the nearest violation count
        assert round(1e-4 * int(m)) == int(viol)


# ---------------------------------------------------------------- Philox4x32-10
_TRITON_SCRIPT = r"""
import os, sys, json
os.environ["TRITON_INTERPRET"] = "1"
import numpy as np, torch, triton, triton.language as tl
@triton.jit
def k(cp, outp, seed, BLOCK: tl.constexpr):
    o = tl.arange(0, BLOCK)
    c0 = tl.load(cp + o * 4 + 0); c1 = tl.load(cp + o * 4 + 1)
    c2 = tl.load(cp + o * 4 + 2); c3 = tl.load(cp + o * 4 + 3)
    a, b, c, d = tl.philox(seed, c0, c1, c2, c3)
    tl.store(outp + o * 4 + 0, a); tl.store(outp + o * 4 + 1, b)
    tl.store(outp + o * 4 + 2, c); tl.store(outp + o * 4 + 3, d)
req = json.loads(sys.stdin.read())
res = []
for seed, ctrs in req:
    c = torch.tensor(np.array(ctrs, dtype=np.uint32).view(np.int32))
    out = torch.zeros_like(c)
    k[(1,)](c, out, seed, BLOCK=c.shape[0])
    res.append(out.numpy().view(np.uint32).tolist())
print(json.dumps(res))
"""


def test_philox_matches_independent_implementation():
    pytest.importorskip("triton")
    rng = np.random.default_rng(5)
    req = []
    seeds = [0, 1, 0xFFFFFFFF, 0x123456789ABCDEF, 2**64 - 1, int(rng.integers(0, 2**63))]
    for s in seeds:
        ctrs = rng.integers(0, 2**32, size=(8, 4), dtype=np.uint64)
        ctrs[0] = 0
        ctrs[1] = 0xFFFFFFFF
        req.append([s, ctrs.tolist()])
    env = dict(os.environ, TRITON_INTERPRET="1")
    out = subprocess.run([sys.executable, "-c", _TRITON_SCRIPT], input=json.dumps(req),
                         capture_output=True, text=True, env=env, timeout=600)
    if out.returncode != 0:
        pytest.skip("triton interpreter unavailable: " + out.stderr[-300:])
    ref = json.loads(out.stdout.strip().splitlines()[-1])
    for (s, ctrs), r in zip(req, ref):
        key = [s & 0xFFFFFFFF, (s >> 32) & 0xFFFFFFFF]
        for c, rr in zip(ctrs, np.array(r, dtype=np.uint64).reshape(-1, 4)):
            got = O.philox4x32_10(c, key)
            assert got.tolist() == rr.tolist(), (s, c)


def test_philox_is_a_bijection_of_the_counter_and_looks_uniform():
    # distinct counters give distinct blocks; bits are balanced
    key = [7, 9]
    outs = np.array([O.philox4x32_10([i, 0, 0, 0], key) for i in range(4096)])
    assert len({tuple(o) for o in outs}) == 4096
    bits = np.unpackbits(outs.view(np.uint8))
    assert abs(bits.mean() - 0.5) < 0.01


# ---------------------------------------------------------------- thresholds, quantisation
def test_threshold_table_against_high_precision():
    mpmath = pytest.importorskip("mpmath")
    mpmath.mp.dps = 60
    tab, L = O.threshold_table()
    assert tab[0] == 2**32 - 1
    # first zero entry: 2^32 exp(-j/256) < 1  <=>  j > 256 * 32 ln 2
    assert L == math.floor(256 * 32 * math.log(2)) + 1
    for j in range(1, L + 3):
        exact = int(mpmath.floor(mpmath.ldexp(mpmath.exp(-mpmath.mpf(j) / 256), 32)))
        exact = min(exact, 2**32 - 1)
        got = int(tab[j]) if j < L else 0
        assert got == exact, j
    assert np.all(np.diff(tab.astype(np.int64)) <= 0)


def test_beta_quantisation_rounds_half_to_even():
    cases = [0.0, 1.0, 0.5, 4.0, 6.0, 0.3, 0.01, 65535.0, 1e-9, 3.5 / 65536, 2.5 / 65536,
             12345.678]
    for b in cases:
        b32 = float(np.float32(b))
        exact = Fraction(b32) * 65536
        assert O.quantize_beta(b32) == round(exact)  # Fraction rounds half to even


def test_uphill_threshold_is_boltzmann_factor_on_the_grid():
    # beta = m/256 and integer dE: beta*dE is on the table's grid, so the threshold is
    # floor(2^32 exp(-beta dE)) up to the 2^32-1 cap
    for m in [1, 7, 64, 255, 256, 300, 1024]:
        bq = m * 256
        for dE in [1, 2, 3, 5, 8, 20]:
            x = m * dE / 256.0
            want = math.floor(math.ldexp(math.exp(-x), 32)) if x < 22.18 else 0
            got = O.uphill_threshold(bq, dE)
            assert abs(got - min(want, 2**32 - 1)) <= 1, (m, dE)
    # off-grid beta: the index truncates beta*dE down to a multiple of 1/256
    rng = np.random.default_rng(3)
    tab, L = O.threshold_table()
    for _ in range(200):
        bq = int(rng.integers(0, 2**20))
        dE = int(rng.integers(1, 50))
        j = (bq * dE) // 256
        assert O.uphill_threshold(bq, dE) == (int(tab[j]) if j < L else 0)


# ---------------------------------------------------------------- k-SAT energy and moves
@pytest.mark.parametrize("n,m,k,pad", [(10, 42, 3, False), (12, 100, 4, False),
                                       (9, 30, 4, True)])
def test_energy_matches_enumeration(n, m, k, pad):
    lits = small_cnf(n, m, k, seed=n * 100 + m, pad_some=pad)
    X = all_states(n)
    want = energies_numpy(lits, X)
    got = np.array([O.ksat_energy(lits, n, x) for x in X])
    assert np.array_equal(got, want)
    assert want.min() >= 0


def _energies_numpy_chunked(lits, n, chunk=1 << 15):
    out = []
    for s0 in range(0, 1 << n, chunk):
        idx = np.arange(s0, min(s0 + chunk, 1 << n), dtype=np.int64)
        X = ((idx[:, None] >> np.arange(n)[None, :]) & 1).astype(np.uint8)
        out.append(energies_numpy(lits, X))
    return np.concatenate(out)


@pytest.mark.parametrize("case", ["planted_3sat", "unsat_4sat", "padded_mixed"])
def test_energy_and_ground_states_by_enumeration_n20(case):
    """All 2^20 assignments of a 20-variable formula: the oracle's energy equals the independent
    evaluator on every one, and the ground-state energy and the set of ground states agree. A
    formula with a planted solution (clauses that solution violates are dropped) has ground
    energy 0 with the planted state among its ground states, each of which satisfies every clause
    when checked literal by literal; an over-constrained 4-SAT formula has no solution."""
    n = 20
    rng = np.random.default_rng({"planted_3sat": 1, "unsat_4sat": 2, "padded_mixed": 3}[case])
    if case == "planted_3sat":
        lits = small_cnf(n, 140, 3, seed=201)
        plant = rng.integers(0, 2, size=n, dtype=np.uint8)
        keep = [energies_numpy(row[None], plant[None])[0] == 0 for row in lits]
        lits = lits[np.array(keep)]
    elif case == "unsat_4sat":
        lits = small_cnf(n, 400, 4, seed=202)
    else:
        lits = small_cnf(n, 180, 5, seed=203, pad_some=True)
    X = all_states(n)
    got = O.ksat_energies(lits, n, X)
    want = _energies_numpy_chunked(lits, n)
    assert np.array_equal(got, want)
    e0 = int(want.min())
    ground = set(np.nonzero(got == e0)[0].tolist())
    assert ground == set(np.nonzero(want == e0)[0].tolist())
    if case == "planted_3sat":
        assert e0 == 0
        assert int((plant.astype(np.int64) << np.arange(n)).sum()) in ground
        for s in list(ground)[:64]:
            x = X[s]
            for row in lits:
                assert any(x[abs(l) - 1] == (l > 0) for l in row if l != 0)
    if case == "unsat_4sat":
        assert e0 > 0


def test_energy_of_generated_instance_matches_independent_count():
    lits = W.random_ksat(300, 9.6, 4, 11)
    rng = np.random.default_rng(1)
    X = rng.integers(0, 2, size=(20, 300), dtype=np.uint8)
    want = energies_numpy(lits, X)
    got = np.array([O.ksat_energy(lits, 300, x) for x in X])
    assert np.array_equal(got, want)


@pytest.mark.parametrize("n,m,k,pad", [(15, 60, 3, False), (20, 190, 4, False),
                                       (14, 70, 5, True)])
def test_delta_matches_recomputation(n, m, k, pad):
    lits = small_cnf(n, m, k, seed=7 * n + m, pad_some=pad)
    rng = np.random.default_rng(n)
    for _ in range(6):
        x = rng.integers(0, 2, size=n, dtype=np.uint8)
        e0 = energies_numpy(lits, x[None])[0]
        for v in range(n):
            y = x.copy()
            y[v] ^= 1
            e1 = energies_numpy(lits, y[None])[0]
            assert O.ksat_delta(lits, n, x, v) == e1 - e0


def _adjacency(lits, n):
    adj = [set() for _ in range(n)]
    for row in lits:
        vs = [abs(int(l)) - 1 for l in row if l != 0]
        for a in vs:
            for b in vs:
                if a != b:
                    adj[a].add(b)
    return adj


@pytest.mark.parametrize("n,alpha,k", [(200, 9.6, 4), (500, 4.2, 3), (50, 2.0, 5)])
def test_colouring_is_proper_and_minimal(n, alpha, k):
    lits = W.random_ksat(n, alpha, k, 99 + n)
    col, nc = O.ksat_colour(lits, n)
    adj = _adjacency(lits, n)
    assert col.min() == 0 and col.max() == nc - 1
    for v in range(n):
        assert all(col[u] != col[v] for u in adj[v])  # classes are independent sets
        # a variable takes the smallest colour its earlier-coloured neighbours leave free, so
        # every smaller colour is held by one of its neighbours
        assert set(range(col[v])) <= {int(col[u]) for u in adj[v]}


def _two_clauses(edges):
    return np.array([[a + 1, b + 1] for a, b in edges], dtype=np.int32)


def test_dsatur_textbook_cases():
    # one clause of k variables is a k-clique: k colours
    for k in (3, 5, 8):
        col, nc = O.ksat_colour(np.arange(1, k + 1, dtype=np.int32)[None, :], k)
        assert nc == k and sorted(col.tolist()) == list(range(k))
    # cycles: 2 colours when even, 3 when odd
    for length in (6, 7, 10, 11):
        col, nc = O.ksat_colour(_two_clauses([(i, (i + 1) % length) for i in range(length)]), length)
        assert nc == (2 if length % 2 == 0 else 3)
    # DSatur colours bipartite graphs with 2 colours (Brelaz 1979). The crown graph (a_i ~ b_j
    # for i != j) with ids interleaved a_0, b_0, a_1, b_1, ... is the classic case where greedy
    # colouring in id order needs h colours.
    for h in (4, 7):
        edges = [(2 * i, 2 * j + 1) for i in range(h) for j in range(h) if i != j]
        col, nc = O.ksat_colour(_two_clauses(edges), 2 * h)
        assert nc == 2
        assert all(col[a] != col[b] for a, b in edges)
    # DSatur is also exact on wheels (a hub joined to every vertex of a cycle): 3 colours
    # around an even rim, 4 around an odd one; the hub, of highest degree, comes first
    for rim in (6, 7, 10, 11):
        edges = [(0, i) for i in range(1, rim + 1)] + \
                [(i, i % rim + 1) for i in range(1, rim + 1)]
        col, nc = O.ksat_colour(_two_clauses(edges), rim + 1)
        assert nc == (3 if rim % 2 == 0 else 4) and col[0] == 0
        assert all(col[a] != col[b] for a, b in edges)


def test_dsatur_worked_path():
    # path 0-1-2-3, worked by hand from the selection rule: 1 and 2 have two occurrences, 1 is
    # smaller -> colour 0; 0 and 2 now see one colour, 2 has more occurrences -> colour 1; 0 and
    # 3 tie on both, 0 is smaller -> colour 1; then 3 -> colour 0. (Id order would give 0,1,0,1.)
    col, nc = O.ksat_colour(_two_clauses([(0, 1), (1, 2), (2, 3)]), 4)
    assert nc == 2 and col.tolist() == [1, 0, 1, 0]


# ---------------------------------------------------------------- closed forms of the chain
def test_beta_zero_flips_every_variable_every_sweep():
    n = 60
    lits = W.random_ksat(n, 4.2, 3, 5)
    beta = np.zeros((n, 9), dtype=np.float32)
    r0 = O.ksat_anneal(lits, n, beta, 0, 0, seed=3, replicas=40)
    for t1 in [1, 2, 5, 9]:
        r = O.ksat_anneal(lits, n, beta, 0, t1, seed=3, replicas=40)
        assert np.array_equal(r["states"], r0["states"] ^ np.uint8(t1 & 1))
        assert np.array_equal(r["energies"], energies_numpy(lits, r["states"]))


def test_infinite_beta_never_goes_uphill():
    n = 120
    lits = W.random_ksat(n, 9.6, 4, 8)
    T = 12
    beta = np.full((n, T), 65535.0, dtype=np.float32)
    st = O.ksat_anneal(lits, n, beta, 0, 0, seed=4, replicas=16)
    prev = st["energies"].copy()
    best = st["best_energies"].copy()
    bstates = st["best_states"].copy()
    for t in range(T):
        st = O.ksat_anneal(lits, n, beta, t, t + 1, seed=4, replicas=16, init=st["states"],
                           init_best=bstates, init_best_energy=best)
        assert np.all(st["energies"] <= prev)
        prev = st["energies"].copy()
        best, bstates = st["best_energies"], st["best_states"]
    assert np.array_equal(best, prev)  # a descent's best is its last state


def test_invariants_segments_and_replica_subsets():
    wl = W.workload_ksat_small(60)
    lits, n, beta = wl["lits"], wl["n_vars"], wl["beta"]
    full = O.ksat_anneal(lits, n, beta, 0, 60, seed=1, replicas=24)
    assert np.all(full["energies"] >= 0)
    assert np.array_equal(full["energies"], energies_numpy(lits, full["states"]))
    assert np.array_equal(full["best_energies"], energies_numpy(lits, full["best_states"]))
    assert np.all(full["best_energies"] <= full["energies"])
    init = O.ksat_anneal(lits, n, beta, 0, 0, seed=1, replicas=24)
    assert np.all(full["best_energies"] <= init["energies"])
    # segment invariance: [0,25) then [25,60) from the resident state and best
    a = O.ksat_anneal(lits, n, beta, 0, 25, seed=1, replicas=24)
    b = O.ksat_anneal(lits, n, beta, 25, 60, seed=1, replicas=24, init=a["states"],
                      init_best=a["best_states"], init_best_energy=a["best_energies"])
    for key in ["states", "energies", "best_energies", "best_states"]:
        assert np.array_equal(b[key], full[key]), key
    # best is the minimum over sweep ends, earliest kept
    st, mins = init, init["energies"].copy()
    for t in range(60):
        st = O.ksat_anneal(lits, n, beta, t, t + 1, seed=1, replicas=24, init=st["states"],
                           init_best=st["best_states"], init_best_energy=st["best_energies"])
        mins = np.minimum(mins, st["energies"])
    assert np.array_equal(mins, full["best_energies"])
    # a replica's trajectory does not depend on which other replicas run
    ids = np.array([23, 0, 7], dtype=np.int32)
    sub = O.ksat_anneal(lits, n, beta, 0, 60, seed=1, replica_ids=ids)
    assert np.array_equal(sub["states"], full["states"][ids])
    assert np.array_equal(sub["best_energies"], full["best_energies"][ids])
    # the thread split does not matter
    one = O.ksat_anneal(lits, n, beta, 0, 60, seed=1, replicas=24, n_threads=1)
    assert np.array_equal(one["states"], full["states"])


def _chi2_pvalue(counts, probs):
    from scipy import stats
    counts = np.asarray(counts, dtype=np.float64)
    exp = np.asarray(probs) * counts.sum()
    order = np.argsort(exp)
    # pool the smallest expected cells until each pooled cell expects >= 5
    obs_p, exp_p, co, ce = [], [], 0.0, 0.0
    for i in order:
        co += counts[i]
        ce += exp[i]
        if ce >= 5:
            obs_p.append(co)
            exp_p.append(ce)
            co, ce = 0.0, 0.0
    if ce > 0:
        obs_p[-1] += co
        exp_p[-1] += ce
    return stats.chisquare(obs_p, exp_p).pvalue


@pytest.mark.parametrize("beta_num", [128, 256, 512])
def test_homogeneous_chain_samples_boltzmann(beta_num):
    """At a fixed homogeneous beta every single-site Metropolis kernel, and so the
    colour-ordered sweep, leaves exp(-beta E) invariant. beta = beta_num/256 sits on the
    threshold grid, so the integer rule is exact up to 2^-32."""
    n = 7
    lits = small_cnf(n, 24, 3, seed=beta_num)
    beta_v = beta_num / 256.0
    T = 25
    beta = np.full((n, T), beta_v, dtype=np.float32)
    R = 24000
    r = O.ksat_anneal(lits, n, beta, 0, T, seed=77 + beta_num, replicas=R)
    idx = (r["states"].astype(np.int64) << np.arange(n)).sum(axis=1)
    counts = np.bincount(idx, minlength=2 ** n)
    E = energies_numpy(lits, all_states(n))
    w = np.exp(-beta_v * E)
    p = _chi2_pvalue(counts, w / w.sum())
    assert p > 1e-4, p
    # a flipped sign of the energy change would sample exp(+beta E): clearly rejected
    w_bad = np.exp(+beta_v * E)
    assert _chi2_pvalue(counts, w_bad / w_bad.sum()) < 1e-6


# ---------------------------------------------------------------- QAP
def _qap_cost_numpy(F, D, p):
    p = np.asarray(p)
    return int((F * D[np.ix_(p, p)]).sum())


@pytest.mark.parametrize("n", [3, 5, 7, 8])
def test_qap_cost_matches_enumeration(n):
    """All n! permutations (n <= 8): the oracle's cost equals the independent evaluator on every
    one, and so do the optimum and the set of optimal permutations."""
    F, D = W.random_qap(n, 40 + n)
    perms = np.array(list(itertools.permutations(range(n))), dtype=np.int16)
    got = np.array([O.qap_cost(F, D, p) for p in perms])
    # independent evaluator, vectorised over the permutations: sum_ij F_ij D_{p(i) p(j)}
    P = perms.astype(np.int64)
    want = (F[None, :, :] * D[P[:, :, None], P[:, None, :]]).sum(axis=(1, 2))
    assert np.array_equal(got, want)
    assert want.min() >= 0
    best = int(want.min())
    assert set(np.nonzero(got == best)[0].tolist()) == set(np.nonzero(want == best)[0].tolist())
    # F and D symmetric with zero diagonals: every unordered pair is counted twice, so every
    # cost is even
    assert np.all(got % 2 == 0)


def test_qap_swap_delta_matches_recomputation():
    for n in [2, 3, 6, 17]:
        F, D = W.random_qap(n, 60 + n)
        rng = np.random.default_rng(n)
        for _ in range(4):
            p = rng.permutation(n).astype(np.int16)
            c0 = _qap_cost_numpy(F, D, p)
            for r in range(n):
                for s in range(n):
                    if r == s:
                        continue
                    q = p.copy()
                    q[r], q[s] = q[s], q[r]
                    assert O.qap_swap_delta(F, D, p, r, s) == _qap_cost_numpy(F, D, q) - c0


def test_qap_chain_invariants_and_segments():
    n = 11
    F, D = W.random_qap(n, 3)
    beta = W.beta_scaled_linear(n, 40, 0.01, 1.0, 0.5, 1.5, 4)
    full = O.qap_anneal(F, D, beta, 0, 40, seed=9, replicas=20)
    for j in range(20):
        assert sorted(full["perms"][j].tolist()) == list(range(n))
        assert full["energies"][j] == _qap_cost_numpy(F, D, full["perms"][j])
        assert full["best_energies"][j] == _qap_cost_numpy(F, D, full["best_perms"][j])
    assert np.all(full["best_energies"] <= full["energies"])
    a = O.qap_anneal(F, D, beta, 0, 13, seed=9, replicas=20)
    b = O.qap_anneal(F, D, beta, 13, 40, seed=9, replicas=20, init=a["perms"],
                     init_best=a["best_perms"], init_best_energy=a["best_energies"])
    for k1, k2 in [("perms", "perms"), ("energies", "energies"),
                   ("best_energies", "best_energies"), ("best_perms", "best_perms")]:
        assert np.array_equal(b[k1], full[k2])
    ids = np.array([19, 4], dtype=np.int32)
    sub = O.qap_anneal(F, D, beta, 0, 40, seed=9, replica_ids=ids)
    assert np.array_equal(sub["perms"], full["perms"][ids])


def test_qap_infinite_beta_never_goes_uphill():
    n = 20
    F, D = W.random_qap(n, 5)
    T = 10
    beta = np.full((n, T), 65535.0, dtype=np.float32)
    st = O.qap_anneal(F, D, beta, 0, 0, seed=2, replicas=8)
    prev = st["energies"].copy()
    for t in range(T):
        st = O.qap_anneal(F, D, beta, t, t + 1, seed=2, replicas=8, init=st["perms"],
                          init_best=st["best_perms"], init_best_energy=st["best_energies"])
        assert np.all(st["energies"] <= prev)
        prev = st["energies"].copy()


def test_qap_homogeneous_chain_samples_boltzmann():
    n = 4
    rng = np.random.default_rng(8)
    F = rng.integers(0, 4, size=(n, n))
    F = np.triu(F, 1)
    F = (F + F.T).astype(np.int32)
    D = rng.integers(0, 4, size=(n, n))
    D = np.triu(D, 1)
    D = (D + D.T).astype(np.int32)
    beta_v = 64 / 256.0
    T = 20
    beta = np.full((n, T), beta_v, dtype=np.float32)
    R = 24000
    r = O.qap_anneal(F, D, beta, 0, T, seed=31, replicas=R)
    perms = list(itertools.permutations(range(n)))
    index = {p: i for i, p in enumerate(perms)}
    counts = np.zeros(len(perms))
    for row in r["perms"]:
        counts[index[tuple(int(v) for v in row)]] += 1
    E = np.array([_qap_cost_numpy(F, D, np.array(p)) for p in perms])
    w = np.exp(-beta_v * (E - E.min()))
    assert _chi2_pvalue(counts, w / w.sum()) > 1e-4
    w_bad = np.exp(+beta_v * (E - E.min()))
    assert _chi2_pvalue(counts, w_bad / w_bad.sum()) < 1e-6


# ---------------------------------------------------------------- replica exchange (PT)
def test_pt_with_equal_ladder_is_the_plain_chain():
    """All slot temperatures 1.0: every exchange is accepted (d = 0) and the replicas' own
    dynamics (Philox streams by replica id) are those of the plain anneal."""
    wl = W.workload_ksat_small(24)
    lits, n, beta = wl["lits"], wl["n_vars"], wl["beta"]
    L, G = 12, 3
    pt = O.ksat_pt_anneal(lits, n, beta, np.ones(L, np.float32), 0, 24, 3, seed=4,
                          replicas=G * L)
    plain = O.ksat_anneal(lits, n, beta, 0, 24, 4, replicas=G * L)
    for key in ("states", "energies", "best_energies", "best_states"):
        assert np.array_equal(pt[key], plain[key]), key
    # every ladder exchanges within itself: its slots stay a permutation of 0..L-1, and with
    # every exchange accepted the slots follow the closed-form walk of the even/odd pairing:
    # after 8 rounds the replica that started at slot 0 of each ladder sits at slot 8
    for g in range(G):
        assert sorted(pt["slots"][g * L:(g + 1) * L].tolist()) == list(range(L))
        assert pt["slots"][g * L] == 8
    walk = np.arange(L)
    for q in range(8):
        for k in range(q & 1, L - 1, 2):
            a, b = np.where(walk == k)[0][0], np.where(walk == k + 1)[0][0]
            walk[a], walk[b] = k + 1, k
    for g in range(G):
        assert np.array_equal(pt["slots"][g * L:(g + 1) * L], walk)


def test_pt_segments_and_invariants():
    n = 60
    lits = W.random_ksat(n, 4.2, 3, 12)
    beta = W.beta_constant(n, 30, 1.0)
    ladder = W.geometric_profile(0.25, 3.0, 10).astype(np.float32)
    full = O.ksat_pt_anneal(lits, n, beta, ladder, 0, 30, 2, seed=6)
    a = O.ksat_pt_anneal(lits, n, beta, ladder, 0, 11, 2, seed=6)
    b = O.ksat_pt_anneal(lits, n, beta, ladder, 11, 30, 2, seed=6, slots=a["slots"],
                         init=a["states"], init_best=a["best_states"],
                         init_best_energy=a["best_energies"])
    for key in ("states", "energies", "best_energies", "best_states", "slots"):
        assert np.array_equal(b[key], full[key]), key
    assert np.array_equal(full["energies"], energies_numpy(lits, full["states"]))
    assert np.all(full["best_energies"] <= full["energies"])
    assert sorted(full["slots"].tolist()) == list(range(10))
    assert not np.array_equal(full["slots"], np.arange(10))  # some exchanges happened


def test_pt_exchange_keeps_each_slot_boltzmann():
    """Two replicas at beta 0.5 and 2.0 with an exchange round after every sweep: the joint
    chain leaves prod_k exp(-beta_k E(x at slot k)) invariant, so the state found at each slot
    follows the Boltzmann law of that slot's temperature. (Exchanging with the sign of the
    energy difference reversed would break this.)"""
    n = 6
    lits = small_cnf(n, 20, 3, seed=2)
    ladder = np.array([0.5, 2.0], dtype=np.float32)
    T = 24
    beta = W.beta_constant(n, T, 1.0)
    E = energies_numpy(lits, all_states(n))
    counts = [np.zeros(2 ** n), np.zeros(2 ** n)]
    for run in range(1250):  # two ladders per run
        res = O.ksat_pt_anneal(lits, n, beta, ladder, 0, T, 1, seed=1000 + run, replicas=4)
        for r in range(4):
            k = res["slots"][r]
            idx = int((res["states"][r].astype(np.int64) << np.arange(n)).sum())
            counts[k][idx] += 1
    for k, b in enumerate(ladder):
        w = np.exp(-float(b) * E)
        assert _chi2_pvalue(counts[k], w / w.sum()) > 1e-4, k
    w_swapped = np.exp(-float(ladder[1]) * E)
    assert _chi2_pvalue(counts[0], w_swapped / w_swapped.sum()) < 1e-6


# ---------------------------------------------------------------- energy statistics, ladder
def test_energy_statistics_match_the_recorded_trajectory():
    """The sums of E and E^2 over sweeps >= stats_from equal those of the trajectory recorded
    one sweep at a time, with every energy recounted by the independent evaluator."""
    wl = W.workload_ksat_small(30)
    lits, n, beta, R = wl["lits"], wl["n_vars"], wl["beta"], 10
    res = O.ksat_anneal(lits, n, beta, 3, 30, 9, replicas=R, stats_from=12)
    s1 = np.zeros(R, np.int64)
    s2 = np.zeros(R, np.int64)
    state = dict(init=None)
    x = None
    for t in range(3, 30):
        if x is None:
            step = O.ksat_anneal(lits, n, beta, 3, 4, 9, replicas=R)
        else:
            step = O.ksat_anneal(lits, n, beta, t, t + 1, 9, replicas=R, init=x)
        x = step["states"]
        if t >= 12:
            e = energies_numpy(lits, x)
            s1 += e
            s2 += e * e
    assert np.array_equal(res["states"], x)
    assert np.array_equal(res["e_sum"], s1) and np.array_equal(res["e_sq"], s2)


def test_adaptive_ladder_follows_its_definition():
    """Each sigma is the standard deviation of the recorded energies of its level (recounted
    independently, two-pass variance), each step is beta + alpha / sigma, and the ladder stops
    at the first sigma <= sigma_min."""
    n = 60
    lits = W.random_ksat(n, 4.2, 3, 21)
    R, eq, meas = 8, 4, 6
    betas, sigmas = O.adaptive_ladder(lits, n, R, 5, 0.2, 1.1, 0.9, 12, eq, meas)
    T = eq + meas
    x = None
    for i, b in enumerate(betas):
        sched = np.full((n, (i + 1) * T), np.float32(b), np.float32)
        es = []
        for t in range(i * T, (i + 1) * T):
            step = (O.ksat_anneal(lits, n, sched, t, t + 1, 5, replicas=R) if x is None else
                    O.ksat_anneal(lits, n, sched, t, t + 1, 5, replicas=R, init=x))
            x = step["states"]
            if t >= i * T + eq:
                es.append(energies_numpy(lits, x))
        sig = float(np.std(np.concatenate(es)))
        assert abs(sig - sigmas[i]) <= 1e-9 * max(1.0, sig), i
        if i + 1 < len(betas):
            assert betas[i + 1] == b + 1.1 / sigmas[i]
            assert sigmas[i] > 0.9
    assert sigmas[-1] <= 0.9 or len(betas) == 12
    assert np.all(np.diff(betas) > 0)
    # max_temps bounds the ladder; a large sigma_min stops it at once
    b1, s1 = O.adaptive_ladder(lits, n, R, 5, 0.2, 1.1, 1e9, 12, eq, meas)
    assert len(b1) == 1 and b1[0] == np.float64(0.2)
    b3, _ = O.adaptive_ladder(lits, n, R, 5, 0.2, 1.1, 0.0, 3, eq, meas)
    assert len(b3) == 3 and np.array_equal(b3, betas[:3])


def test_adaptive_ladder_measures_the_equilibrium_fluctuation():
    """On a 7-variable formula the sweeps mix fast, so each level's sigma estimates the exact
    canonical standard deviation of E at that level's beta (enumeration of all 2^7 states)."""
    n = 7
    lits = small_cnf(n, 24, 3, seed=8)
    E = energies_numpy(lits, all_states(n)).astype(np.float64)
    betas, sigmas = O.adaptive_ladder(lits, n, 256, 3, 0.1, 0.8, 0.05, 5, 20, 60)
    assert len(betas) >= 3
    for b, sg in zip(betas, sigmas):
        w = np.exp(-float(np.float32(b)) * E)
        w /= w.sum()
        exact = math.sqrt(float((w * E * E).sum() - (w * E).sum() ** 2))
        assert abs(sg - exact) <= 0.06 * exact + 0.01, (b, sg, exact)


# ---------------------------------------------------------------- frozen units, cluster moves
def _state_index(X):
    X = np.asarray(X, dtype=np.int64)
    return (X << np.arange(X.shape[1])).sum(axis=1)


def test_frozen_variables_hold_and_the_rest_is_conditionally_boltzmann():
    """beta = +inf holds a variable; the others then sample the Boltzmann law conditioned on the
    held values (each chain of the two-chain scheme is detailed-balanced on its own subset)."""
    n = 7
    lits = small_cnf(n, 26, 3, seed=12)
    frozen = {1: 1, 4: 0}
    R, T, b = 3000, 30, 0.9
    rng = np.random.default_rng(4)
    init = rng.integers(0, 2, size=(R, n), dtype=np.uint8)
    for v, val in frozen.items():
        init[:, v] = val
    beta = W.beta_constant(n, T, b)
    for v in frozen:
        beta[v, :] = np.inf
    res = O.ksat_anneal(lits, n, beta, 0, T, 7, replicas=R, init=init)
    for v, val in frozen.items():
        assert np.all(res["states"][:, v] == val)
    X = all_states(n)
    keep = np.all([X[:, v] == val for v, val in frozen.items()], axis=0)
    E = energies_numpy(lits, X[keep]).astype(np.float64)
    pos = {int(i): j for j, i in enumerate(_state_index(X[keep]))}
    counts = np.zeros(len(E))
    for i in _state_index(res["states"]):
        counts[pos[int(i)]] += 1
    w = np.exp(-np.float64(np.float32(b)) * E)
    assert _chi2_pvalue(counts, w / w.sum()) > 1e-4
    assert np.array_equal(res["energies"], energies_numpy(lits, res["states"]))


def test_fully_frozen_schedule_changes_nothing():
    wl = W.workload_ksat_small(12)
    beta = np.full_like(wl["beta"], np.inf)
    a = O.ksat_anneal(wl["lits"], wl["n_vars"], beta, 0, 12, 3, replicas=9)
    b = O.ksat_anneal(wl["lits"], wl["n_vars"], beta, 0, 0, 3, replicas=9)
    for key in ("states", "energies", "best_energies", "best_states"):
        assert np.array_equal(a[key], b[key]), key


def test_frozen_qap_facility_holds_and_the_rest_is_conditionally_boltzmann():
    n = 5
    F, D = W.random_qap(n, 77, max_entry=9)
    R, T, b = 3000, 40, 0.08
    beta = W.beta_constant(n, T, b)
    beta[2, :] = np.inf
    rng = np.random.default_rng(3)
    init = np.zeros((R, n), dtype=np.int16)
    for r in range(R):
        rest = rng.permutation([0, 1, 3, 4])
        init[r] = [rest[0], rest[1], 2, rest[2], rest[3]]
    res = O.qap_anneal(F, D, beta, 0, T, 5, replicas=R, init=init)
    assert np.all(res["perms"][:, 2] == 2)
    perms = [p for p in itertools.permutations(range(n)) if p[2] == 2]
    pos = {p: j for j, p in enumerate(perms)}
    E = np.array([_qap_cost_numpy(F, D, np.array(p)) for p in perms], dtype=np.float64)
    counts = np.zeros(len(perms))
    for p in res["perms"]:
        counts[pos[tuple(int(x) for x in p)]] += 1
    w = np.exp(-np.float64(np.float32(b)) * (E - E.min()))
    assert _chi2_pvalue(counts, w / w.sum()) > 1e-4


def test_schedule_is_read_at_the_sweep_and_the_variable_it_names():
    """beta[v][t] is 0 (every attempt flips) or +inf (held), alternating in t with a phase of its
    own per variable: after t1 sweeps variable v has flipped once for every free sweep t < t1,
    so reading another sweep's column or another variable's row changes the final state."""
    n, T, R = 40, 9, 33
    lits = W.random_ksat(n, 4.2, 3, 19)
    phase = W.seeded_subset(n, 0.5, 21).astype(np.int64)  # variable v is held when t % 2 == phase
    t = np.arange(T)
    held = (t[None, :] % 2) == phase[:, None]
    beta = np.where(held, np.float32(np.inf), np.float32(0.0)).astype(np.float32)
    x0 = O.ksat_anneal(lits, n, beta, 0, 0, seed=4, replicas=R)["states"]
    for t1 in (1, 2, 5, 9):
        res = O.ksat_anneal(lits, n, beta, 0, t1, seed=4, replicas=R)
        free = (~held[:, :t1]).sum(axis=1) % 2
        assert np.array_equal(res["states"], x0 ^ free[None, :].astype(np.uint8)), t1
        assert np.array_equal(res["energies"], energies_numpy(lits, res["states"]))


def test_qap_schedule_is_read_at_the_step_it_names():
    """Every facility free at beta = 0 on even steps and held on odd ones: an odd step changes
    no permutation, an even one changes almost all of them."""
    n, R, T = 9, 64, 8
    F, D = W.random_qap(n, 23)
    beta = np.zeros((n, T), dtype=np.float32)
    beta[:, 1::2] = np.inf
    perms = [O.qap_anneal(F, D, beta, 0, t1, 6, replicas=R)["perms"] for t1 in range(T + 1)]
    for t in range(T):
        if t % 2:
            assert np.array_equal(perms[t + 1], perms[t]), t
        else:
            assert (perms[t + 1] != perms[t]).any(axis=1).mean() > 0.9, t


def _perm_parity(p):
    p, seen, odd = list(p), set(), 0
    for i in range(len(p)):
        if i in seen:
            continue
        j, length = i, 0
        while j not in seen:
            seen.add(j)
            j, length = p[j], length + 1
        odd ^= (length - 1) & 1
    return odd


def test_qap_step_is_n_transpositions_at_beta_zero():
    """At beta = 0 every swap attempt is accepted and every attempt exchanges two distinct
    facilities, so one step of n attempts multiplies the permutation's sign by (-1)^n. A step of
    another length, or a proposal that can pick r = s, breaks the closed form."""
    for n in (3, 4, 5, 7):
        F, D = W.random_qap(n, 50 + n)
        T, R = 6, 50
        beta = np.zeros((n, T), dtype=np.float32)
        p0 = O.qap_anneal(F, D, beta, 0, 0, 8, replicas=R)["perms"]
        par0 = np.array([_perm_parity(p) for p in p0])
        for t1 in range(1, T + 1):
            pt = O.qap_anneal(F, D, beta, 0, t1, 8, replicas=R)["perms"]
            part = np.array([_perm_parity(p) for p in pt])
            assert np.array_equal(part, par0 ^ ((n * t1) & 1)), (n, t1)


def _chain_of(lits, n, states):
    e = energies_numpy(lits, states)
    return dict(states=states.copy(), energies=e, best_states=states.copy(), best_energies=e.copy())


def test_cluster_flip_limits():
    """beta 0 accepts every proposal; beta 65535 accepts exactly the non-increasing ones; the
    best-so-far is the minimum of the energies seen."""
    n = 40
    lits = W.random_ksat(n, 4.2, 3, 31)
    rng = np.random.default_rng(5)
    X = rng.integers(0, 2, size=(64, n), dtype=np.uint8)
    M = rng.integers(0, 2, size=(64, n), dtype=np.uint8)
    ch = _chain_of(lits, n, X)
    hot = O.ksat_cluster_flip(lits, n, ch, M, 0.0, 1, 9)
    assert np.all(hot["accepted"] == 1)
    assert np.array_equal(hot["states"], X ^ M)
    assert np.array_equal(hot["energies"], energies_numpy(lits, X ^ M))
    assert np.array_equal(hot["best_energies"], np.minimum(ch["energies"], hot["energies"]))
    cold = O.ksat_cluster_flip(lits, n, ch, M, 65535.0, 1, 9)
    down = energies_numpy(lits, X ^ M) <= ch["energies"]
    assert np.array_equal(cold["accepted"].astype(bool), down)
    want = np.where(down[:, None], X ^ M, X)
    assert np.array_equal(cold["states"], want)
    # one shared mask row acts on every replica
    one = O.ksat_cluster_flip(lits, n, ch, M[:1], 0.0, 1, 9)
    assert np.array_equal(one["states"], X ^ M[:1])


def test_cluster_flip_sampled_replicas_with_their_own_masks():
    """A sample of replicas, given by id with one mask row per row passed, moves exactly as the
    same replicas do inside the whole set (ids far beyond the sample's size included): the id
    picks the Philox stream, row r of the mask goes with row r of the states."""
    n, R = 40, 64
    lits = W.random_ksat(n, 4.2, 3, 32)
    rng = np.random.default_rng(6)
    X = rng.integers(0, 2, size=(R, n), dtype=np.uint8)
    M = rng.integers(0, 2, size=(R, n), dtype=np.uint8)
    beta = np.linspace(0.2, 1.5, R).astype(np.float32)
    whole = O.ksat_cluster_flip(lits, n, _chain_of(lits, n, X), M, beta, 7, 11)
    assert 0 < int(whole["accepted"].sum()) < R  # both outcomes occur
    ids = np.array([63, 5, 40, 0, 62])
    part = O.ksat_cluster_flip(lits, n, _chain_of(lits, n, X[ids]), M[ids], beta[ids], 7, 11,
                               replica_ids=ids)
    for key in ("states", "energies", "best_energies", "best_states", "accepted"):
        assert np.array_equal(part[key], whole[key][ids]), key
    # a mask with neither one row nor one per row passed is rejected
    with pytest.raises(ValueError):
        O.ksat_cluster_flip(lits, n, _chain_of(lits, n, X[ids]), M, beta[ids], 7, 11,
                            replica_ids=ids)


def test_cluster_flip_accepts_with_the_boltzmann_factor():
    """A proposal with energy change dE > 0 at beta = 0.5 (on the table's grid) is accepted with
    frequency exp(-0.5 dE) over independent draws (replicas and move ids)."""
    n = 30
    lits = W.random_ksat(n, 4.2, 3, 8)
    rng = np.random.default_rng(1)
    while True:
        x = rng.integers(0, 2, size=n, dtype=np.uint8)
        m = rng.integers(0, 2, size=n, dtype=np.uint8)
        dE = int(energies_numpy(lits, (x ^ m)[None])[0] - energies_numpy(lits, x[None])[0])
        if 1 <= dE <= 4:
            break
    R = 4096
    ch = _chain_of(lits, n, np.repeat(x[None], R, axis=0))
    hits = 0
    for mid in range(5):
        hits += int(O.ksat_cluster_flip(lits, n, ch, m, 0.5, mid, 3)["accepted"].sum())
    p = math.exp(-0.5 * dE)
    tot = 5 * R
    z = (hits - tot * p) / math.sqrt(tot * p * (1 - p))
    assert abs(z) < 4.5, (dE, hits / tot, p)


def test_cluster_moves_keep_the_boltzmann_law():
    """Sweeps interleaved with collective flips of a fixed half of the variables (a symmetric
    proposal) at one beta: the final states follow the Boltzmann law."""
    n = 6
    lits = small_cnf(n, 20, 3, seed=4)
    R, rounds, b = 3000, 12, 0.8
    beta = W.beta_constant(n, rounds, b)
    mask = np.array([1, 0, 1, 1, 0, 0], dtype=np.uint8)
    ch = None
    for t in range(rounds):
        if ch is None:
            ch = O.ksat_anneal(lits, n, beta, 0, 1, 21, replicas=R)
        else:
            ch = O.ksat_anneal(lits, n, beta, t, t + 1, 21, replicas=R, init=ch["states"],
                               init_best=ch["best_states"], init_best_energy=ch["best_energies"])
        ch = O.ksat_cluster_flip(lits, n, ch, mask, b, t, 21)
    E = energies_numpy(lits, all_states(n)).astype(np.float64)
    counts = np.bincount(_state_index(ch["states"]), minlength=2 ** n)
    w = np.exp(-np.float64(np.float32(b)) * E)
    assert _chi2_pvalue(counts, w / w.sum()) > 1e-4
    w_bad = np.exp(+np.float64(np.float32(b)) * E)
    assert _chi2_pvalue(counts, w_bad / w_bad.sum()) < 1e-6


# ---------------------------------------------------------------- CNF LBP and backbones
def _tree_cnf(seed):
    """A CNF whose factor graph is a tree: every clause after the first shares exactly one
    variable with the clauses before it. 13 variables, clauses of 2 to 4 literals."""
    rng = np.random.default_rng(seed)
    groups = [[0, 1, 2], [2, 3, 4], [2, 5], [4, 6, 7], [7, 8, 9, 10], [1, 11], [11, 12]]
    lits = np.zeros((len(groups), 4), np.int32)
    for a, g in enumerate(groups):
        lits[a, :len(g)] = (np.array(g) + 1) * rng.choice([-1, 1], size=len(g))
    return lits, 13


def _exact_cnf_marginals(lits, n, x_star, eps, beta, lam):
    """<r_i> and <prod_{i in a} r_i> under P(r) ~ prod_a omega_a(r) prod_i exp(lam eps_i s*_i r_i)
    by enumeration of all 2^n states (omega_a = exp(-2 beta) when clause a is violated)."""
    X = all_states(n)
    Rs = 2.0 * X - 1.0
    viol = energies_numpy(lits, X).astype(np.float64)
    s = 2.0 * np.asarray(x_star, np.float64) - 1.0
    logw = -2.0 * beta * viol + (Rs * (lam * np.asarray(eps) * s)).sum(axis=1)
    w = np.exp(logw - logw.max())
    w /= w.sum()
    marg = (w[:, None] * Rs).sum(axis=0)
    corr = []
    for row in lits:
        vs = np.abs(row[row != 0]) - 1
        corr.append(float((w * Rs[:, vs].prod(axis=1)).sum()))
    return marg, np.array(corr)


@pytest.mark.parametrize("seed,beta,lam", [(1, 0.7, 0.3), (2, 2.0, 0.1), (3, 1.2, 0.0),
                                           (4, 3.0, 0.05)])
def test_lbp_is_exact_on_a_tree(seed, beta, lam):
    """Belief propagation is exact on a tree factor graph: the oracle's fixed point gives the
    enumerated marginals and clause correlations of the surrogate distribution."""
    lits, n = _tree_cnf(seed)
    x = np.random.default_rng(seed + 10).integers(0, 2, n).astype(np.uint8)
    eps = O.clause_degrees(lits, n)
    r = O.cnf_lbp(lits, n, x, beta, [lam], 1e-15, 200, eps=eps)
    assert r["n_done"] == 1
    marg, corr = _exact_cnf_marginals(lits, n, x, eps, beta, lam)
    assert np.allclose(r["marg"], marg, atol=1e-10, rtol=0)
    assert np.allclose(r["corr"], corr, atol=1e-10, rtol=0)
    s = 2.0 * x - 1.0
    assert abs(r["p"] - float((s * marg).mean())) < 1e-10
    assert abs(r["q1"] - float((marg ** 2).mean())) < 1e-10


def test_lbp_at_zero_beta_leaves_the_bias_alone():
    n = 60
    lits = W.random_ksat(n, 4.2, 3, 2)
    x = np.random.default_rng(3).integers(0, 2, n).astype(np.uint8)
    eps = O.clause_degrees(lits, n)
    r = O.cnf_lbp(lits, n, x, 0.0, [0.07], 1e-14, 50, eps=eps)
    field = 0.07 * eps * (2.0 * x - 1.0)
    assert np.allclose(r["marg"], np.tanh(field), atol=1e-14, rtol=0)
    want = [np.prod(np.tanh(field[np.abs(row[row != 0]) - 1])) for row in lits]
    assert np.allclose(r["corr"], want, atol=1e-14, rtol=0)


def test_lbp_continuation_falls_back_to_the_last_converged_lambda():
    n = 300
    lits = W.random_ksat(n, 9.6, 4, 6)
    x = np.random.default_rng(4).integers(0, 2, n).astype(np.uint8)
    lams = [0.5, 0.2, 0.1, 0.05, 0.02, 0.01, 0.005]
    full = O.cnf_lbp(lits, n, x, 1.0, lams, 1e-9, 15)
    k = full["n_done"]
    assert 0 < k < len(lams), full["iters"]
    assert full["iters"][k] == 15 and full["deltas"][k] >= 1e-9 and full["lam"] == lams[k - 1]
    part = O.cnf_lbp(lits, n, x, 1.0, lams[:k], 1e-9, 15)
    assert part["n_done"] == k
    for key in ("marg", "corr"):
        assert np.array_equal(full[key], part[key]), key
    assert np.all(full["iters"][k + 1:] == 0)


def _components_union_find(lits, n, corr, beta, seed_thr, cutoff):
    parent = list(range(n))

    def find(a):
        while parent[a] != a:
            parent[a] = parent[parent[a]]
            a = parent[a]
        return a
    jt = np.arctanh(np.abs(corr)) / beta
    link = (jt > cutoff) | (jt > seed_thr)
    touched = np.zeros(n, bool)
    for a, row in enumerate(lits):
        if not link[a]:
            continue
        vs = np.abs(row[row != 0]) - 1
        touched[vs] = True
        for v in vs[1:]:
            ra, rb = find(int(vs[0])), find(int(v))
            if ra != rb:
                parent[max(ra, rb)] = min(ra, rb)
    seeded = set()
    for a, row in enumerate(lits):
        if jt[a] > seed_thr:
            seeded.add(find(int(np.abs(row[row != 0])[0]) - 1))
    lab = np.full(n, -1, np.int32)
    for v in range(n):
        if touched[v] and find(v) in seeded:
            lab[v] = find(v)
    return lab


@pytest.mark.parametrize("seed", [0, 1, 2])
def test_backbones_are_the_seeded_components(seed):
    """Clusters grown seed by seed (the oracle) equal the connected components, under the
    factors above the cutoff, that hold a seed factor (union-find), labelled by their smallest
    variable."""
    n = 400
    lits = W.random_ksat(n, 4.2, 3, 70 + seed)
    rng = np.random.default_rng(seed)
    corr = np.tanh(rng.exponential(0.6, lits.shape[0])) * rng.choice([-1, 1], lits.shape[0])
    for seed_thr, cutoff in [(1.5, 1.2), (2.0, 0.9), (0.8, 1.0)]:
        lab, nc = O.cnf_backbone(lits, n, corr, 1.0, seed_thr, cutoff)
        want = _components_union_find(lits, n, corr, 1.0, seed_thr, cutoff)
        assert np.array_equal(lab, want)
        assert nc == len(set(want[want >= 0].tolist()))


def test_backbone_schedule_layout():
    lab = np.array([-1, 3, 3, -1, 0], np.int32)
    b = O.backbone_schedule(lab, 2.0, 4.0, 2, 3, 2, 1)
    assert b.shape == (5, 12) and b.dtype == np.float32
    hot, cold, unl = b[:, 0:3], b[:, 3:5], b[:, 5:6]
    bb = lab >= 0
    assert np.all(hot[bb] == np.float32(0.5)) and np.all(np.isinf(hot[~bb]))
    assert np.all(np.isinf(cold[bb])) and np.all(cold[~bb] == 2.0)
    assert np.all(unl == 2.0)
    assert np.array_equal(b[:, :6], b[:, 6:])


# ---------------------------------------------------------------- whitening
def _blocking(lits, n, x, star, generalized):
    """blocked[v]: some clause containing v is neither satisfied by another of its variables nor
    holds another white variable (and, generalized, is satisfied by v) — numpy, per clause."""
    lits = np.asarray(lits)
    used = lits != 0
    var = np.where(used, np.abs(lits) - 1, 0)
    val = (x[var] == (lits > 0)) & used
    st = star[var] & used
    blocked = np.zeros(n, bool)
    for q in range(lits.shape[1]):
        others = np.ones(lits.shape[1], bool)
        others[q] = False
        other_true = val[:, others].any(axis=1)
        other_star = st[:, others].any(axis=1)
        b = used[:, q] & ~other_true & ~other_star
        if generalized:
            b &= val[:, q]
        np.logical_or.at(blocked, var[b, q], True)
    return blocked


@pytest.mark.parametrize("generalized", [True, False])
def test_whitening_is_the_least_fixed_point(generalized):
    """The oracle's one-at-a-time result is a fixed point (white = unblocked, frozen = blocked,
    by an independent evaluator) and equals the parallel-round closure from no white variable."""
    n = 400
    lits = W.random_ksat(n, 4.2, 3, 12)
    beta = W.beta_constant(n, 60, 4.0)
    X = O.ksat_anneal(lits, n, beta, 0, 60, 2, replicas=6)["states"]
    for x in X:
        fr, cnt = O.ksat_whitening(lits, n, x, generalized)
        star = fr == 0
        assert cnt == int(fr.sum())
        blocked = _blocking(lits, n, x, star, generalized)
        assert np.array_equal(blocked, ~star)
        s = np.zeros(n, bool)
        while True:
            s2 = s | ~_blocking(lits, n, x, s, generalized)
            if np.array_equal(s2, s):
                break
            s = s2
        assert np.array_equal(s, star)


def test_whitening_reports_no_false_frozen_variables():
    """On solutions of small satisfiable formulas, a variable the procedure calls frozen takes
    the same value in every solution reachable from the given one by single flips through
    solutions (its cluster), found by enumerating all 2^14 assignments."""
    n = 14
    seen_frozen = 0
    for seed in range(6):
        lits = small_cnf(n, 50, 3, seed=100 + seed)
        X = all_states(n)
        sol = X[energies_numpy(lits, X) == 0]
        if len(sol) == 0:
            continue
        idx = {int(i): j for j, i in enumerate(_state_index(sol))}
        for j0 in range(0, len(sol), max(1, len(sol) // 5)):
            comp, todo = {j0}, [j0]
            while todo:
                j = todo.pop()
                for v in range(n):
                    y = sol[j].copy()
                    y[v] ^= 1
                    k = idx.get(int(_state_index(y[None])[0]))
                    if k is not None and k not in comp:
                        comp.add(k)
                        todo.append(k)
            cl = sol[sorted(comp)]
            fr, _ = O.ksat_whitening(lits, n, sol[j0])
            fr_std, _ = O.ksat_whitening(lits, n, sol[j0], generalized=False)
            assert np.array_equal(fr, fr_std)  # no violated clause: both forms agree
            for v in np.nonzero(fr)[0]:
                assert np.all(cl[:, v] == sol[j0, v]), (seed, j0, v)
            seen_frozen += int(fr.sum())
    assert seen_frozen > 0


def test_whitening_generalized_whitens_more_on_low_energy_states():
    n = 300
    lits = W.random_ksat(n, 9.6, 4, 5)
    X = O.ksat_anneal(lits, n, W.beta_constant(n, 80, 3.0), 0, 80, 4, replicas=5)["states"]
    assert energies_numpy(lits, X).min() > 0
    for x in X:
        g, cg = O.ksat_whitening(lits, n, x, True)
        s, cs = O.ksat_whitening(lits, n, x, False)
        assert np.all(g <= s) and cg <= cs
    # a unit clause is the only satisfier of its variable: frozen; nothing else is
    lits2 = np.array([[1, 0, 0], [2, 3, 0]], np.int32)
    fr, c = O.ksat_whitening(lits2, 3, np.array([1, 1, 1], np.uint8))
    assert fr.tolist() == [1, 0, 0] and c == 1


# ---------------------------------------------------------------- QAP replica exchange
def test_qap_pt_equal_ladder_is_the_plain_chain_and_segments():
    n, T = 9, 20
    F, D = W.random_qap(n, 31)
    beta = W.beta_scaled_linear(n, T, 0.01, 1.0, 0.5, 1.5, 2)
    L, G = 6, 2
    pt = O.qap_pt_anneal(F, D, beta, np.ones(L, np.float32), 0, T, 2, 5, replicas=G * L)
    plain = O.qap_anneal(F, D, beta, 0, T, 5, replicas=G * L)
    for a, b in (("perms", "perms"), ("energies", "energies"), ("best_energies", "best_energies"),
                 ("best_perms", "best_perms")):
        assert np.array_equal(pt[a], plain[b]), a
    ladder = W.geometric_profile(0.02, 0.5, L).astype(np.float32)
    full = O.qap_pt_anneal(F, D, beta, ladder, 0, T, 3, 5, replicas=G * L)
    a = O.qap_pt_anneal(F, D, beta, ladder, 0, 7, 3, 5, replicas=G * L)
    b = O.qap_pt_anneal(F, D, beta, ladder, 7, T, 3, 5, replicas=G * L, slots=a["slots"],
                        init=a["perms"], init_best=a["best_perms"],
                        init_best_energy=a["best_energies"])
    for key in ("perms", "energies", "best_energies", "best_perms", "slots"):
        assert np.array_equal(b[key], full[key]), key
    for r in range(G * L):
        assert full["energies"][r] == _qap_cost_numpy(F, D, full["perms"][r])
    for g in range(G):
        assert sorted(full["slots"][g * L:(g + 1) * L].tolist()) == list(range(L))


def test_qap_pt_keeps_each_slot_boltzmann():
    n = 4
    F, D = W.random_qap(n, 14, max_entry=9)
    perms = list(itertools.permutations(range(n)))
    pos = {p: j for j, p in enumerate(perms)}
    E = np.array([_qap_cost_numpy(F, D, np.array(p)) for p in perms], dtype=np.float64)
    ladder = np.array([0.02, 0.15], dtype=np.float32)
    T = 24
    beta = W.beta_constant(n, T, 1.0)
    counts = [np.zeros(len(perms)), np.zeros(len(perms))]
    for run in range(1250):
        res = O.qap_pt_anneal(F, D, beta, ladder, 0, T, 1, 3000 + run, replicas=4)
        for r in range(4):
            counts[res["slots"][r]][pos[tuple(int(x) for x in res["perms"][r])]] += 1
    for k, b in enumerate(ladder):
        w = np.exp(-np.float64(b) * (E - E.min()))
        assert _chi2_pvalue(counts[k], w / w.sum()) > 1e-4, k
    w = np.exp(-np.float64(ladder[0]) * (E - E.min()))
    assert _chi2_pvalue(counts[1], w / w.sum()) < 1e-6


def test_qap_energy_statistics_and_ladder_follow_their_definition():
    n = 7
    F, D = W.random_qap(n, 41)
    R, eq, meas = 6, 3, 5
    betas, sigmas = O.qap_adaptive_ladder(F, D, R, 5, 0.001, 1.1, 0.5, 6, eq, meas)
    T = eq + meas
    x = None
    for i, b in enumerate(betas):
        sched = np.full((n, (i + 1) * T), np.float32(b), np.float32)
        es = []
        for t in range(i * T, (i + 1) * T):
            step = (O.qap_anneal(F, D, sched, t, t + 1, 5, replicas=R) if x is None else
                    O.qap_anneal(F, D, sched, t, t + 1, 5, replicas=R, init=x))
            x = step["perms"]
            if t >= i * T + eq:
                es.append([_qap_cost_numpy(F, D, p) for p in x])
        es = np.array(es, dtype=np.float64)  # [steps, replicas]
        sig = float(np.std(es))
        assert abs(sig - sigmas[i]) <= 1e-9 * max(1.0, sig), i
        if i + 1 < len(betas):
            assert betas[i + 1] == b + 1.1 / sigmas[i]
    # the statistics themselves: per replica, the costs of the measured steps summed in order
    res = O.qap_anneal(F, D, np.full((n, 12), np.float32(0.01), np.float32), 0, 12, 2,
                       replicas=R, stats_from=4)
    y = None
    s1 = np.zeros(R)
    s2 = np.zeros(R)
    for t in range(12):
        step = (O.qap_anneal(F, D, np.full((n, 12), np.float32(0.01), np.float32), t, t + 1, 2,
                             replicas=R) if y is None else
                O.qap_anneal(F, D, np.full((n, 12), np.float32(0.01), np.float32), t, t + 1, 2,
                             replicas=R, init=y))
        y = step["perms"]
        if t >= 4:
            c = np.array([_qap_cost_numpy(F, D, p) for p in y], dtype=np.float64)
            s1 += c
            s2 += c * c
    assert np.array_equal(res["e_sum"], s1) and np.array_equal(res["e_sq"], s2)


def test_qap_ladder_measures_the_equilibrium_fluctuation():
    n = 4
    F, D = W.random_qap(n, 14, max_entry=9)
    perms = list(itertools.permutations(range(n)))
    E = np.array([_qap_cost_numpy(F, D, np.array(p)) for p in perms], dtype=np.float64)
    betas, sigmas = O.qap_adaptive_ladder(F, D, 512, 3, 0.005, 0.6, 1.0, 5, 20, 60)
    assert len(betas) >= 3
    for b, sg in zip(betas, sigmas):
        w = np.exp(-float(np.float32(b)) * (E - E.min()))
        w /= w.sum()
        exact = math.sqrt(float((w * E * E).sum() - (w * E).sum() ** 2))
        assert abs(sg - exact) <= 0.06 * exact + 0.05, (b, sg, exact)
