"""The batched-sweep autotuner: it must leave the replica sets exactly as it found them, report
launchable shapes, and the tuned launches must still match the oracle bit for bit."""
import numpy as np
import pytest

import nmc_inputs as W
import oracle as O

pytestmark = pytest.mark.gpu
KEYS = ("states", "energies", "best_energies", "best_states")


def test_autotune_leaves_sets_alone_and_tuned_runs_match_oracle():
    import paper_2111_13628_gb300 as nmc
    ctx = nmc.Context(0)
    specs = [(700, 9.6, 4, 70, 11), (1200, 4.2, 3, 40, 12), (300, 2.5, 6, 33, 13)]
    T = 24
    sets, want = [], []
    for n, alpha, k, R, seed in specs:
        lits = W.random_ksat(n, alpha, k, seed)
        beta = W.beta_inhomogeneous_linear(n, T, 0.3, 3.0, 0.3, 0.5, seed + 7)
        inst = ctx.load_ksat(lits, n)
        ctx.set_schedule(inst, beta)
        rs = ctx.replicas_create(inst, R, seed)
        ctx.replicas_run(rs, 0, 5)
        sets.append(rs)
        want.append(O.ksat_anneal(lits, n, beta, 0, T, seed, replicas=R))
    before = [ctx.replicas_read(rs) for rs in sets]
    shapes = ctx.batch_autotune(sets, 5, 6)
    after = [ctx.replicas_read(rs) for rs in sets]
    for b, a in zip(before, after):
        for key in KEYS:
            assert np.array_equal(a[key], b[key]), key
    for q in range(2):  # both occurrence widths are present in this batch
        cs, lanes, us = shapes[q]
        assert cs in (1, 2, 4, 8) and lanes in (1, 4, 8) and us > 0, shapes
    ctx.batch_run(sets, 5, T)          # the tuned shapes
    for rs, w in zip(sets, want):
        got = ctx.replicas_read(rs)
        for key in KEYS:
            assert np.array_equal(got[key], w[key]), key
    for rs in sets:                    # single sets through the tuned table as well
        ctx.replicas_reset(rs, 99)
    ctx.close()


def test_autotune_argument_checks():
    import paper_2111_13628_gb300 as nmc
    ctx = nmc.Context(0)
    n = 50
    inst = ctx.load_ksat(W.random_ksat(n, 4.2, 3, 1), n)
    ctx.set_schedule(inst, W.beta_constant(n, 4, 1.0))
    rs = ctx.replicas_create(inst, 32, 1)
    for t0, sweeps, code in [(0, 0, nmc.NMC_EINVAL), (-1, 2, nmc.NMC_EINVAL), (2, 5, nmc.NMC_ESTATE)]:
        with pytest.raises(nmc.NmcError) as e:
            ctx.batch_autotune([rs], t0, sweeps)
        assert e.value.code == code
    ctx.close()
