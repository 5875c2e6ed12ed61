"""nmc_batch_run_noalloc against nmc_batch_run (GPU).

nmc_batch_run_noalloc serves host programs that cannot allocate device memory when they run
a batch: for example a plugin inside a framework whose caching allocator holds all free device
memory, or a loop that cannot afford the device-wide synchronisation an allocation may bring.
Its work list lives in a fixed 1 MiB device array of the library. This file is collected last
so that a failure here cannot stop the other GPU tests from running first.
"""
import ctypes

import numpy as np
import pytest

import nmc_inputs as W

pytestmark = pytest.mark.gpu
KEYS = ("states", "energies", "best_energies", "best_states")


def _noalloc(ctx, rs, t0, t1):
    """Calls the entry point through the C ABI with plain int32 arrays."""
    n = len(rs)
    arr = ctypes.c_int32 * n
    return ctx._lib.nmc_batch_run_noalloc(ctx._h, n, arr(*rs), arr(*t0), arr(*t1))


def test_noalloc_matches_batch_run_on_two_calls():
    import paper_2111_13628_gb300 as nmc
    ctx = nmc.Context(0)
    specs = [(400, 9.6, 4, 70, 40), (1200, 4.2, 3, 33, 40), (150, 2.0, 6, 96, 40)]
    a_sets, b_sets, insts = [], [], []
    for i, (n, alpha, k, R, T) in enumerate(specs):
        lits = W.random_ksat(n, alpha, k, 900 + i)
        inst = ctx.load_ksat(lits, n)
        ctx.set_schedule(inst, W.beta_inhomogeneous_linear(n, T, 0.5, 4.0, 0.3, 0.5, 910 + i))
        a_sets.append(ctx.replicas_create(inst, R, seed=920 + i))
        b_sets.append(ctx.replicas_create(inst, R, seed=920 + i))
        insts.append(inst)
    for t0, t1 in [(0, 15), (15, 40)]:  # two calls in a row
        ctx.batch_run(a_sets, t0, t1)
        assert _noalloc(ctx, b_sets, [t0] * 3, [t1] * 3) == nmc.NMC_OK
        for a, b in zip(a_sets, b_sets):
            ga, gb = ctx.replicas_read(a), ctx.replicas_read(b)
            for key in KEYS:
                assert np.array_equal(ga[key], gb[key]), (t0, key)
    for a, b, inst in zip(a_sets, b_sets, insts):
        ctx.replicas_destroy(a)
        ctx.replicas_destroy(b)
        ctx.unload(inst)
    ctx.close()


def test_noalloc_rejects_more_items_than_its_array_holds():
    import paper_2111_13628_gb300 as nmc
    ctx = nmc.Context(0)
    n = 20
    inst = ctx.load_ksat(W.random_ksat(n, 4.2, 3, 1), n)
    ctx.set_schedule(inst, W.beta_constant(n, 2, 1.0))
    # the array holds (1 MiB - 256 B) / 136 B = 7708 items (32-replica words)
    sets = [ctx.replicas_create(inst, 4096, seed=s) for s in range(61)]  # 61 x 128 = 7808 words
    rc = _noalloc(ctx, sets, [0] * 61, [1] * 61)
    assert rc == nmc.NMC_EINVAL
    assert b"scratch" in ctx._lib.nmc_last_error(ctx._h)
    # 7680 words fit: the items near the top of the array give what nmc_batch_run gives for
    # twin sets (same seeds), set by set
    twins = [ctx.replicas_create(inst, 4096, seed=s) for s in range(60)]
    assert _noalloc(ctx, sets[:60], [0] * 60, [1] * 60) == nmc.NMC_OK
    ctx.batch_run(twins, 0, 1)
    for a, b in zip(sets[:60], twins):
        ga, gb = ctx.replicas_read(a), ctx.replicas_read(b)
        for key in KEYS:
            assert np.array_equal(ga[key], gb[key]), key
    ctx.sync()
    for s in sets + twins:
        ctx.replicas_destroy(s)
    ctx.unload(inst)
    ctx.close()
