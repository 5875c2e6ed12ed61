"""Serving loop: requests that overlap on the device give, each, exactly what they give alone,
and that is the oracle's result for the request (bit for bit: all outputs are integers)."""
import threading
import time

import numpy as np
import pytest

import nmc_inputs as W
import oracle as O

pytestmark = pytest.mark.gpu
KEYS = ("states", "energies", "best_energies", "best_states")


def _requests():
    reqs = []
    for i, (n, alpha, k, T, R) in enumerate([(700, 9.6, 4, 60, 32), (2500, 9.2, 4, 40, 32),
                                             (300, 4.2, 3, 90, 64), (5000, 9.8, 4, 25, 32),
                                             (150, 9.6, 4, 200, 96)]):
        lits = W.random_ksat(n, alpha, k, 300 + i)
        beta = W.beta_inhomogeneous_linear(n, T, 0.5, 4.0, 0.3, 0.5, 400 + i)
        reqs.append(("ksat", dict(lits=lits, n_vars=n, beta=beta, replicas=R, seed=500 + i)))
    for i, (n, T, R) in enumerate([(40, 12, 256), (97, 6, 256)]):
        F, D = W.random_qap(n, 600 + i)
        beta = W.beta_scaled_linear(n, T, 0.01, 1.0, 0.5, 1.5, 700 + i)
        reqs.append(("qap", dict(F=F, D=D, beta=beta, replicas=R, seed=800 + i)))
    return reqs


def _oracle(kind, r):
    T = r["beta"].shape[1]
    if kind == "ksat":
        return O.ksat_anneal(r["lits"], r["n_vars"], r["beta"], 0, T, r["seed"],
                             replicas=r["replicas"])
    o = O.qap_anneal(r["F"], r["D"], r["beta"], 0, T, r["seed"], replicas=r["replicas"])
    return dict(states=o["perms"], energies=o["energies"], best_energies=o["best_energies"],
                best_states=o["best_perms"])


def _alone(kind, r):
    import paper_2111_13628_gb300 as nmc
    with nmc.Context(0) as ctx:
        if kind == "ksat":
            inst = ctx.load_ksat(r["lits"], r["n_vars"])
        else:
            inst = ctx.load_qap(r["F"], r["D"])
        ctx.set_schedule(inst, r["beta"])
        return ctx.anneal(inst, r["replicas"], 0, r["beta"].shape[1], r["seed"])


def test_mixed_requests_match_alone():
    import paper_2111_13628_gb300 as nmc
    reqs = _requests()
    ids = [None] * len(reqs)
    with nmc.Server(0, max_active=4, slice_log2=14) as srv:
        def submit(i):
            time.sleep(0.002 * i)  # staggered arrivals while earlier requests run
            kind, r = reqs[i]
            if kind == "ksat":
                ids[i] = srv.submit_ksat(r["lits"], r["n_vars"], beta=r["beta"],
                                         replicas=r["replicas"], seed=r["seed"])
            else:
                ids[i] = srv.submit_qap(r["F"], r["D"], beta=r["beta"], replicas=r["replicas"],
                                        seed=r["seed"])
        th = [threading.Thread(target=submit, args=(i,)) for i in range(len(reqs))]
        for t in th:
            t.start()
        for t in th:
            t.join()
        outs = []
        for i in ids:
            deadline = time.time() + 120
            while srv.poll(i, wait_ms=200) in (0, 1) and time.time() < deadline:
                pass
            outs.append(srv.result(i))
        st = srv.stats()
        assert st["ticks"] > 1 and st["attempts"] > 0
    for (kind, r), (got, lat) in zip(reqs, outs):
        assert lat > 0
        want = _alone(kind, r)
        orc = _oracle(kind, r)
        for key in KEYS:
            assert np.array_equal(got[key], want[key]), (kind, key)
            assert np.array_equal(got[key], orc[key]), (kind, key)


def test_factored_requests_match_alone():
    import paper_2111_13628_gb300 as nmc
    n, T = 3000, 50
    lits = W.random_ksat(n, 9.6, 4, 41)
    base = W.linear_profile(0.5, 4.0, T).astype(np.float32)
    factor = np.where(W.seeded_subset(n, 0.3, 42), 0.5, 1.0).astype(np.float32)
    with nmc.Server(0, max_active=8, slice_log2=13) as srv:
        ids = [srv.submit_ksat(lits, n, base=base, factor=factor, replicas=32, seed=s)
               for s in range(3)]
        outs = []
        for i in ids:
            deadline = time.time() + 120
            while srv.poll(i, wait_ms=200) in (0, 1) and time.time() < deadline:
                pass
            outs.append(srv.result(i)[0])
    beta = (factor[:, None] * base[None, :]).astype(np.float32)
    for s, got in enumerate(outs):
        req = dict(lits=lits, n_vars=n, beta=beta, replicas=32, seed=s)
        want = _alone("ksat", req)
        orc = _oracle("ksat", req)
        for key in KEYS:
            assert np.array_equal(got[key], want[key]), key
            assert np.array_equal(got[key], orc[key]), key


def test_admission_limits_cancel_and_errors():
    import paper_2111_13628_gb300 as nmc
    lits = W.random_ksat(400, 9.6, 4, 1)
    beta = W.beta_constant(400, 3000, 2.0)
    with nmc.Server(0, max_active=1, memory_budget=64 << 20, slice_log2=12) as srv:
        big = srv.submit_ksat(W.random_ksat(20000, 9.6, 4, 2), 20000,
                              base=np.ones(400, np.float32), factor=np.ones(20000, np.float32),
                              replicas=1024, seed=1)                     # > 64 MB budget
        a = srv.submit_ksat(lits, 400, beta=beta, replicas=32, seed=1)
        b = srv.submit_ksat(lits, 400, beta=beta, replicas=32, seed=2)   # waits for the slot
        bad = srv.submit_ksat(np.array([[1, -1, 2]], np.int32), 5, beta=W.beta_constant(5, 2, 1.0),
                              replicas=32, seed=3)
        assert srv.poll(big, wait_ms=30000) == nmc.NMC_ENOMEM
        with pytest.raises(nmc.NmcError):
            srv.result(big)
        time.sleep(0.05)
        assert srv.poll(b) == 0          # still queued behind a (one active slot)
        srv.cancel(a)
        srv.cancel(b)
        assert srv.poll(a, wait_ms=30000) == nmc.NMC_ESTATE
        assert srv.poll(b, wait_ms=30000) == nmc.NMC_ESTATE
        assert srv.poll(bad, wait_ms=60000) == nmc.NMC_EINVAL
