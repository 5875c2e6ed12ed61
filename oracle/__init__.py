"""CPU oracle for the NMC inhomogeneous Metropolis sweep (ctypes wrapper over nmc_oracle.c).

TEST INFRASTRUCTURE ONLY: imported by the tests, by the smoke check and by the bench's
CPU-baseline / reference leg. The product path (the CUDA library and its binding) never
imports this package, and this package never imports the product.

The definitions it implements are stated at the top of nmc_oracle.c. Most functions here are
thin argument marshallers over the C files. Four hold arithmetic of their own, in plain Python
and numpy: `adaptive_ladder` and `qap_adaptive_ladder` (each level's sigma from the C anneal's
energy sums, and the next beta = beta + alpha / sigma), `clause_degrees` (the default eps_i of the
surrogate Hamiltonian) and `backbone_schedule` (the two-chain schedule as an array).

Parity status: every function is pinned by tests/test_oracle_pins.py (brute-force
enumeration, recomputation, closed forms, a chi-square against the exact Boltzmann law and an
independent Philox implementation); none is "parity unpinned".
"""
from __future__ import annotations

import ctypes as C
import math
import os
import subprocess
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "nmc_oracle.c")
_SRCS = [_SRC, os.path.join(_HERE, "lbp_oracle.c")]
_LIB = os.path.join(_HERE, "libnmc_oracle.so")
_lock = threading.Lock()
_lib = None


def build(force: bool = False) -> str:
    """Compiles the oracle's C files with gcc (plain -O2, no fast-math) into libnmc_oracle.so."""
    newest = max(os.path.getmtime(f) for f in _SRCS)
    if force or not os.path.exists(_LIB) or os.path.getmtime(_LIB) < newest:
        tmp = _LIB + f".tmp{os.getpid()}"
        subprocess.check_call(["gcc", "-O2", "-std=c11", "-fPIC", "-shared", "-o", tmp, *_SRCS,
                               "-lm", "-lpthread"])
        os.replace(tmp, _LIB)
    return _LIB


def _load():
    global _lib
    with _lock:
        if _lib is None:
            build()
            lib = C.CDLL(_LIB)
            P = C.c_void_p
            i32, i64, u32, u64 = C.c_int32, C.c_int64, C.c_uint32, C.c_uint64
            lib.orc_philox4x32_10.argtypes = [P, P, P]
            lib.orc_threshold_table.argtypes = [P, C.c_int]
            lib.orc_threshold_table.restype = C.c_int
            lib.orc_quantize_beta.argtypes = [C.c_float]
            lib.orc_quantize_beta.restype = u32
            lib.orc_uphill_threshold.argtypes = [u32, i64]
            lib.orc_uphill_threshold.restype = u32
            lib.orc_ksat_energy.argtypes = [i32, i32, i32, P, P]
            lib.orc_ksat_energy.restype = i64
            lib.orc_ksat_energies.argtypes = [i32, i32, i32, P, i64, P, P]
            lib.orc_ksat_energies.restype = None
            lib.orc_ksat_delta.argtypes = [i32, i32, i32, P, P, i32]
            lib.orc_ksat_delta.restype = i64
            lib.orc_ksat_colour.argtypes = [i32, i32, i32, P, P]
            lib.orc_ksat_colour.restype = i32
            lib.orc_ksat_anneal.argtypes = [i32, i32, i32, P, i32, P, i32, P, i32, i32, u64, P, P,
                                            P, i32, P, P, P, P, i32, P, P]
            lib.orc_ksat_anneal.restype = C.c_int
            lib.orc_ksat_pt_anneal.argtypes = [i32, i32, i32, P, i32, P, i32, i32, P, P, i32, i32,
                                               i32, u64, P, P, P, P, P, P, P]
            lib.orc_ksat_pt_anneal.restype = C.c_int
            lib.orc_ksat_cluster_flip.argtypes = [i32, i32, i32, P, i32, P, P, P, P, i32, P, P,
                                                  u32, u64, P, P]
            lib.orc_ksat_cluster_flip.restype = C.c_int
            dbl = C.c_double
            lib.orc_cnf_lbp.argtypes = [i32, i32, i32, P, P, P, dbl, i32, P, dbl, i32, P, P, P, P,
                                        P, P, P]
            lib.orc_cnf_lbp.restype = C.c_int
            lib.orc_cnf_backbone.argtypes = [i32, i32, i32, P, P, dbl, dbl, dbl, P]
            lib.orc_cnf_backbone.restype = i32
            lib.orc_ksat_whitening.argtypes = [i32, i32, i32, P, P, i32, P]
            lib.orc_ksat_whitening.restype = i32
            lib.orc_qap_pt_anneal.argtypes = [i32, P, P, i32, P, i32, i32, P, P, i32, i32, i32, u64,
                                              P, P, P, P, P, P, P]
            lib.orc_qap_pt_anneal.restype = C.c_int
            lib.orc_qap_cost.argtypes = [i32, P, P, P]
            lib.orc_qap_cost.restype = i64
            lib.orc_qap_swap_delta.argtypes = [i32, P, P, P, i32, i32]
            lib.orc_qap_swap_delta.restype = i64
            lib.orc_qap_anneal.argtypes = [i32, P, P, i32, P, i32, P, i32, i32, u64, P, P, P,
                                           i32, P, P, P, P, i32, P, P]
            lib.orc_qap_anneal.restype = C.c_int
            _lib = lib
    return _lib


def _p(a):
    return None if a is None else a.ctypes.data_as(C.c_void_p)


def _c(a, dtype):
    return None if a is None else np.ascontiguousarray(a, dtype=dtype)


TAG_KSAT_INIT = 0x4B494E49
TAG_KSAT_SWEEP = 0x4B535750
TAG_QAP_INIT = 0x51494E49
TAG_QAP_STEP = 0x51535450
TAG_PT_SWAP = 0x50545357
TAG_CLUSTER = 0x434C5354


def philox4x32_10(ctr, key) -> np.ndarray:
    """One Philox4x32-10 block: ctr 4 x uint32, key 2 x uint32 -> 4 x uint32."""
    lib = _load()
    c = np.ascontiguousarray(ctr, dtype=np.uint32)
    k = np.ascontiguousarray(key, dtype=np.uint32)
    out = np.zeros(4, dtype=np.uint32)
    lib.orc_philox4x32_10(_p(c), _p(k), _p(out))
    return out


def threshold_table(cap: int = 8192):
    """(table uint32[L], L): Tab[j] = min(2^32-1, floor(2^32 exp(-j/256))), L = first zero."""
    lib = _load()
    t = np.zeros(cap, dtype=np.uint32)
    n = lib.orc_threshold_table(_p(t), cap)
    if n < 0:
        raise RuntimeError("threshold table capacity too small")
    return t[:n].copy(), n


def quantize_beta(beta: float) -> int:
    return int(_load().orc_quantize_beta(float(beta)))


def uphill_threshold(bq: int, dE: int) -> int:
    return int(_load().orc_uphill_threshold(int(bq), int(dE)))


def _cnf(lits):
    lits = np.ascontiguousarray(lits, dtype=np.int32)
    if lits.ndim != 2:
        raise ValueError("lits must be [M, kmax]")
    return lits, lits.shape[0], lits.shape[1]


def ksat_energy(lits, n_vars: int, x) -> int:
    lits, m, k = _cnf(lits)
    x = _c(x, np.uint8)
    return int(_load().orc_ksat_energy(n_vars, m, k, _p(lits), _p(x)))


def ksat_energies(lits, n_vars: int, X) -> np.ndarray:
    """int64[S]: the energy of every row of X (S x N, 0/1)."""
    lits, m, k = _cnf(lits)
    X = _c(X, np.uint8).reshape(-1, n_vars)
    e = np.zeros(X.shape[0], dtype=np.int64)
    _load().orc_ksat_energies(n_vars, m, k, _p(lits), X.shape[0], _p(X), _p(e))
    return e


def ksat_delta(lits, n_vars: int, x, v: int) -> int:
    lits, m, k = _cnf(lits)
    x = _c(x, np.uint8)
    return int(_load().orc_ksat_delta(n_vars, m, k, _p(lits), _p(x), int(v)))


def ksat_colour(lits, n_vars: int):
    """(colour int32[N], n_colours) of the DSatur colouring (the sweep order)."""
    lits, m, k = _cnf(lits)
    col = np.zeros(n_vars, dtype=np.int32)
    nc = _load().orc_ksat_colour(n_vars, m, k, _p(lits), _p(col))
    return col, int(nc)


def ksat_anneal(lits, n_vars, beta, t0, t1, seed, replicas=None, replica_ids=None, init=None,
                init_best=None, init_best_energy=None, n_threads=None, stats_from=None):
    """Runs sweeps t0..t1-1. Returns dict(states uint8[R,N], energies int64[R],
    best_energies int64[R], best_states uint8[R,N]); with stats_from, also e_sum / e_sq int64[R]:
    sums of the end-of-sweep energy and its square over sweeps t >= stats_from.

    replica_ids selects which replica indices (Philox streams) to run; default 0..replicas-1.
    """
    lits, m, k = _cnf(lits)
    beta = np.ascontiguousarray(beta, dtype=np.float32)
    if beta.ndim != 2 or beta.shape[0] != n_vars:
        raise ValueError("beta must be [N, n_steps]")
    ids = None if replica_ids is None else np.ascontiguousarray(replica_ids, dtype=np.int32)
    nr = len(ids) if ids is not None else int(replicas)
    init = _c(init, np.uint8)
    init_best = _c(init_best, np.uint8)
    init_best_energy = _c(init_best_energy, np.int64)
    if n_threads is None:
        n_threads = min(nr, os.cpu_count() or 1)
    out_s = np.zeros((nr, n_vars), dtype=np.uint8)
    out_b = np.zeros((nr, n_vars), dtype=np.uint8)
    e = np.zeros(nr, dtype=np.int64)
    be = np.zeros(nr, dtype=np.int64)
    s1 = s2 = None
    if stats_from is not None:
        s1 = np.zeros(nr, dtype=np.int64)
        s2 = np.zeros(nr, dtype=np.int64)
    rc = _load().orc_ksat_anneal(n_vars, m, k, _p(lits), beta.shape[1], _p(beta), nr, _p(ids),
                                 int(t0), int(t1), int(seed) & (2**64 - 1), _p(init),
                                 _p(init_best), _p(init_best_energy), int(n_threads), _p(out_s),
                                 _p(e), _p(be), _p(out_b),
                                 int(stats_from) if stats_from is not None else 0, _p(s1), _p(s2))
    if rc != 0:
        raise ValueError("orc_ksat_anneal rejected its arguments")
    out = dict(states=out_s, energies=e, best_energies=be, best_states=out_b)
    if stats_from is not None:
        out.update(e_sum=s1, e_sq=s2)
    return out


def ksat_pt_anneal(lits, n_vars, beta, ladder, t0, t1, sweeps_per_round, seed, replicas=None,
                   slots=None, init=None, init_best=None, init_best_energy=None):
    """Replica exchange: R = replicas (default len(ladder)) = G ladders of L = len(ladder)
    slots; replica g*L + i sits at slot slots[r] (default i) of ladder g, with temperature
    multiplier ladder[slot]; exchange rounds after every sweeps_per_round sweeps.
    Returns dict(states, energies, best_energies, best_states, slots)."""
    lits, m, k = _cnf(lits)
    beta = np.ascontiguousarray(beta, dtype=np.float32)
    ladder = np.ascontiguousarray(ladder, dtype=np.float32)
    L = ladder.shape[0]
    R = L if replicas is None else int(replicas)
    slots = (np.arange(R, dtype=np.int32) % L if slots is None
             else np.array(slots, dtype=np.int32))
    init = _c(init, np.uint8)
    init_best = _c(init_best, np.uint8)
    init_best_energy = _c(init_best_energy, np.int64)
    out_s = np.zeros((R, n_vars), dtype=np.uint8)
    out_b = np.zeros((R, n_vars), dtype=np.uint8)
    e = np.zeros(R, dtype=np.int64)
    be = np.zeros(R, dtype=np.int64)
    rc = _load().orc_ksat_pt_anneal(n_vars, m, k, _p(lits), beta.shape[1], _p(beta), R, L,
                                    _p(ladder), _p(slots), int(t0), int(t1), int(sweeps_per_round),
                                    int(seed) & (2**64 - 1), _p(init), _p(init_best),
                                    _p(init_best_energy), _p(out_s), _p(e), _p(be), _p(out_b))
    if rc != 0:
        raise ValueError("orc_ksat_pt_anneal rejected its arguments")
    return dict(states=out_s, energies=e, best_energies=be, best_states=out_b, slots=slots)


def ksat_cluster_flip(lits, n_vars, chain, mask, beta, move_id, seed, replica_ids=None):
    """Collective move of every replica of `chain` (a dict as ksat_anneal returns: states,
    energies, best_states, best_energies): replica r proposes x xor mask_r (mask [1 or R, N] 0/1)
    and accepts by the Metropolis rule at beta[r]. A per-replica mask has one row per row of
    `chain` (row r goes with states row r, like beta[r]). replica_ids: the id (Philox stream) of
    each row, default 0..R-1. Returns a new dict of the same form plus `accepted` uint8[R]."""
    lits, m, k = _cnf(lits)
    st = np.array(chain["states"], dtype=np.uint8, order="C")
    bs = np.array(chain["best_states"], dtype=np.uint8, order="C")
    e = np.array(chain["energies"], dtype=np.int64)
    be = np.array(chain["best_energies"], dtype=np.int64)
    R = st.shape[0]
    mask = np.ascontiguousarray(mask, dtype=np.uint8).reshape(-1, n_vars)
    beta = np.ascontiguousarray(np.broadcast_to(np.asarray(beta, dtype=np.float32), (R,)))
    acc = np.zeros(R, dtype=np.uint8)
    ids = None if replica_ids is None else np.ascontiguousarray(replica_ids, dtype=np.int32)
    rc = _load().orc_ksat_cluster_flip(n_vars, m, k, _p(lits), R, _p(st), _p(e), _p(bs), _p(be),
                                       mask.shape[0], _p(mask), _p(beta), int(move_id) & 0xFFFFFFFF,
                                       int(seed) & (2**64 - 1), _p(acc), _p(ids))
    if rc != 0:
        raise ValueError("orc_ksat_cluster_flip rejected its arguments")
    return dict(states=st, energies=e, best_energies=be, best_states=bs, accepted=acc)


def adaptive_ladder(lits, n_vars, replicas, seed, beta0, alpha, sigma_min, max_temps,
                    sweeps_eq, sweeps_meas):
    """Adaptive inverse-temperature ladder (App. "Adaptive Parallel Tempering").

    Level i runs the replicas (Philox initial states under `seed` at level 0, then each level
    continuing from the previous one) over sweeps [i T, (i+1) T), T = sweeps_eq + sweeps_meas, at
    the homogeneous beta_i (float32, every variable); sigma_i^2 = <E^2> - <E>^2 over the
    end-of-sweep energies of the last sweeps_meas sweeps of all replicas. Stops when
    sigma_i <= sigma_min or after max_temps levels; else beta_{i+1} = beta_i + alpha / sigma_i.
    Returns (betas, sigmas) as float64 arrays.
    """
    T = int(sweeps_eq) + int(sweeps_meas)
    betas, sigmas = [], []
    beta = float(beta0)
    state = dict(init=None, init_best=None, init_best_energy=None)
    for i in range(int(max_temps)):
        t0, t1 = i * T, (i + 1) * T
        sched = np.full((n_vars, t1), np.float32(beta), dtype=np.float32)
        res = ksat_anneal(lits, n_vars, sched, t0, t1, seed, replicas=replicas,
                          stats_from=t0 + int(sweeps_eq), **state)
        state = dict(init=res["states"], init_best=res["best_states"],
                     init_best_energy=res["best_energies"])
        samples = float(int(replicas) * int(sweeps_meas))
        mean = float(int(res["e_sum"].sum())) / samples
        var = float(int(res["e_sq"].sum())) / samples - mean * mean
        sigma = math.sqrt(max(var, 0.0))
        betas.append(beta)
        sigmas.append(sigma)
        if sigma <= sigma_min:
            break
        beta = beta + alpha / sigma
    return np.array(betas, dtype=np.float64), np.array(sigmas, dtype=np.float64)


def ksat_whitening(lits, n_vars, x, generalized=True):
    """(frozen uint8[N], count) of the whitening procedure on assignment x (0/1)."""
    lits, m, k = _cnf(lits)
    x = np.ascontiguousarray(x, dtype=np.uint8)
    fr = np.zeros(n_vars, dtype=np.uint8)
    c = _load().orc_ksat_whitening(n_vars, m, k, _p(lits), _p(x), int(bool(generalized)), _p(fr))
    return fr, int(c)


def clause_degrees(lits, n_vars):
    """eps_i of the surrogate Hamiltonian for a CNF formula: the number of clauses containing
    variable i (the largest energy change a flip of i can cause)."""
    lits = np.asarray(lits)
    v = np.abs(lits[lits != 0]) - 1
    return np.bincount(v, minlength=n_vars).astype(np.float64)


def cnf_lbp(lits, n_vars, x_star, beta, lambdas, tol, max_iter, eps=None):
    """Loopy BP on the surrogate Hamiltonian of a CNF formula around the seed x_star (0/1),
    with lambda continuation over `lambdas`. Returns dict(marg float64[N], corr float64[M],
    iters int32[L], deltas float64[L], n_done, p, q1, lam)."""
    lits, m, k = _cnf(lits)
    x = np.ascontiguousarray(x_star, dtype=np.uint8)
    eps = clause_degrees(lits, n_vars) if eps is None else np.ascontiguousarray(eps, np.float64)
    lam = np.ascontiguousarray(np.atleast_1d(lambdas), dtype=np.float64)
    marg = np.zeros(n_vars)
    corr = np.zeros(m)
    iters = np.zeros(lam.size, dtype=np.int32)
    deltas = np.zeros(lam.size)
    nd = C.c_int32()
    ov = np.zeros(2)
    lo = C.c_double()
    rc = _load().orc_cnf_lbp(n_vars, m, k, _p(lits), _p(x), _p(eps), float(beta), lam.size,
                             _p(lam), float(tol), int(max_iter), _p(marg), _p(corr), _p(iters),
                             _p(deltas), C.byref(nd), _p(ov), C.byref(lo))
    if rc != 0:
        raise ValueError("orc_cnf_lbp rejected its arguments")
    return dict(marg=marg, corr=corr, iters=iters, deltas=deltas, n_done=nd.value, p=ov[0],
                q1=ov[1], lam=lo.value)


def cnf_backbone(lits, n_vars, corr, beta, seed_thr, cutoff):
    """Backbone labels (int32[N], -1 outside every cluster) and the number of clusters."""
    lits, m, k = _cnf(lits)
    corr = np.ascontiguousarray(corr, dtype=np.float64)
    lab = np.zeros(n_vars, dtype=np.int32)
    nc = _load().orc_cnf_backbone(n_vars, m, k, _p(lits), _p(corr), float(beta), float(seed_thr),
                                  float(cutoff), _p(lab))
    return lab, int(nc)


def backbone_schedule(labels, base, heat, cycles, t_hot, t_cold, t_unlearn):
    """The sampling stage's schedule (Algorithm 1) as beta[N][T] float32: every cycle runs
    t_hot sweeps with the backbone at base/heat and the rest held (+inf), t_cold sweeps with the
    backbone held and the rest at base, then t_unlearn homogeneous sweeps at base."""
    labels = np.asarray(labels)
    bb = labels >= 0
    hot = np.float32(base) / np.float32(heat)
    cyc = []
    for _ in range(int(cycles)):
        a = np.where(bb[:, None], hot, np.float32(np.inf)) * np.ones((1, t_hot), np.float32)
        b = np.where(bb[:, None], np.float32(np.inf), np.float32(base)) * np.ones((1, t_cold), np.float32)
        c = np.full((labels.size, t_unlearn), np.float32(base), np.float32)
        cyc += [a.astype(np.float32), b.astype(np.float32), c]
    return np.concatenate(cyc, axis=1) if cyc else np.zeros((labels.size, 0), np.float32)


def qap_cost(F, D, p) -> int:
    F = _c(F, np.int32)
    D = _c(D, np.int32)
    p = _c(p, np.int16)
    return int(_load().orc_qap_cost(F.shape[0], _p(F), _p(D), _p(p)))


def qap_swap_delta(F, D, p, r, s) -> int:
    F = _c(F, np.int32)
    D = _c(D, np.int32)
    p = _c(p, np.int16)
    return int(_load().orc_qap_swap_delta(F.shape[0], _p(F), _p(D), _p(p), int(r), int(s)))


def qap_anneal(F, D, beta, t0, t1, seed, replicas=None, replica_ids=None, init=None,
               init_best=None, init_best_energy=None, n_threads=None, stats_from=None):
    """Runs QAP steps t0..t1-1 (n swap attempts each). Returns dict(perms int16[R,n],
    energies, best_energies, best_perms); with stats_from also e_sum / e_sq float64[R]: the
    end-of-step costs (and squares) of steps t >= stats_from, added in step order."""
    F = _c(F, np.int32)
    D = _c(D, np.int32)
    n = F.shape[0]
    beta = np.ascontiguousarray(beta, dtype=np.float32)
    if beta.ndim != 2 or beta.shape[0] != n:
        raise ValueError("beta must be [n, n_steps]")
    ids = None if replica_ids is None else np.ascontiguousarray(replica_ids, dtype=np.int32)
    nr = len(ids) if ids is not None else int(replicas)
    init = _c(init, np.int16)
    init_best = _c(init_best, np.int16)
    init_best_energy = _c(init_best_energy, np.int64)
    if n_threads is None:
        n_threads = min(nr, os.cpu_count() or 1)
    out_p = np.zeros((nr, n), dtype=np.int16)
    out_b = np.zeros((nr, n), dtype=np.int16)
    e = np.zeros(nr, dtype=np.int64)
    be = np.zeros(nr, dtype=np.int64)
    s1 = s2 = None
    if stats_from is not None:
        s1 = np.zeros(nr, dtype=np.float64)
        s2 = np.zeros(nr, dtype=np.float64)
    rc = _load().orc_qap_anneal(n, _p(F), _p(D), beta.shape[1], _p(beta), nr, _p(ids), int(t0),
                                int(t1), int(seed) & (2**64 - 1), _p(init), _p(init_best),
                                _p(init_best_energy), int(n_threads), _p(out_p), _p(e), _p(be),
                                _p(out_b), int(stats_from) if stats_from is not None else 0,
                                _p(s1), _p(s2))
    if rc != 0:
        raise ValueError("orc_qap_anneal rejected its arguments")
    out = dict(perms=out_p, energies=e, best_energies=be, best_perms=out_b)
    if stats_from is not None:
        out.update(e_sum=s1, e_sq=s2)
    return out


def qap_pt_anneal(F, D, beta, ladder, t0, t1, sweeps_per_round, seed, replicas=None, slots=None,
                  init=None, init_best=None, init_best_energy=None):
    """Replica exchange for the QAP swap chain (see ksat_pt_anneal). Returns dict(perms,
    energies, best_energies, best_perms, slots)."""
    F = _c(F, np.int32)
    D = _c(D, np.int32)
    n = F.shape[0]
    beta = np.ascontiguousarray(beta, dtype=np.float32)
    ladder = np.ascontiguousarray(ladder, dtype=np.float32)
    L = ladder.shape[0]
    R = L if replicas is None else int(replicas)
    slots = (np.arange(R, dtype=np.int32) % L if slots is None
             else np.array(slots, dtype=np.int32))
    init = _c(init, np.int16)
    init_best = _c(init_best, np.int16)
    init_best_energy = _c(init_best_energy, np.int64)
    out_p = np.zeros((R, n), dtype=np.int16)
    out_b = np.zeros((R, n), dtype=np.int16)
    e = np.zeros(R, dtype=np.int64)
    be = np.zeros(R, dtype=np.int64)
    rc = _load().orc_qap_pt_anneal(n, _p(F), _p(D), beta.shape[1], _p(beta), R, L, _p(ladder),
                                   _p(slots), int(t0), int(t1), int(sweeps_per_round),
                                   int(seed) & (2**64 - 1), _p(init), _p(init_best),
                                   _p(init_best_energy), _p(out_p), _p(e), _p(be), _p(out_b))
    if rc != 0:
        raise ValueError("orc_qap_pt_anneal rejected its arguments")
    return dict(perms=out_p, energies=e, best_energies=be, best_perms=out_b, slots=slots)


def qap_adaptive_ladder(F, D, replicas, seed, beta0, alpha, sigma_min, max_temps, steps_eq,
                        steps_meas):
    """The adaptive ladder of adaptive_ladder() for the QAP swap chain: level i runs steps
    [i T, (i+1) T) at the homogeneous beta_i (every facility; float32, then Q16); the per-replica
    double sums of the last steps_meas costs (and squares) are added over the replicas in replica
    order, then sigma_i^2 = <E^2> - <E>^2 and beta_{i+1} = beta_i + alpha / sigma_i."""
    F = _c(F, np.int32)
    n = F.shape[0]
    T = int(steps_eq) + int(steps_meas)
    betas, sigmas = [], []
    beta = float(beta0)
    state = dict(init=None, init_best=None, init_best_energy=None)
    for i in range(int(max_temps)):
        t0, t1 = i * T, (i + 1) * T
        sched = np.full((n, t1), np.float32(beta), dtype=np.float32)
        res = qap_anneal(F, D, sched, t0, t1, seed, replicas=replicas,
                         stats_from=t0 + int(steps_eq), **state)
        state = dict(init=res["perms"], init_best=res["best_perms"],
                     init_best_energy=res["best_energies"])
        s1 = 0.0
        s2 = 0.0
        for r in range(int(replicas)):
            s1 += float(res["e_sum"][r])
            s2 += float(res["e_sq"][r])
        samples = float(int(replicas) * int(steps_meas))
        mean = s1 / samples
        var = s2 / samples - mean * mean
        sigma = math.sqrt(max(var, 0.0))
        betas.append(beta)
        sigmas.append(sigma)
        if sigma <= sigma_min:
            break
        beta = beta + alpha / sigma
    return np.array(betas, dtype=np.float64), np.array(sigmas, dtype=np.float64)
