"""GB300 engine for the inhomogeneous Metropolis sweep of Nonequilibrium Monte Carlo.

Thin ctypes binding over libnmc.so, whose C ABI is declared in include/nmc.h. Every step of
the sweep runs in the library's CUDA kernels; this module only marshals arguments. PyTorch is
used, where the caller wants it, for device buffers and streams (tensors are passed to the
library as raw device pointers). There is no CPU fallback: if the library cannot be built or
loaded, every call raises.
"""
from __future__ import annotations

import ctypes as C
import os
import threading

import numpy as np

from . import _build

NMC_OK = 0
NMC_EINVAL = -1
NMC_ENOMEM = -2
NMC_ECUDA = -3
NMC_ETIMEOUT = -4
NMC_ESTATE = -5
KIND_KSAT = 1
KIND_QAP = 2

_ERRNAMES = {NMC_EINVAL: "EINVAL", NMC_ENOMEM: "ENOMEM", NMC_ECUDA: "ECUDA",
             NMC_ETIMEOUT: "ETIMEOUT", NMC_ESTATE: "ESTATE"}


class NmcError(RuntimeError):
    def __init__(self, code, msg):
        super().__init__(f"nmc {_ERRNAMES.get(code, code)}: {msg}")
        self.code = code


class Schedule(C.Structure):
    _fields_ = [("n_steps", C.c_int32), ("beta", C.c_void_p), ("base", C.c_void_p),
                ("factor", C.c_void_p)]


class Result(C.Structure):
    _fields_ = [("states", C.c_void_p), ("energies", C.c_void_p),
                ("best_energies", C.c_void_p), ("best_states", C.c_void_p)]


_lock = threading.Lock()
_lib = None

# Exported C-ABI symbols (every function declared in include/nmc.h).
SYMBOLS = ["nmc_create", "nmc_destroy", "nmc_last_error", "nmc_sync", "nmc_load_ksat",
           "nmc_load_qap", "nmc_unload", "nmc_ksat_colouring", "nmc_ksat_colour_host",
           "nmc_set_schedule",
           "nmc_set_schedule_device", "nmc_set_schedule_factored", "nmc_replicas_create", "nmc_replicas_reset", "nmc_replicas_restore", "nmc_replicas_destroy",
           "nmc_replicas_run", "nmc_replicas_read", "nmc_replicas_read_device", "nmc_anneal",
           "nmc_threshold_table", "nmc_selftest_wait_timeout", "nmc_batch_run",
           "nmc_batch_max_vars", "nmc_server_create", "nmc_server_destroy",
           "nmc_server_submit_ksat", "nmc_server_submit_qap", "nmc_server_poll",
           "nmc_server_result", "nmc_server_cancel", "nmc_server_stats",
           "nmc_server_last_error", "nmc_batch_run_noalloc", "nmc_qap_batch_run",
           "nmc_replicas_set_ladder", "nmc_replicas_run_pt", "nmc_replicas_read_slots",
           "nmc_adaptive_ladder", "nmc_replicas_cluster_flip", "nmc_cnf_lbp",
           "nmc_cnf_backbone", "nmc_set_schedule_backbone", "nmc_replicas_whitening",
           "nmc_batch_autotune"]


def library_path() -> str:
    return _build.LIB


def load(build_if_missing: bool = True):
    """Loads libnmc.so (building it with nvcc first if it is missing or stale)."""
    global _lib
    with _lock:
        if _lib is not None:
            return _lib
        if build_if_missing and _build.stale():
            _build.build()
        if not os.path.exists(_build.LIB):
            raise RuntimeError("libnmc.so is not built; run __graft_entry__.build()")
        lib = C.CDLL(_build.LIB)
        P, i32, u64 = C.c_void_p, C.c_int32, C.c_uint64
        sig = {
            "nmc_create": ([P, C.c_int, P], C.c_int),
            "nmc_destroy": ([P], None),
            "nmc_last_error": ([P], C.c_char_p),
            "nmc_sync": ([P], C.c_int),
            "nmc_load_ksat": ([P, i32, i32, i32, P, P], C.c_int),
            "nmc_load_qap": ([P, i32, P, P, P], C.c_int),
            "nmc_unload": ([P, i32], C.c_int),
            "nmc_ksat_colouring": ([P, i32, P, P], C.c_int),
            "nmc_ksat_colour_host": ([i32, i32, i32, P, P, P], C.c_int),
            "nmc_set_schedule": ([P, i32, i32, P], C.c_int),
            "nmc_set_schedule_device": ([P, i32, i32, P], C.c_int),
            "nmc_set_schedule_factored": ([P, i32, i32, P, P], C.c_int),
            "nmc_replicas_create": ([P, i32, i32, u64, P, P], C.c_int),
            "nmc_replicas_reset": ([P, i32, u64, P], C.c_int),
            "nmc_replicas_restore": ([P, i32, P], C.c_int),
            "nmc_replicas_destroy": ([P, i32], C.c_int),
            "nmc_replicas_run": ([P, i32, i32, i32], C.c_int),
            "nmc_replicas_read": ([P, i32, P], C.c_int),
            "nmc_replicas_read_device": ([P, i32, P], C.c_int),
            "nmc_anneal": ([P, i32, i32, i32, i32, u64, P, P], C.c_int),
            "nmc_threshold_table": ([P, i32], i32),
            "nmc_selftest_wait_timeout": ([P, i32], C.c_int),
            "nmc_batch_run": ([P, i32, P, P, P], C.c_int),
            "nmc_batch_max_vars": ([P], i32),
            "nmc_batch_run_noalloc": ([P, i32, P, P, P], C.c_int),
            "nmc_qap_batch_run": ([P, i32, P, P, P], C.c_int),
            "nmc_server_create": ([C.c_int, P, P], C.c_int),
            "nmc_server_destroy": ([P], None),
            "nmc_server_submit_ksat": ([P, i32, i32, i32, P, P, i32, u64, P], C.c_int),
            "nmc_server_submit_qap": ([P, i32, P, P, P, i32, u64, P], C.c_int),
            "nmc_server_poll": ([P, C.c_int64, i32, P], C.c_int),
            "nmc_server_result": ([P, C.c_int64, P, P], C.c_int),
            "nmc_server_cancel": ([P, C.c_int64], C.c_int),
            "nmc_server_stats": ([P, P, P, P, P, P, P], C.c_int),
            "nmc_server_last_error": ([P], C.c_char_p),
            "nmc_replicas_set_ladder": ([P, i32, i32, P, P], C.c_int),
            "nmc_replicas_run_pt": ([P, i32, i32, i32, i32], C.c_int),
            "nmc_replicas_read_slots": ([P, i32, P], C.c_int),
            "nmc_adaptive_ladder": ([P, i32, i32, u64, C.c_double, C.c_double, C.c_double, i32,
                                     i32, i32, P, P, P], C.c_int),
            "nmc_replicas_cluster_flip": ([P, i32, i32, P, P, C.c_uint32, P], C.c_int),
            "nmc_cnf_lbp": ([P, i32, i32, P, P, C.c_double, i32, P, C.c_double, i32, P, P, P, P,
                             P, P], C.c_int),
            "nmc_cnf_backbone": ([P, i32, i32, P, C.c_double, C.c_double, C.c_double, P, P],
                                 C.c_int),
            "nmc_set_schedule_backbone": ([P, i32, P, i32, i32, i32, i32, C.c_float, C.c_float],
                                          C.c_int),
            "nmc_replicas_whitening": ([P, i32, i32, i32, P, P, P], C.c_int),
            "nmc_batch_autotune": ([P, i32, P, i32, i32, P], C.c_int),
        }
        for name, (args, res) in sig.items():
            fn = getattr(lib, name)
            fn.argtypes = args
            fn.restype = res
        _lib = lib
        return lib


def _ptr(a):
    if a is None:
        return None
    if hasattr(a, "data_ptr"):
        return C.c_void_p(a.data_ptr())
    return a.ctypes.data_as(C.c_void_p)


def ksat_colour_host(lits, n_vars: int):
    """(colour int32[N], n_colours): the library's sweep-order colouring, built on the host."""
    lib = load()
    lits = np.ascontiguousarray(lits, dtype=np.int32)
    col = np.zeros(int(n_vars), dtype=np.int32)
    nc = C.c_int32()
    rc = lib.nmc_ksat_colour_host(int(n_vars), lits.shape[0], lits.shape[1], _ptr(lits), _ptr(col),
                                  C.byref(nc))
    if rc != 0:
        raise NmcError(rc, "nmc_ksat_colour_host rejected the formula")
    return col, int(nc.value)


def threshold_table(cap: int = 8192):
    """(table uint32[L], L) as built by the library."""
    lib = load()
    out = np.zeros(cap, dtype=np.uint32)
    n = lib.nmc_threshold_table(_ptr(out), cap)
    return out[:n].copy(), int(n)


class Context:
    """One nmc_ctx: a device, a stream, and the instances / replica sets resident on it."""

    def __init__(self, device: int = 0, stream=None):
        self._lib = load()
        self._kinds = {}
        self._units = {}
        self._clauses = {}
        self._rs = {}
        h = C.c_void_p()
        s = None
        if stream is not None:
            s = C.c_void_p(stream if isinstance(stream, int) else stream.cuda_stream)
        rc = self._lib.nmc_create(C.byref(h), int(device), s)
        if rc != NMC_OK:
            raise NmcError(rc, "nmc_create failed")
        self._h = h

    # -- plumbing
    def _check(self, rc):
        if rc != NMC_OK:
            raise NmcError(rc, self._lib.nmc_last_error(self._h).decode())

    def close(self):
        if getattr(self, "_h", None):
            self._lib.nmc_destroy(self._h)
            self._h = None

    def __enter__(self):
        return self

    def __exit__(self, *exc):
        self.close()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def selftest_wait_timeout(self, timeout_ms: int) -> int:
        """Return code of nmc_selftest_wait_timeout (NMC_ETIMEOUT when the wait expired)."""
        return int(self._lib.nmc_selftest_wait_timeout(self._h, int(timeout_ms)))

    def sync(self):
        self._check(self._lib.nmc_sync(self._h))

    # -- instances
    def load_ksat(self, lits, n_vars: int) -> int:
        lits = np.ascontiguousarray(lits, dtype=np.int32)
        if lits.ndim != 2:
            raise ValueError("lits must be [n_clauses, k_max]")
        inst = C.c_int32()
        self._check(self._lib.nmc_load_ksat(self._h, int(n_vars), lits.shape[0], lits.shape[1],
                                            _ptr(lits), C.byref(inst)))
        self._kinds[inst.value] = KIND_KSAT
        self._units[inst.value] = int(n_vars)
        self._clauses[inst.value] = lits.shape[0]
        return inst.value

    def load_qap(self, F, D) -> int:
        F = np.ascontiguousarray(F, dtype=np.int32)
        D = np.ascontiguousarray(D, dtype=np.int32)
        if F.ndim != 2 or F.shape[0] != F.shape[1] or D.shape != F.shape:
            raise ValueError("F and D must be n x n")
        inst = C.c_int32()
        self._check(self._lib.nmc_load_qap(self._h, F.shape[0], _ptr(F), _ptr(D), C.byref(inst)))
        self._kinds[inst.value] = KIND_QAP
        self._units[inst.value] = F.shape[0]
        return inst.value

    def unload(self, inst: int):
        self._check(self._lib.nmc_unload(self._h, int(inst)))

    def ksat_colouring(self, inst: int):
        n = self._units[inst]
        col = np.zeros(n, dtype=np.int32)
        nc = C.c_int32()
        self._check(self._lib.nmc_ksat_colouring(self._h, int(inst), _ptr(col), C.byref(nc)))
        return col, nc.value

    def set_schedule(self, inst: int, beta):
        """beta: [n_units, n_steps] float32, numpy (host) or a CUDA torch tensor (device)."""
        if hasattr(beta, "is_cuda") and beta.is_cuda:
            if beta.dtype.__str__() != "torch.float32" or not beta.is_contiguous():
                raise ValueError("device beta must be a contiguous float32 tensor")
            self._check(self._lib.nmc_set_schedule_device(self._h, int(inst), beta.shape[1],
                                                          _ptr(beta)))
            return
        if hasattr(beta, "numpy"):
            beta = beta.numpy()
        beta = np.ascontiguousarray(beta, dtype=np.float32)
        if beta.ndim != 2 or beta.shape[0] != self._units[inst]:
            raise ValueError("beta must be [n_units, n_steps]")
        self._check(self._lib.nmc_set_schedule(self._h, int(inst), beta.shape[1], _ptr(beta)))

    def set_schedule_factored(self, inst: int, base, factor):
        """beta[u][t] = float32(base[t] * factor[u])."""
        base = np.ascontiguousarray(base, dtype=np.float32)
        factor = np.ascontiguousarray(factor, dtype=np.float32)
        if factor.shape[0] != self._units[inst]:
            raise ValueError("factor must have one entry per unit")
        self._check(self._lib.nmc_set_schedule_factored(self._h, int(inst), base.shape[0],
                                                        _ptr(base), _ptr(factor)))

    # -- replica sets
    def replicas_create(self, inst: int, replicas: int, seed: int, init=None) -> int:
        if init is not None:
            dt = np.uint8 if self._kinds[inst] == KIND_KSAT else np.int16
            init = np.ascontiguousarray(init, dtype=dt)
            if init.shape != (replicas, self._units[inst]):
                raise ValueError("init must be [replicas, n_units]")
        rs = C.c_int32()
        self._check(self._lib.nmc_replicas_create(self._h, int(inst), int(replicas),
                                                  int(seed) & (2**64 - 1), _ptr(init),
                                                  C.byref(rs)))
        self._rs[rs.value] = (inst, int(replicas))
        return rs.value

    def batch_run(self, rs, t0, t1):
        """Runs sweeps t0[i]..t1[i]-1 of k-SAT replica sets rs[i] in one batched launch."""
        rs = np.ascontiguousarray(rs, dtype=np.int32)
        t0 = np.ascontiguousarray(np.broadcast_to(t0, rs.shape), dtype=np.int32)
        t1 = np.ascontiguousarray(np.broadcast_to(t1, rs.shape), dtype=np.int32)
        self._check(self._lib.nmc_batch_run(self._h, rs.size, _ptr(rs), _ptr(t0), _ptr(t1)))

    def batch_run_noalloc(self, rs, t0, t1):
        """nmc_batch_run_noalloc: the batched sweep with its work list in the library's fixed
        device array (no device allocation during the call)."""
        rs = np.ascontiguousarray(rs, dtype=np.int32)
        t0 = np.ascontiguousarray(np.broadcast_to(t0, rs.shape), dtype=np.int32)
        t1 = np.ascontiguousarray(np.broadcast_to(t1, rs.shape), dtype=np.int32)
        self._check(self._lib.nmc_batch_run_noalloc(self._h, rs.size, _ptr(rs), _ptr(t0),
                                                    _ptr(t1)))

    def qap_batch_run(self, rs, t0, t1):
        """Runs steps t0[i]..t1[i]-1 of QAP replica sets rs[i] in one batched launch."""
        rs = np.ascontiguousarray(rs, dtype=np.int32)
        t0 = np.ascontiguousarray(np.broadcast_to(t0, rs.shape), dtype=np.int32)
        t1 = np.ascontiguousarray(np.broadcast_to(t1, rs.shape), dtype=np.int32)
        self._check(self._lib.nmc_qap_batch_run(self._h, rs.size, _ptr(rs), _ptr(t0), _ptr(t1)))

    def batch_autotune(self, rs, t0: int, sweeps: int):
        """Times every batched-sweep shape on these sets and keeps the fastest for this context.
        Returns int32 [2, 3]: (CTAs per item, lanes per variable, us per sweep) per width."""
        rs = np.ascontiguousarray(np.atleast_1d(rs), dtype=np.int32)
        out = np.zeros((2, 3), np.int32)
        self._check(self._lib.nmc_batch_autotune(self._h, rs.size, _ptr(rs), int(t0), int(sweeps),
                                                 _ptr(out)))
        return out

    def batch_max_vars(self) -> int:
        return int(self._lib.nmc_batch_max_vars(self._h))

    def replicas_reset(self, rs: int, seed: int, init=None):
        inst, R = self._rs[rs]
        if init is not None:
            dt = np.uint8 if self._kinds[inst] == KIND_KSAT else np.int16
            init = np.ascontiguousarray(init, dtype=dt)
            if init.shape != (R, self._units[inst]):
                raise ValueError("init must be [replicas, n_units]")
        self._check(self._lib.nmc_replicas_reset(self._h, int(rs), int(seed) & (2**64 - 1),
                                                 _ptr(init)))

    def replicas_restore(self, rs: int, checkpoint: dict):
        """Restores states and best states saved by replicas_read (checkpoint resume)."""
        inst, R = self._rs[rs]
        dt = np.uint8 if self._kinds[inst] == KIND_KSAT else np.int16
        st = np.ascontiguousarray(checkpoint["states"], dtype=dt)
        bs = np.ascontiguousarray(checkpoint["best_states"], dtype=dt)
        if st.shape != (R, self._units[inst]) or bs.shape != st.shape:
            raise ValueError("checkpoint arrays must be [replicas, n_units]")
        res = Result(_ptr(st), None, None, _ptr(bs))
        self._check(self._lib.nmc_replicas_restore(self._h, int(rs), C.byref(res)))

    def replicas_destroy(self, rs: int):
        self._check(self._lib.nmc_replicas_destroy(self._h, int(rs)))
        self._rs.pop(rs, None)

    def replicas_run(self, rs: int, t0: int, t1: int):
        self._check(self._lib.nmc_replicas_run(self._h, int(rs), int(t0), int(t1)))

    # -- replica exchange
    def set_ladder(self, rs: int, ladder, slots=None):
        """Attaches a temperature ladder (n_temps floats) to a k-SAT replica set of R = G *
        n_temps replicas; slots: [R] int32 slot of every replica in its ladder (None: identity)."""
        ladder = np.ascontiguousarray(ladder, dtype=np.float32)
        _, R = self._rs[rs]
        if slots is not None:
            slots = np.ascontiguousarray(slots, dtype=np.int32)
            if slots.shape != (R,):
                raise ValueError("slots must have one entry per replica")
        self._check(self._lib.nmc_replicas_set_ladder(self._h, int(rs), ladder.shape[0],
                                                      _ptr(ladder), _ptr(slots)))

    def run_pt(self, rs: int, t0: int, t1: int, sweeps_per_round: int):
        """Sweeps t0..t1-1 with an exchange round after every sweeps_per_round sweeps."""
        self._check(self._lib.nmc_replicas_run_pt(self._h, int(rs), int(t0), int(t1),
                                                  int(sweeps_per_round)))

    def read_slots(self, rs: int):
        _, R = self._rs[rs]
        out = np.zeros(R, dtype=np.int32)
        self._check(self._lib.nmc_replicas_read_slots(self._h, int(rs), _ptr(out)))
        return out

    def cluster_flip(self, rs: int, mask, beta, move_id: int, accepted: bool = False):
        """Collective move: replica r proposes flipping the variables of mask[r] (mask [1 or R,
        n_vars] 0/1) and accepts at beta[r] (scalar or R floats). With accepted=True, returns
        the uint8[R] acceptance flags (synchronises)."""
        inst, R = self._rs[rs]
        n = self._units[inst]
        mask = np.ascontiguousarray(mask, dtype=np.uint8).reshape(-1, n)
        beta = np.ascontiguousarray(np.broadcast_to(np.asarray(beta, dtype=np.float32), (R,)))
        out = np.zeros(R, dtype=np.uint8) if accepted else None
        self._check(self._lib.nmc_replicas_cluster_flip(self._h, int(rs), mask.shape[0], _ptr(mask),
                                                        _ptr(beta), int(move_id) & 0xFFFFFFFF,
                                                        _ptr(out)))
        return out

    # -- learning stage (k-SAT)
    def cnf_lbp(self, inst: int, x_star, beta: float, lambdas, tol: float, max_iter: int,
                eps=None) -> dict:
        """LBP around seeds x_star ([S, N] or [N] 0/1). Returns dict(marg [S,N], corr [S,M],
        iters [S,L], deltas [S,L], n_done [S], p [S], q1 [S]) (one seed: the rows alone)."""
        n = self._units[inst]
        x = np.ascontiguousarray(x_star, dtype=np.uint8)
        one = x.ndim == 1
        x = x.reshape(-1, n)
        S = x.shape[0]
        lam = np.ascontiguousarray(np.atleast_1d(lambdas), dtype=np.float64)
        eps = None if eps is None else np.ascontiguousarray(eps, dtype=np.float64)
        m = self._clauses[inst]
        out = dict(marg=np.zeros((S, n)), corr=np.zeros((S, m)),
                   iters=np.zeros((S, lam.size), np.int32), deltas=np.zeros((S, lam.size)),
                   n_done=np.zeros(S, np.int32))
        ov = np.zeros((S, 2))
        self._check(self._lib.nmc_cnf_lbp(self._h, int(inst), S, _ptr(x), _ptr(eps), float(beta),
                                          lam.size, _ptr(lam), float(tol), int(max_iter),
                                          _ptr(out["marg"]), _ptr(out["corr"]),
                                          _ptr(out["iters"]), _ptr(out["deltas"]),
                                          _ptr(out["n_done"]), _ptr(ov)))
        out["p"], out["q1"] = ov[:, 0].copy(), ov[:, 1].copy()
        if one:
            out = {k: v[0] for k, v in out.items()}
        return out

    def cnf_backbone(self, inst: int, corr, beta: float, seed_thr: float, cutoff: float):
        """(labels int32 [S, N] or [N], n_clusters) from clause correlations [S, M] or [M]."""
        n, m = self._units[inst], self._clauses[inst]
        c = np.ascontiguousarray(corr, dtype=np.float64)
        one = c.ndim == 1
        c = c.reshape(-1, m)
        S = c.shape[0]
        lab = np.zeros((S, n), np.int32)
        nc = np.zeros(S, np.int32)
        self._check(self._lib.nmc_cnf_backbone(self._h, int(inst), S, _ptr(c), float(beta),
                                               float(seed_thr), float(cutoff), _ptr(lab),
                                               _ptr(nc)))
        return (lab[0], int(nc[0])) if one else (lab, nc)

    def set_schedule_backbone(self, inst: int, labels, cycles: int, t_hot: int, t_cold: int,
                              t_unlearn: int, base: float, heat: float):
        lab = np.ascontiguousarray(labels, dtype=np.int32)
        if lab.shape != (self._units[inst],):
            raise ValueError("labels must have one entry per variable")
        self._check(self._lib.nmc_set_schedule_backbone(self._h, int(inst), _ptr(lab), int(cycles),
                                                        int(t_hot), int(t_cold), int(t_unlearn),
                                                        float(base), float(heat)))

    def whitening(self, rs: int, use_best: bool = False, generalized: bool = True,
                  masks: bool = False):
        """Frozen-variable counts (int32 [R]) of the whitening procedure; with masks=True also
        the frozen flags (uint8 [R, N]) and the number of parallel rounds."""
        inst, R = self._rs[rs]
        cnt = np.zeros(R, np.int32)
        fr = np.zeros((R, self._units[inst]), np.uint8) if masks else None
        rounds = C.c_int32()
        self._check(self._lib.nmc_replicas_whitening(self._h, int(rs), int(bool(use_best)),
                                                     int(bool(generalized)), _ptr(cnt), _ptr(fr),
                                                     C.byref(rounds)))
        return (cnt, fr, rounds.value) if masks else cnt

    def adaptive_ladder(self, inst: int, replicas: int, seed: int, beta0: float, alpha: float,
                        sigma_min: float, max_temps: int, sweeps_eq: int, sweeps_meas: int):
        """(betas float64[L], sigmas float64[L]) of the adaptive ladder."""
        betas = np.zeros(max_temps, dtype=np.float64)
        sigmas = np.zeros(max_temps, dtype=np.float64)
        nt = C.c_int32()
        self._check(self._lib.nmc_adaptive_ladder(self._h, int(inst), int(replicas),
                                                  int(seed) & (2**64 - 1), float(beta0),
                                                  float(alpha), float(sigma_min), int(max_temps),
                                                  int(sweeps_eq), int(sweeps_meas), _ptr(betas),
                                                  _ptr(sigmas), C.byref(nt)))
        return betas[:nt.value].copy(), sigmas[:nt.value].copy()

    def _alloc_out(self, inst, R, host=True):
        n = self._units[inst]
        dt = np.uint8 if self._kinds[inst] == KIND_KSAT else np.int16
        return dict(states=np.zeros((R, n), dtype=dt), energies=np.zeros(R, dtype=np.int64),
                    best_energies=np.zeros(R, dtype=np.int64),
                    best_states=np.zeros((R, n), dtype=dt))

    def replicas_read(self, rs: int) -> dict:
        inst, R = self._rs[rs]
        out = self._alloc_out(inst, R)
        res = Result(_ptr(out["states"]), _ptr(out["energies"]), _ptr(out["best_energies"]),
                     _ptr(out["best_states"]))
        self._check(self._lib.nmc_replicas_read(self._h, int(rs), C.byref(res)))
        return out

    def replicas_read_device(self, rs: int, states=None, energies=None, best_energies=None,
                             best_states=None):
        """Writes into caller-owned CUDA tensors (any may be None), asynchronously."""
        res = Result(_ptr(states), _ptr(energies), _ptr(best_energies), _ptr(best_states))
        self._check(self._lib.nmc_replicas_read_device(self._h, int(rs), C.byref(res)))

    def anneal(self, inst: int, replicas: int, t0: int, t1: int, seed: int, init=None,
               out=None) -> dict:
        """One-shot anneal through host buffers (nmc_anneal)."""
        if init is not None:
            dt = np.uint8 if self._kinds[inst] == KIND_KSAT else np.int16
            init = np.ascontiguousarray(init, dtype=dt)
        if out is None:
            out = self._alloc_out(inst, replicas)
        res = Result(_ptr(out.get("states")), _ptr(out.get("energies")),
                     _ptr(out.get("best_energies")), _ptr(out.get("best_states")))
        self._check(self._lib.nmc_anneal(self._h, int(inst), int(replicas), int(t0), int(t1),
                                         int(seed) & (2**64 - 1), _ptr(init), C.byref(res)))
        return out


class ServerConfig(C.Structure):
    _fields_ = [("max_active", C.c_int32), ("memory_budget", C.c_int64), ("slice_log2", C.c_int32)]


class Server:
    """Continuous-batching anneal server (nmc_server_*); thread-safe."""

    def __init__(self, device: int = 0, max_active: int = 256, memory_budget: int = 64 << 30,
                 slice_log2: int = 22):
        self._lib = load()
        cfg = ServerConfig(int(max_active), int(memory_budget), int(slice_log2))
        h = C.c_void_p()
        rc = self._lib.nmc_server_create(int(device), C.byref(cfg), C.byref(h))
        if rc != NMC_OK:
            raise NmcError(rc, "nmc_server_create failed")
        self._h = h
        self._meta = {}

    def close(self):
        if getattr(self, "_h", None):
            self._lib.nmc_server_destroy(self._h)
            self._h = None

    def __enter__(self):
        return self

    def __exit__(self, *exc):
        self.close()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def _id(self, rc, req, meta):
        if rc != NMC_OK:
            raise NmcError(rc, "submit rejected")
        self._meta[req.value] = meta
        return req.value

    @staticmethod
    def _sched(beta=None, base=None, factor=None):
        keep = []
        if beta is not None:
            beta = np.ascontiguousarray(beta, dtype=np.float32)
            keep.append(beta)
            return Schedule(beta.shape[1], _ptr(beta), None, None), keep
        base = np.ascontiguousarray(base, dtype=np.float32)
        factor = np.ascontiguousarray(factor, dtype=np.float32)
        keep += [base, factor]
        return Schedule(base.shape[0], None, _ptr(base), _ptr(factor)), keep

    def submit_ksat(self, lits, n_vars, beta=None, replicas=32, seed=0, base=None,
                    factor=None) -> int:
        """Queues a k-SAT anneal; schedule as beta [n, T] or as base [T] x factor [n]."""
        lits = np.ascontiguousarray(lits, dtype=np.int32)
        sc, keep = self._sched(beta, base, factor)
        req = C.c_int64()
        rc = self._lib.nmc_server_submit_ksat(self._h, int(n_vars), lits.shape[0], lits.shape[1],
                                              _ptr(lits), C.byref(sc), int(replicas),
                                              int(seed) & (2**64 - 1), C.byref(req))
        del keep
        return self._id(rc, req, (KIND_KSAT, int(n_vars), int(replicas)))

    def submit_qap(self, F, D, beta=None, replicas=256, seed=0, base=None, factor=None) -> int:
        F = np.ascontiguousarray(F, dtype=np.int32)
        D = np.ascontiguousarray(D, dtype=np.int32)
        sc, keep = self._sched(beta, base, factor)
        req = C.c_int64()
        rc = self._lib.nmc_server_submit_qap(self._h, F.shape[0], _ptr(F), _ptr(D), C.byref(sc),
                                             int(replicas), int(seed) & (2**64 - 1), C.byref(req))
        del keep
        return self._id(rc, req, (KIND_QAP, F.shape[0], int(replicas)))

    def poll(self, req: int, wait_ms: int = 0) -> int:
        st = C.c_int32()
        rc = self._lib.nmc_server_poll(self._h, C.c_int64(req), int(wait_ms), C.byref(st))
        if rc != NMC_OK:
            raise NmcError(rc, "poll failed")
        return st.value

    def result(self, req: int):
        """(dict of arrays, latency seconds); raises NmcError if the request failed."""
        kind, n, R = self._meta[req]
        dt = np.uint8 if kind == KIND_KSAT else np.int16
        out = dict(states=np.zeros((R, n), dtype=dt), energies=np.zeros(R, dtype=np.int64),
                   best_energies=np.zeros(R, dtype=np.int64), best_states=np.zeros((R, n), dtype=dt))
        res = Result(_ptr(out["states"]), _ptr(out["energies"]), _ptr(out["best_energies"]),
                     _ptr(out["best_states"]))
        lat = C.c_double()
        rc = self._lib.nmc_server_result(self._h, C.c_int64(req), C.byref(res), C.byref(lat))
        if rc != NMC_OK:
            raise NmcError(rc, self._lib.nmc_server_last_error(self._h).decode())
        self._meta.pop(req, None)
        return out, lat.value

    def cancel(self, req: int):
        rc = self._lib.nmc_server_cancel(self._h, C.c_int64(req))
        if rc != NMC_OK:
            raise NmcError(rc, "cancel failed")

    def stats(self) -> dict:
        t, a, q, act, mem = C.c_int64(), C.c_int64(), C.c_int32(), C.c_int32(), C.c_int64()
        busy = C.c_double()
        self._lib.nmc_server_stats(self._h, C.byref(t), C.byref(a), C.byref(busy), C.byref(q),
                                   C.byref(act), C.byref(mem))
        return dict(ticks=t.value, attempts=a.value, busy_s=busy.value, queued=q.value,
                    active=act.value, mem_in_use=mem.value)
