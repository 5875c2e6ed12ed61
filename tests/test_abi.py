"""The C-ABI library builds, loads and exports every function include/nmc.h declares (CPU).

No compute call runs here; the threshold table is host code of the library and is compared
with the oracle's own table (both built from floor(2^32 exp(-j/256)) independently).
"""
import ctypes
import os
import re
import subprocess

import numpy as np
import pytest

import oracle as O

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _declared():
    src = open(os.path.join(ROOT, "include", "nmc.h")).read()
    src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
    return sorted(set(re.findall(r"\b(nmc_[a-z_]+)\s*\(", src)))


@pytest.fixture(scope="module")
def lib():
    from paper_2111_13628_gb300 import _build
    return ctypes.CDLL(_build.build())


def test_library_exports_every_declared_symbol(lib):
    import paper_2111_13628_gb300 as nmc
    declared = _declared()
    assert declared, "no declarations parsed"
    assert sorted(nmc.SYMBOLS) == declared
    out = subprocess.run(["nm", "-D", "--defined-only", nmc.library_path()],
                         capture_output=True, text=True, check=True).stdout
    exported = set(re.findall(r"\bT (nmc_[a-z_]+)", out))
    missing = [s for s in declared if s not in exported]
    assert not missing, missing
    for s in declared:
        assert hasattr(lib, s)


def test_threshold_table_matches_oracle():
    import paper_2111_13628_gb300 as nmc
    t_lib, L_lib = nmc.threshold_table()
    t_or, L_or = O.threshold_table()
    assert L_lib == L_or
    assert np.array_equal(t_lib, t_or)


def test_create_without_device_fails_cleanly():
    import torch
    if torch.cuda.is_available():
        pytest.skip("a device is present")
    import paper_2111_13628_gb300 as nmc
    with pytest.raises(nmc.NmcError):
        nmc.Context(0)


@pytest.mark.parametrize("n,alpha,k,seed", [(2000, 9.6, 4, 1), (3000, 4.2, 3, 2), (500, 30.0, 8, 9),
                                            (300, 2.0, 5, 4)])
def test_host_colouring_matches_oracle(n, alpha, k, seed):
    """The library's sweep-order colouring (host code, no device) equals the oracle's; the last
    case needs more than 64 colours."""
    import nmc_inputs as W
    import paper_2111_13628_gb300 as nmc
    lits = W.random_ksat(n, alpha, k, seed)
    col, nc = nmc.ksat_colour_host(lits, n)
    ocol, onc = O.ksat_colour(lits, n)
    assert nc == onc and np.array_equal(col, ocol)


def test_host_colouring_crown_graph_and_rejects():
    import paper_2111_13628_gb300 as nmc
    h = 5
    lits = np.array([[2 * i + 1, 2 * j + 2] for i in range(h) for j in range(h) if i != j],
                    dtype=np.int32)
    col, nc = nmc.ksat_colour_host(lits, 2 * h)
    assert nc == 2 and np.array_equal(col, O.ksat_colour(lits, 2 * h)[0])
    with pytest.raises(nmc.NmcError):
        nmc.ksat_colour_host(np.array([[1, 1, 2]], dtype=np.int32), 3)  # repeated variable
    for rim in (10, 11):  # wheels: 3 / 4 colours, as the oracle
        lits = np.array([[1, i + 1] for i in range(1, rim + 1)] +
                        [[i + 1, i % rim + 2] for i in range(1, rim + 1)], dtype=np.int32)
        col, nc = nmc.ksat_colour_host(lits, rim + 1)
        assert nc == (3 if rim % 2 == 0 else 4)
        assert np.array_equal(col, O.ksat_colour(lits, rim + 1)[0])


@pytest.mark.parametrize("fault", ["repeat", "range", "empty", "degree"])
def test_host_build_rejects_a_late_fault_in_a_large_formula(fault):
    """Checks run over clause ranges on several threads: a fault in the last clauses of a
    20,000-clause formula is still found, and the valid formula itself is accepted."""
    import nmc_inputs as W
    import paper_2111_13628_gb300 as nmc
    n = 4000
    lits = W.random_ksat(n, 5.0, 4, 77).copy()
    assert lits.shape[0] == 20000
    nmc.ksat_colour_host(lits, n)
    if fault == "repeat":
        lits[19990, 2] = lits[19990, 0]
    elif fault == "range":
        lits[19999, 3] = n + 1
    elif fault == "empty":
        lits[19998, :] = 0
    else:  # variable 1 in 1,024 clauses (rows that do not hold it elsewhere)
        rows = np.flatnonzero(~np.any(np.abs(lits[:, 1:]) == 1, axis=1))[:1024]
        lits[rows, 0] = 1
        assert (np.abs(lits) == 1).sum() >= 1024
    with pytest.raises(nmc.NmcError):
        nmc.ksat_colour_host(lits, n)
