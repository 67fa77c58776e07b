"""CPU oracle for low(A^T A) -- TEST INFRASTRUCTURE ONLY.

Only the tests, ``__graft_entry__.smoke()`` and the CPU-baseline leg of
``bench.py`` may import this package.  The product library never does, and the
two share no code: the oracle is plain C (``ata_oracle.c``) compiled by gcc with
``-ffp-contract=off``, loaded here through ctypes.

Functions (all FP64; A is m x n row-major, C is n x n row-major):

* ``ata_lower(A)``            plain definition C_jk = sum_i a_ij a_ik, k <= j
                              (Section 3.1, Eq. "Cij").
* ``abs_ata_lower(A)``        D_jk = sum_i |a_ij||a_ik| (error-metric denominator).
* ``ata_full(A)``             full square product (symmetry check).
* ``ata_entries(A, rows, cols)`` sampled (C_jk, D_jk) pairs.
* ``dot_pairs(colj, colk)``   sampled entries from extracted column pairs.
* ``ata_recursive(A, cutoff, depth)`` the AtA recursion of Algorithm 1 with
                              textbook Strassen; returns (low C, counts).
* ``strassen_atb(A, B, depth)`` Strassen C = A^T B alone.

``oracle.fp8`` (plain numpy) is the reference of the FP8 mode: E4M3
rounding from the format definition, the exact product of the quantised
columns, and the mode's error bounds.
"""
from __future__ import annotations

import ctypes
import os

import numpy as np

from .build import build_oracle, library_path

__all__ = [
    "lib", "set_threads", "ata_lower", "abs_ata_lower", "ata_full", "ata_entries",
    "dot_pairs", "ata_recursive", "strassen_atb", "set_mutation", "COUNT_NAMES",
]

COUNT_NAMES = ("mults", "syrk_leaves", "gemm_leaves", "ata_calls",
               "strassen_levels", "block_adds")

_lib = None
_i64 = ctypes.c_int64
_dp = ctypes.POINTER(ctypes.c_double)
_lp = ctypes.POINTER(ctypes.c_int64)
_up = ctypes.POINTER(ctypes.c_uint64)


def lib():
    """Load (building first if needed) the oracle shared library."""
    global _lib
    if _lib is None:
        path = library_path()
        if not os.path.exists(path):
            build_oracle()
        L = ctypes.CDLL(path)
        L.oracle_set_threads.argtypes = [ctypes.c_int]
        L.oracle_set_threads.restype = ctypes.c_int
        L.oracle_set_mutation.argtypes = [ctypes.c_int]
        L.oracle_set_mutation.restype = None
        for name in ("oracle_ata_lower", "oracle_abs_ata_lower", "oracle_ata_full"):
            f = getattr(L, name)
            f.argtypes = [_i64, _i64, _dp, _i64, _dp, _i64]
            f.restype = None
        L.oracle_ata_entries.argtypes = [_i64, _i64, _dp, _i64, _i64, _lp, _lp, _dp, _dp]
        L.oracle_ata_entries.restype = None
        L.oracle_dot_pairs.argtypes = [_i64, _i64, _dp, _dp, _dp, _dp]
        L.oracle_dot_pairs.restype = None
        L.oracle_ata_recursive.argtypes = [_i64, _i64, _dp, _i64, _dp, _i64, _i64,
                                           ctypes.c_int, _up]
        L.oracle_ata_recursive.restype = ctypes.c_int
        L.oracle_strassen_atb.argtypes = [_i64, _i64, _i64, _dp, _i64, _dp, _i64, _dp,
                                          _i64, ctypes.c_int, _up]
        L.oracle_strassen_atb.restype = ctypes.c_int
        _lib = L
    return _lib


def _f64(a):
    a = np.ascontiguousarray(a, dtype=np.float64)
    return a, a.ctypes.data_as(_dp)


def set_threads(t: int) -> int:
    """Host threads for the definition loops (0 = all available).  Returns the
    count in use (1 if the oracle was built without OpenMP)."""
    return int(lib().oracle_set_threads(int(t)))


def set_mutation(mu: int) -> None:
    """Test-only: plant a known mistake in the recursion oracle (0 = none)."""
    lib().oracle_set_mutation(int(mu))


def ata_lower(A, out=None):
    """low(A^T A) by the plain definition; upper triangle of the result is 0
    (or left as found in ``out``)."""
    A, pa = _f64(A)
    m, n = A.shape
    C = np.zeros((n, n), np.float64) if out is None else out
    lib().oracle_ata_lower(m, n, pa, n, C.ctypes.data_as(_dp), C.shape[1])
    return C


def abs_ata_lower(A):
    A, pa = _f64(A)
    m, n = A.shape
    D = np.zeros((n, n), np.float64)
    lib().oracle_abs_ata_lower(m, n, pa, n, D.ctypes.data_as(_dp), n)
    return D


def ata_full(A):
    A, pa = _f64(A)
    m, n = A.shape
    C = np.zeros((n, n), np.float64)
    lib().oracle_ata_full(m, n, pa, n, C.ctypes.data_as(_dp), n)
    return C


def ata_entries(A, rows, cols):
    """(C_jk, D_jk) for the sampled pairs (rows[t], cols[t])."""
    A, pa = _f64(A)
    m, n = A.shape
    rows = np.ascontiguousarray(rows, dtype=np.int64)
    cols = np.ascontiguousarray(cols, dtype=np.int64)
    out = np.empty(rows.shape[0], np.float64)
    dout = np.empty(rows.shape[0], np.float64)
    lib().oracle_ata_entries(m, n, pa, n, rows.shape[0], rows.ctypes.data_as(_lp),
                             cols.ctypes.data_as(_lp), out.ctypes.data_as(_dp),
                             dout.ctypes.data_as(_dp))
    return out, dout


def dot_pairs(colj, colk):
    """colj, colk: (count, m) arrays of column pairs -> (C entries, D entries)."""
    colj, pj = _f64(colj)
    colk, pk = _f64(colk)
    count, m = colj.shape
    out = np.empty(count, np.float64)
    dout = np.empty(count, np.float64)
    lib().oracle_dot_pairs(m, count, pj, pk, out.ctypes.data_as(_dp), dout.ctypes.data_as(_dp))
    return out, dout


def ata_recursive(A, cutoff: int, depth: int, C=None):
    """Algorithm 1 (AtA) with Strassen depth ``depth`` on each A^T B call.
    Returns (C, counts) with low(C) += low(A^T A)."""
    A, pa = _f64(A)
    m, n = A.shape
    if C is None:
        C = np.zeros((n, n), np.float64)
    counts = np.zeros(6, np.uint64)
    rc = lib().oracle_ata_recursive(m, n, pa, n, C.ctypes.data_as(_dp), C.shape[1],
                                    int(cutoff), int(depth), counts.ctypes.data_as(_up))
    if rc != 0:
        raise ValueError("oracle_ata_recursive: invalid arguments")
    return C, dict(zip(COUNT_NAMES, (int(c) for c in counts)))


def strassen_atb(A, B, depth: int):
    """C = A^T B by at most ``depth`` Strassen levels; returns (C, counts)."""
    A, pa = _f64(A)
    B, pb = _f64(B)
    r, p = A.shape
    r2, q = B.shape
    assert r == r2
    C = np.zeros((p, q), np.float64)
    counts = np.zeros(6, np.uint64)
    rc = lib().oracle_strassen_atb(r, p, q, pa, p, pb, q, C.ctypes.data_as(_dp), q,
                                   int(depth), counts.ctypes.data_as(_up))
    if rc != 0:
        raise ValueError("oracle_strassen_atb: invalid arguments")
    return C, dict(zip(COUNT_NAMES, (int(c) for c in counts)))
