"""Python side of the CPU oracle (test infrastructure only).

Only the tests, ``__graft_entry__.smoke()`` and the benchmark's CPU-baseline leg
may import this module.  The product library never does.

Wraps ``gd_oracle.c`` (plain C, built here with gcc into ``liboracle.so``):

* ``triad_census``     -- Algorithm 1 (3-node counts).
* ``alg2_global``      -- Algorithm 2, literal (O1), single thread.
* ``alg2_per_edge``    -- per-edge counts from the definitions of Sec. 4.2
                          (restricted counts N^(e)_{a,b,1}) and Corollaries 1-14.
* ``edges_direct``     -- the same per-edge record for a chosen list of edges.
* ``o2_global`` / ``o2_per_edge`` -- the independent method (O2), OpenMP.
* ``complete``         -- Step 4 alone on hand-fed sums.

Counts are returned as Python ints (global) or numpy uint64 arrays (per edge),
in Table 1 order [g31 g32 g33 g34 g41 ... g4_10 g4_11].
"""
from __future__ import annotations

import ctypes
import os
import subprocess
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_LIB = os.path.join(_HERE, "liboracle.so")
_SRC = os.path.join(_HERE, "gd_oracle.c")
_lib = None
_lock = threading.Lock()

GRAPHLETS = ["g31", "g32", "g33", "g34", "g41", "g42", "g43", "g44", "g45", "g46",
             "g47", "g48", "g49", "g4_10", "g4_11"]
RAW_FIELDS = ["T", "Su", "Sv", "I", "cliq", "cyc", "TSu1", "TSv1", "SuSu1", "SvSv1",
              "TI1", "SuI1", "SvI1", "II1"]
SUM_FIELDS = ["sT", "sS", "sI", "sCliq", "sCyc", "nTT", "nSuSv", "nTS", "nSS", "nTI",
              "nSI", "nII", "nII1"]
ERRORS = {1: "invalid CSR", 2: "out of memory", 3: "inexact division or underflow"}


class OracleError(RuntimeError):
    pass


def build(force: bool = False) -> str:
    """Compile the oracle (gcc, OpenMP)."""
    if (not force and os.path.exists(_LIB)
            and os.path.getmtime(_LIB) >= os.path.getmtime(_SRC)):
        return _LIB
    tmp = _LIB + f".tmp{os.getpid()}"
    subprocess.check_call(["gcc", "-O2", "-std=c11", "-fPIC", "-shared", "-fopenmp",
                           "-o", tmp, _SRC])
    os.replace(tmp, _LIB)
    return _LIB


def _load():
    global _lib
    with _lock:
        if _lib is None:
            build()
            lib = ctypes.CDLL(_LIB)
            vp, i32, i64 = ctypes.c_void_p, ctypes.c_int32, ctypes.c_int64
            for name, args in {
                "oracle_triad_census": [i32, vp, vp, vp],
                "oracle_alg2_global": [i32, vp, vp, vp, vp],
                "oracle_alg2_per_edge": [i32, vp, vp, vp, vp],
                "oracle_edges_direct": [i32, vp, vp, i64, vp, vp, vp, vp],
                "oracle_o2_per_edge": [i32, vp, vp, ctypes.c_int, vp, vp],
                "oracle_o2_global": [i32, vp, vp, ctypes.c_int, vp, vp],
                "oracle_complete": [vp, ctypes.c_uint64, vp],
            }.items():
                f = getattr(lib, name)
                f.argtypes = args
                f.restype = ctypes.c_int
            lib.oracle_max_threads.restype = ctypes.c_int
            lib.oracle_raw_width.restype = ctypes.c_int
            _lib = lib
        return _lib


def _csr(g):
    rp = np.ascontiguousarray(g.row_ptr, dtype=np.int32)
    ci = np.ascontiguousarray(g.col_idx, dtype=np.int32)
    if ci.size == 0:
        ci = np.zeros(1, dtype=np.int32)
    return g.n, rp, ci


def _check(rc):
    if rc:
        raise OracleError(ERRORS.get(rc, f"oracle error {rc}"))


def _u128(buf, k):
    return [int(buf[2 * i]) | (int(buf[2 * i + 1]) << 64) for i in range(k)]


def max_threads() -> int:
    return _load().oracle_max_threads()


def triad_census(g) -> list[int]:
    n, rp, ci = _csr(g)
    out = np.zeros(8, dtype=np.uint64)
    _check(_load().oracle_triad_census(n, rp.ctypes.data, ci.ctypes.data, out.ctypes.data))
    return _u128(out, 4)


def alg2_global(g, with_sums: bool = False):
    n, rp, ci = _csr(g)
    out = np.zeros(30, dtype=np.uint64)
    sums = np.zeros(26, dtype=np.uint64)
    _check(_load().oracle_alg2_global(n, rp.ctypes.data, ci.ctypes.data, out.ctypes.data,
                                      sums.ctypes.data))
    if with_sums:
        return _u128(out, 15), dict(zip(SUM_FIELDS, _u128(sums, 13)))
    return _u128(out, 15)


def alg2_per_edge(g, raw: bool = False):
    n, rp, ci = _csr(g)
    m = g.m
    cols = np.zeros((max(m, 1), 15), dtype=np.uint64)
    rw = np.zeros((max(m, 1), len(RAW_FIELDS)), dtype=np.uint64)
    _check(_load().oracle_alg2_per_edge(n, rp.ctypes.data, ci.ctypes.data, cols.ctypes.data,
                                        rw.ctypes.data))
    return (cols[:m], rw[:m]) if raw else cols[:m]


def edges_direct(g, edges, raw: bool = False):
    """Per-edge O1 record for the given (k, 2) edges (any orientation)."""
    n, rp, ci = _csr(g)
    e = np.ascontiguousarray(np.asarray(edges, dtype=np.int32).reshape(-1, 2))
    k = e.shape[0]
    eu = np.ascontiguousarray(e[:, 0])
    ev = np.ascontiguousarray(e[:, 1])
    cols = np.zeros((max(k, 1), 15), dtype=np.uint64)
    rw = np.zeros((max(k, 1), len(RAW_FIELDS)), dtype=np.uint64)
    _check(_load().oracle_edges_direct(n, rp.ctypes.data, ci.ctypes.data, k, eu.ctypes.data,
                                       ev.ctypes.data, cols.ctypes.data, rw.ctypes.data))
    return (cols[:k], rw[:k]) if raw else cols[:k]


def o2_per_edge(g, threads: int = 0, raw: bool = False):
    n, rp, ci = _csr(g)
    m = g.m
    cols = np.zeros((max(m, 1), 15), dtype=np.uint64)
    rw = np.zeros((max(m, 1), len(RAW_FIELDS)), dtype=np.uint64)
    _check(_load().oracle_o2_per_edge(n, rp.ctypes.data, ci.ctypes.data, threads,
                                      cols.ctypes.data, rw.ctypes.data))
    return (cols[:m], rw[:m]) if raw else cols[:m]


def o2_global(g, threads: int = 0, with_sums: bool = False):
    n, rp, ci = _csr(g)
    out = np.zeros(30, dtype=np.uint64)
    sums = np.zeros(26, dtype=np.uint64)
    _check(_load().oracle_o2_global(n, rp.ctypes.data, ci.ctypes.data, threads,
                                    out.ctypes.data, sums.ctypes.data))
    if with_sums:
        return _u128(out, 15), dict(zip(SUM_FIELDS, _u128(sums, 13)))
    return _u128(out, 15)


def complete(sums: dict, n: int) -> list[int]:
    buf = np.zeros(26, dtype=np.uint64)
    for i, k in enumerate(SUM_FIELDS):
        v = int(sums[k])
        buf[2 * i] = v & 0xFFFFFFFFFFFFFFFF
        buf[2 * i + 1] = v >> 64
    out = np.zeros(30, dtype=np.uint64)
    _check(_load().oracle_complete(buf.ctypes.data, n, out.ctypes.data))
    return _u128(out, 15)
