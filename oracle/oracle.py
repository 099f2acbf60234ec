"""ctypes wrapper around the plain C oracle (ltl_oracle.c).

TEST INFRASTRUCTURE ONLY: imported by the tests, by the smoke check and by the
benchmark's CPU-baseline leg, never by the library path.  It shares no code
with the CUDA path.

`learn` returns the minimal separating formula found by the exhaustive
enumeration of Section 3 of the paper (exact dedup), plus per-level unique
and candidate counts; `evaluate` returns the truth of a formula at every
position of every trace (the characteristic matrix of Section 4, one byte per
position).
"""
from __future__ import annotations

import ctypes
import os
import subprocess
import threading
from typing import Dict, List, Optional

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))
SRC = os.path.join(HERE, "ltl_oracle.c")
LIB = os.path.join(HERE, "libltl_oracle.so")
SRC_PAR = os.path.join(HERE, "ltl_oracle_par.c")
LIB_PAR = os.path.join(HERE, "libltl_oracle_par.so")

STATUS = {0: "found", 1: "not_found", 2: "cap", -1: "invalid", -3: "nomem", -5: "bufsize"}
OPS_ALL = 127
_lock = threading.Lock()
_lib = None
_lib_par = None


def build(force: bool = False) -> str:
    """Compile the oracle with gcc (plain -O2, no vectorisation pragmas)."""
    if force or not os.path.exists(LIB) or os.path.getmtime(LIB) < os.path.getmtime(SRC):
        tmp = LIB + ".tmp.%d" % os.getpid()
        subprocess.check_call(["gcc", "-O2", "-std=c11", "-fPIC", "-shared", "-o", tmp, SRC])
        os.replace(tmp, LIB)
    return LIB


def build_par(force: bool = False) -> str:
    """Compile the multi-core variant (ltl_oracle_par.c, which includes
    ltl_oracle.c unchanged) with gcc -fopenmp."""
    newest = max(os.path.getmtime(SRC), os.path.getmtime(SRC_PAR))
    if force or not os.path.exists(LIB_PAR) or os.path.getmtime(LIB_PAR) < newest:
        tmp = LIB_PAR + ".tmp.%d" % os.getpid()
        subprocess.check_call(["gcc", "-O2", "-std=c11", "-fPIC", "-shared", "-fopenmp", "-o", tmp, SRC_PAR])
        os.replace(tmp, LIB_PAR)
    return LIB_PAR


def _load_par():
    global _lib_par
    with _lock:
        if _lib_par is None:
            build_par()
            lib = ctypes.CDLL(LIB_PAR)
            u64p = ctypes.POINTER(ctypes.c_uint64)
            lib.oracle_learn_par.argtypes = [ctypes.c_void_p, ctypes.c_void_p, ctypes.c_uint64, ctypes.c_uint64,
                                             ctypes.c_int, ctypes.c_uint32, ctypes.c_int, ctypes.c_int,
                                             ctypes.c_uint64, ctypes.c_int, ctypes.c_uint64,
                                             ctypes.c_char_p, ctypes.c_size_t, ctypes.POINTER(ctypes.c_int),
                                             u64p, u64p, ctypes.POINTER(ctypes.c_double),
                                             ctypes.POINTER(ctypes.c_int), ctypes.POINTER(ctypes.c_int)]
            lib.oracle_learn_par.restype = ctypes.c_int
            _lib_par = lib
    return _lib_par


def _load():
    global _lib
    with _lock:
        if _lib is None:
            build()
            lib = ctypes.CDLL(LIB)
            u64p = ctypes.POINTER(ctypes.c_uint64)
            lib.oracle_eval.argtypes = [ctypes.c_char_p, ctypes.c_void_p, ctypes.c_void_p,
                                        ctypes.c_uint64, ctypes.c_int, ctypes.c_void_p]
            lib.oracle_eval.restype = ctypes.c_int
            lib.oracle_size.argtypes = [ctypes.c_char_p]
            lib.oracle_size.restype = ctypes.c_int
            lib.oracle_learn.argtypes = [ctypes.c_void_p, ctypes.c_void_p, ctypes.c_uint64,
                                         ctypes.c_uint64, ctypes.c_int, ctypes.c_uint32,
                                         ctypes.c_int, ctypes.c_int, ctypes.c_uint64,
                                         ctypes.c_char_p, ctypes.c_size_t,
                                         ctypes.POINTER(ctypes.c_int), u64p, u64p,
                                         ctypes.POINTER(ctypes.c_double),
                                         ctypes.POINTER(ctypes.c_int)]
            lib.oracle_learn.restype = ctypes.c_int
            lib.oracle_learn_ex.argtypes = [ctypes.c_void_p, ctypes.c_void_p, ctypes.c_uint64,
                                            ctypes.c_uint64, ctypes.c_int, ctypes.c_uint32,
                                            ctypes.c_int, ctypes.c_int, ctypes.c_uint64,
                                            ctypes.c_void_p, ctypes.c_int, ctypes.c_uint64,
                                            ctypes.c_char_p, ctypes.c_size_t,
                                            ctypes.POINTER(ctypes.c_int), u64p, u64p,
                                            ctypes.POINTER(ctypes.c_double),
                                            ctypes.POINTER(ctypes.c_int)]
            lib.oracle_learn_ex.restype = ctypes.c_int
            _lib = lib
    return _lib


def _concat(P, N):
    """(letters, offsets) of P followed by N; P and N are TraceSet-like."""
    lp, ln = np.asarray(P.letters, np.uint32), np.asarray(N.letters, np.uint32)
    op, on = np.asarray(P.offsets, np.uint64), np.asarray(N.offsets, np.uint64)
    letters = np.ascontiguousarray(np.concatenate([lp, ln]).astype(np.uint32))
    offsets = np.ascontiguousarray(np.concatenate([op, on[1:] + op[-1]]).astype(np.uint64))
    return letters, offsets


def size(formula: str) -> int:
    return _load().oracle_size(formula.encode())


def evaluate(formula: str, letters, offsets, n_props: int) -> np.ndarray:
    """uint8 truth value per position (same order as `letters`)."""
    letters = np.ascontiguousarray(np.asarray(letters, np.uint32))
    offsets = np.ascontiguousarray(np.asarray(offsets, np.uint64))
    n = offsets.shape[0] - 1
    out = np.zeros(max(int(offsets[-1]), 1), dtype=np.uint8)
    rc = _load().oracle_eval(formula.encode(), letters.ctypes.data, offsets.ctypes.data,
                             n, n_props, out.ctypes.data)
    if rc != 0:
        raise ValueError("oracle_eval(%r) failed: %s" % (formula, STATUS.get(rc, rc)))
    return out[: int(offsets[-1])]


def evaluate_traces(formula: str, traces, n_props: int) -> List[np.ndarray]:
    """Per-trace truth arrays for a TraceSet-like object."""
    out = evaluate(formula, traces.letters, traces.offsets, n_props)
    off = np.asarray(traces.offsets, np.uint64)
    return [out[int(off[i]):int(off[i + 1])] for i in range(off.shape[0] - 1)]


def separates(formula: str, P, N, n_props: int) -> bool:
    """eq. (dagger): true at position 0 of every positive, false on every negative."""
    letters, offsets = _concat(P, N)
    v = evaluate(formula, letters, offsets, n_props)
    nP = P.offsets.shape[0] - 1
    for t in range(offsets.shape[0] - 1):
        a, b = int(offsets[t]), int(offsets[t + 1])
        at0 = bool(v[a]) if b > a else False
        if at0 != (t < nP):
            return False
    return True


def learn(P, N, n_props: int, ops: int = OPS_ALL, max_size: int = 7, stop_mode: int = 1,
          max_entries: int = 0, costs=None, nnf: bool = False, max_errors: int = 0) -> Dict:
    """Exhaustive enumeration (Section 3) with exact dedup.

    stop_mode: 1 = stop at the first separator, 2 = finish that level,
    0 = enumerate every level up to max_size.  costs: 8 connective costs
    (atom, Not, And, Or, X, F, G, U), levels are then costs; nnf: negation on
    atoms only; max_errors: misclassified traces a separator may have.
    """
    letters, offsets = _concat(P, N)
    nP, nN = P.offsets.shape[0] - 1, N.offsets.shape[0] - 1
    K = max_size
    uniq = (ctypes.c_uint64 * (K + 1))()
    cand = (ctypes.c_uint64 * (K + 1))()
    secs = (ctypes.c_double * (K + 1))()
    fsz = ctypes.c_int(0)
    done = ctypes.c_int(0)
    buf = ctypes.create_string_buffer(1 << 16)
    carr = None
    if costs is not None:
        carr = (ctypes.c_int * 8)(*[int(x) for x in costs])
    rc = _load().oracle_learn_ex(letters.ctypes.data, offsets.ctypes.data, nP, nN, n_props, ops,
                                 K, stop_mode, max_entries, ctypes.cast(carr, ctypes.c_void_p) if carr else None,
                                 1 if nnf else 0, int(max_errors), buf, len(buf), ctypes.byref(fsz),
                                 uniq, cand, secs, ctypes.byref(done))
    if rc < 0:
        raise RuntimeError("oracle_learn failed: %s" % STATUS.get(rc, rc))
    return {
        "status": STATUS[rc],
        "formula": buf.value.decode() if rc == 0 else None,
        "size": fsz.value if rc == 0 else None,
        "unique": [int(uniq[c]) for c in range(K + 1)],
        "candidates": [int(cand[c]) for c in range(K + 1)],
        "seconds": [float(secs[c]) for c in range(K + 1)],
        "levels_done": done.value,
    }


def learn_par(P, N, n_props: int, ops: int = OPS_ALL, max_size: int = 7, stop_mode: int = 1,
              max_entries: int = 0, threads: int = 0, block_bytes: int = 0) -> Dict:
    """`learn` (uniform cost, exact separation) with each block of a level's
    candidates built on `threads` host cores (0: every core OpenMP offers) and
    admitted in enumeration order, so every result equals `learn`'s.  The
    returned dict also holds "threads", the team size used."""
    letters, offsets = _concat(P, N)
    nP, nN = P.offsets.shape[0] - 1, N.offsets.shape[0] - 1
    K = max_size
    uniq = (ctypes.c_uint64 * (K + 1))()
    cand = (ctypes.c_uint64 * (K + 1))()
    secs = (ctypes.c_double * (K + 1))()
    fsz, done, used = ctypes.c_int(0), ctypes.c_int(0), ctypes.c_int(0)
    buf = ctypes.create_string_buffer(1 << 16)
    rc = _load_par().oracle_learn_par(letters.ctypes.data, offsets.ctypes.data, nP, nN, n_props, ops, K,
                                      stop_mode, max_entries, int(threads), int(block_bytes), buf, len(buf),
                                      ctypes.byref(fsz), uniq, cand, secs, ctypes.byref(done), ctypes.byref(used))
    if rc < 0:
        raise RuntimeError("oracle_learn_par failed: %s" % STATUS.get(rc, rc))
    return {
        "status": STATUS[rc],
        "formula": buf.value.decode() if rc == 0 else None,
        "size": fsz.value if rc == 0 else None,
        "unique": [int(uniq[c]) for c in range(K + 1)],
        "candidates": [int(cand[c]) for c in range(K + 1)],
        "seconds": [float(secs[c]) for c in range(K + 1)],
        "levels_done": done.value,
        "threads": used.value,
    }
