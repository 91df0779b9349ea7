"""CPU oracle for top-k n-gram counting - TEST INFRASTRUCTURE ONLY.

Only the tests, ``__graft_entry__.smoke()`` and the CPU-baseline leg of
``bench.py`` may import this module. It wraps ``intergrams_oracle.c`` (plain
C, single-threaded, built here with gcc) and shares no code with the CUDA
library.

Functions follow the paper directly:

* :func:`exhaustive` - Eq. 1 / Eq. 2 (Sec. 2) counted by the naive method of
  Sec. 3: every n-gram is counted, sorted by count, the top k kept.
* :func:`intergrams` - Algorithm 3 (Sec. 7), with Algorithm 2 (Sec. 6) as
  its first pass generalised to a base length ``base_n``.
* :func:`count_pass` - one counting step of Algorithm 3 on its own (used by
  ``oracle/sharded.py`` to run the oracle over groups of whole sequences on
  several cores).

Output keys are returned as an ``(r, n)`` uint8 array of symbol codes (one
code per symbol; for 2-bit data the codes are 0..3) and the counts as a
``uint64[r]`` array, in rank order: count descending, then symbols ascending.
"""
from __future__ import annotations

import ctypes
import subprocess
from pathlib import Path

import numpy as np

HERE = Path(__file__).resolve().parent
SRC = HERE / "intergrams_oracle.c"
LIB = HERE / "_lib" / "liboracle.so"

EQ2_ONCE_PER_SEQUENCE = 0
EQ1_EVERY_OCCURRENCE = 1

_lib = None


def build(force: bool = False) -> Path:
    """Compile the oracle with gcc (no optimisation tricks, -O2)."""
    LIB.parent.mkdir(exist_ok=True)
    if force or not LIB.exists() or SRC.stat().st_mtime > LIB.stat().st_mtime:
        tmp = LIB.with_suffix(".so.tmp")
        r = subprocess.run(["gcc", "-O2", "-std=c11", "-Wall", "-shared", "-fPIC", "-o", str(tmp), str(SRC)],
                           stdout=subprocess.PIPE, stderr=subprocess.STDOUT, text=True)
        if r.returncode != 0:
            raise RuntimeError("oracle build failed:\n" + r.stdout)
        tmp.replace(LIB)
    return LIB


def _load():
    global _lib
    if _lib is None:
        lib = ctypes.CDLL(str(build()))
        P, U32, U64 = ctypes.c_void_p, ctypes.c_uint32, ctypes.c_uint64
        lib.oracle_exhaustive.restype = ctypes.c_int
        lib.oracle_exhaustive.argtypes = [P, P, U32, U32, U32, U32, U64, P, P, P]
        lib.oracle_intergrams.restype = ctypes.c_int
        lib.oracle_intergrams.argtypes = [P, P, U32, U32, U32, U32, U64, U32, U64, U32, P, P, P, P]
        lib.oracle_count_keys.restype = ctypes.c_int
        lib.oracle_count_keys.argtypes = [P, P, U32, U32, U32, U32, P, U64, P]
        lib.oracle_count_pass.restype = ctypes.c_int
        lib.oracle_count_pass.argtypes = [P, P, U32, U32, U32, U32, P, U64, U32, P, P, U64, P]
        lib.oracle_features.restype = ctypes.c_int
        lib.oracle_features.argtypes = [P, P, U32, U32, U32, P, U32, P, P, U64, P]
        _lib = lib
    return _lib


def _prep(data, offsets):
    data = np.ascontiguousarray(np.asarray(data, dtype=np.uint8))
    if data.size == 0:
        data = np.zeros(1, np.uint8)
    offsets = np.ascontiguousarray(np.asarray(offsets, dtype=np.uint64))
    return data, offsets, len(offsets) - 1


def exhaustive(data, offsets, n: int, k: int, count_mode: int = EQ2_ONCE_PER_SEQUENCE,
               symbol_bits: int = 8):
    """Exact top-k n-grams of the corpus (Eq. 2 by default, Eq. 1 if count_mode=1)."""
    lib = _load()
    data, offsets, m = _prep(data, offsets)
    keys = np.zeros((max(k, 1), max(n, 1)), np.uint8)
    counts = np.zeros(max(k, 1), np.uint64)
    kout = ctypes.c_uint64(0)
    rc = lib.oracle_exhaustive(data.ctypes.data, offsets.ctypes.data, m, symbol_bits, n,
                               count_mode, k, keys.ctypes.data, counts.ctypes.data, ctypes.byref(kout))
    if rc != 0:
        raise ValueError(f"oracle_exhaustive failed: {rc}")
    r = kout.value
    return keys[:r].copy(), counts[:r].copy()


def intergrams(data, offsets, n: int, k: int, candidates: int, base_n: int = 3,
               count_mode: int = EQ2_ONCE_PER_SEQUENCE, symbol_bits: int = 8,
               stop_j: int = 0, want_survivors: bool = False):
    """Top-k of Algorithm 3 after pass ``stop_j`` (default: after pass n).

    With ``want_survivors`` the number of windows counted in that pass (their
    (j-1)-prefix was a candidate; all windows for the first pass) is returned
    as a third value.
    """
    lib = _load()
    data, offsets, m = _prep(data, offsets)
    j = stop_j if stop_j else n
    keys = np.zeros((max(k, 1), max(j, 1)), np.uint8)
    counts = np.zeros(max(k, 1), np.uint64)
    kout = ctypes.c_uint64(0)
    surv = ctypes.c_uint64(0)
    rc = lib.oracle_intergrams(data.ctypes.data, offsets.ctypes.data, m, symbol_bits, n, base_n,
                               candidates, count_mode, k, stop_j, keys.ctypes.data,
                               counts.ctypes.data, ctypes.byref(kout),
                               ctypes.byref(surv) if want_survivors else None)
    if rc != 0:
        raise ValueError(f"oracle_intergrams failed: {rc}")
    r = kout.value
    if want_survivors:
        return keys[:r].copy(), counts[:r].copy(), surv.value
    return keys[:r].copy(), counts[:r].copy()


def count_pass(data, offsets, j: int, prefixes=None, count_mode: int = EQ2_ONCE_PER_SEQUENCE,
               symbol_bits: int = 8):
    """One counting step of Algorithm 3: every distinct j-gram whose
    (j-1)-prefix is a row of ``prefixes`` (an (r, j-1) uint8 array of symbol
    codes in ascending order; None = every j-gram, the dense pass) with its
    Eq. 2 (or Eq. 1) count. Returns (keys (d, j) uint8 ascending, counts
    uint64[d])."""
    lib = _load()
    data, offsets, m = _prep(data, offsets)
    use = prefixes is not None
    pre = np.ascontiguousarray(np.asarray(prefixes if use else np.zeros((1, 1)), dtype=np.uint8))
    npre = pre.shape[0] if use else 0
    if use and npre == 0:
        pre = np.zeros((1, max(j - 1, 1)), np.uint8)
    cap = 1 << 16
    while True:
        keys = np.zeros((cap, j), np.uint8)
        counts = np.zeros(cap, np.uint64)
        nout = ctypes.c_uint64(0)
        rc = lib.oracle_count_pass(data.ctypes.data, offsets.ctypes.data, m, symbol_bits, j, count_mode,
                                   pre.ctypes.data, npre, 1 if use else 0, keys.ctypes.data, counts.ctypes.data,
                                   cap, ctypes.byref(nout))
        d = nout.value
        if rc == 0:
            return keys[:d].copy(), counts[:d].copy()
        if d <= cap:
            raise ValueError(f"oracle_count_pass failed: {rc}")
        cap = int(d)


def count_keys(data, offsets, keys, count_mode: int = EQ2_ONCE_PER_SEQUENCE, symbol_bits: int = 8):
    """Exact Eq. 2 (or Eq. 1) counts of the given n-grams (rows of symbol codes)."""
    lib = _load()
    data, offsets, m = _prep(data, offsets)
    keys = np.ascontiguousarray(np.asarray(keys, dtype=np.uint8))
    nk, n = keys.shape
    out = np.zeros(max(nk, 1), np.uint64)
    rc = lib.oracle_count_keys(data.ctypes.data, offsets.ctypes.data, m, symbol_bits, n, count_mode,
                               keys.ctypes.data, nk, out.ctypes.data)
    if rc != 0:
        raise ValueError(f"oracle_count_keys failed: {rc}")
    return out[:nk].copy()


def features(data, offsets, keys, symbol_bits: int = 8):
    """Boolean sequence x feature matrix (Sec. 1, Fig. 1) for the n-grams in
    `keys` (rows of symbol codes, distinct): CSR (row_ptr uint64[m + 1],
    cols uint32 ascending within each row)."""
    lib = _load()
    data, offsets, m = _prep(data, offsets)
    keys = np.ascontiguousarray(np.asarray(keys, dtype=np.uint8))
    nk, n = keys.shape
    row_ptr = np.zeros(m + 1, np.uint64)
    nnz = ctypes.c_uint64(0)
    cap = 1 << 16
    while True:
        cols = np.zeros(cap, np.uint32)
        rc = lib.oracle_features(data.ctypes.data, offsets.ctypes.data, m, symbol_bits, n, keys.ctypes.data, nk,
                                 row_ptr.ctypes.data, cols.ctypes.data, cap, ctypes.byref(nnz))
        if rc == 0:
            return row_ptr, cols[: nnz.value].copy()
        if nnz.value <= cap:
            raise ValueError(f"oracle_features failed: {rc}")
        cap = int(nnz.value)
