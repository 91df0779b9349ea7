"""The CPU oracle of Algorithm 3 on several cores - TEST INFRASTRUCTURE ONLY.

Only the tests, ``__graft_entry__.smoke()`` and the CPU-baseline leg of
``bench.py`` may import this module; the product path never does.

Sequences are independent under Eq. 1 and Eq. 2 (Sec. 2): a sequence's
windows never cross into another sequence, and under Eq. 2 each sequence
adds one per distinct n-gram it contains. So the counts of one step of
Algorithm 3 (Sec. 7) over a corpus split into groups of whole sequences are
exactly the sums of the groups' counts. This module runs the oracle's
counting step (``oracle.count_pass``, plain C) on each group in its own
process, adds the counts up (numpy), and does the selection between passes
itself: ``P^(j)`` = the top-Z j-grams by (count desc, symbols asc), the
reading the oracle takes at every selection. Everything else is the
single-threaded oracle's arithmetic; ``tests/test_oracle.py`` pins this
harness against ``oracle.intergrams`` row for row.
"""
from __future__ import annotations

import multiprocessing as mp
import os
import shutil
import tempfile

import numpy as np

from oracle import oracle as _oracle


def shard_groups(offsets, groups: int):
    """Sequence indices split into at most `groups` groups of about equal
    total length: longest sequence first, each to the group with the fewest
    symbols so far (greedy by bytes). Every sequence is in exactly one group,
    in ascending order within it."""
    L = np.diff(np.asarray(offsets, dtype=np.uint64).astype(np.int64))
    m = len(L)
    groups = max(1, min(int(groups), max(m, 1)))
    load = np.zeros(groups, np.int64)
    members = [[] for _ in range(groups)]
    for i in np.argsort(-L, kind="stable"):
        g = int(np.argmin(load))
        members[g].append(int(i))
        load[g] += L[i]
    out = [np.array(sorted(g), np.int64) for g in members if g]
    return out or [np.zeros(0, np.int64)]


def _gather_corpus(data, offsets, idx, symbol_bits: int):
    """Sequences `idx` as a corpus of their own (offsets from 0; 2-bit codes
    repacked from the group's first base)."""
    off = np.asarray(offsets, dtype=np.uint64).astype(np.int64)
    L = off[idx + 1] - off[idx]
    sub_off = np.zeros(len(idx) + 1, np.uint64)
    sub_off[1:] = np.cumsum(L)
    if symbol_bits == 8:
        parts = [np.asarray(data[off[i]:off[i + 1]]) for i in idx]
        return (np.concatenate(parts) if parts else np.zeros(0, np.uint8)), sub_off
    g = np.concatenate([np.arange(off[i], off[i + 1], dtype=np.int64) for i in idx]) if len(idx) else \
        np.zeros(0, np.int64)
    codes = (np.asarray(data)[g >> 2] >> (6 - 2 * (g & 3)).astype(np.uint8)) & 3
    pad = (-len(codes)) % 4
    codes = np.concatenate([codes, np.zeros(pad, np.uint8)]).reshape(-1, 4)
    packed = (codes[:, 0] << 6) | (codes[:, 1] << 4) | (codes[:, 2] << 2) | codes[:, 3]
    return packed.astype(np.uint8), sub_off


def _count_group(args):
    path, g, j, prefixes, count_mode, symbol_bits = args
    data = np.load(os.path.join(path, "data.npy"), mmap_mode="r")
    offsets = np.load(os.path.join(path, "offsets.npy"))
    idx = np.load(os.path.join(path, f"group{g}.npy"))
    d, o = _gather_corpus(data, offsets, idx, symbol_bits)
    return _oracle.count_pass(d, o, j, prefixes, count_mode=count_mode, symbol_bits=symbol_bits)


def _as_sortable(keys):
    """Rows of symbol codes as values whose order is the rows' order."""
    r, j = keys.shape
    if j <= 8:
        v = np.zeros(r, np.uint64)
        for t in range(j):
            v = (v << np.uint64(8)) | keys[:, t].astype(np.uint64)
        return v
    return np.ascontiguousarray(keys).view(np.dtype((np.void, j))).reshape(r)


def merge_counts(parts):
    """Sum the counts of equal rows over the groups' (keys, counts); rows
    come out in ascending symbol order."""
    parts = [p for p in parts if len(p[1])]
    if not parts:
        j = 1
        return np.zeros((0, j), np.uint8), np.zeros(0, np.uint64)
    keys = np.concatenate([p[0] for p in parts])
    counts = np.concatenate([p[1] for p in parts])
    sk = _as_sortable(keys)
    order = np.argsort(sk, kind="stable")
    sk, keys, counts = sk[order], keys[order], counts[order]
    start = np.ones(len(sk), bool)
    start[1:] = sk[1:] != sk[:-1]
    idx = np.flatnonzero(start)
    return keys[idx], np.add.reduceat(counts, idx).astype(np.uint64)


def top_rows(keys, counts, t: int):
    """Indices of the top-t rows by (count desc, symbols asc); `keys` are in
    ascending symbol order, so a stable sort on the counts alone keeps ties
    in symbol order."""
    order = np.argsort(-counts.astype(np.int64), kind="stable")
    return order[:t]


def intergrams(data, offsets, n: int, k: int, candidates: int, base_n: int = 3, count_mode: int = 0,
               symbol_bits: int = 8, workers: int | None = None, per_pass: bool = False):
    """Algorithm 3 (as ``oracle.intergrams``) over groups of sequences in
    ``workers`` processes (default: every core). Returns the final top-k
    (keys (r, n) uint8 codes, counts uint64) or, with ``per_pass``, a list of
    (j, keys, counts) with the top-k after every pass j."""
    workers = workers or os.cpu_count() or 1
    data = np.ascontiguousarray(np.asarray(data, dtype=np.uint8))
    offsets = np.ascontiguousarray(np.asarray(offsets, dtype=np.uint64))
    groups = shard_groups(offsets, workers)
    b = min(base_n, n)
    tmp = tempfile.mkdtemp(prefix="ig_oracle_")
    out = []
    try:
        np.save(os.path.join(tmp, "data.npy"), data if data.size else np.zeros(1, np.uint8))
        np.save(os.path.join(tmp, "offsets.npy"), offsets)
        for g, idx in enumerate(groups):
            np.save(os.path.join(tmp, f"group{g}.npy"), idx)
        ctx = mp.get_context("spawn")  # never fork a process that may hold a GPU context
        with ctx.Pool(min(workers, len(groups))) as pool:
            P = None
            for j in range(b, n + 1):
                tasks = [(tmp, g, j, P, count_mode, symbol_bits) for g in range(len(groups))]
                keys, counts = merge_counts(pool.map(_count_group, tasks))
                if keys.shape[1] != j:
                    keys = np.zeros((0, j), np.uint8)
                top = top_rows(keys, counts, k)
                if per_pass or j == n:
                    out.append((j, keys[top].copy(), counts[top].copy()))
                if j < n:
                    sel = np.sort(top_rows(keys, counts, candidates))  # ascending symbols
                    P = np.ascontiguousarray(keys[sel]) if len(sel) else np.zeros((0, j), np.uint8)
    finally:
        shutil.rmtree(tmp, ignore_errors=True)
    if per_pass:
        return out
    return out[-1][1], out[-1][2]
