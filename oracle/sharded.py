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


def shard_bounds(offsets, groups: int):
    """Contiguous sequence ranges [a, b) of about equal total length (symbols),
    one per group (fewer when there are fewer sequences)."""
    off = np.asarray(offsets, dtype=np.uint64).astype(np.int64)
    m = len(off) - 1
    groups = max(1, min(int(groups), max(m, 1)))
    total = int(off[-1])
    cuts = [0]
    for g in range(1, groups):
        c = int(np.searchsorted(off, total * g // groups, side="left"))
        cuts.append(min(max(c, cuts[-1]), m))
    cuts.append(m)
    return [(cuts[i], cuts[i + 1]) for i in range(len(cuts) - 1) if cuts[i + 1] > cuts[i]] or [(0, m)]


def _slice_corpus(data, offsets, a: int, b: int, symbol_bits: int):
    """Sequences a..b-1 as their own corpus (offsets from 0; 2-bit codes repacked)."""
    off = np.asarray(offsets, dtype=np.uint64)
    s0, s1 = int(off[a]), int(off[b])
    sub_off = (off[a:b + 1] - off[a]).astype(np.uint64)
    if symbol_bits == 8:
        return np.ascontiguousarray(data[s0:s1]), sub_off
    g = np.arange(s0, s1, dtype=np.int64)
    codes = (np.asarray(data)[g >> 2] >> (6 - 2 * (g & 3)).astype(np.uint8)) & 3
    pad = (-len(codes)) % 4
    codes = np.concatenate([codes, np.zeros(pad, np.uint8)]).reshape(-1, 4)
    packed = (codes[:, 0] << 6) | (codes[:, 1] << 4) | (codes[:, 2] << 2) | codes[:, 3]
    return packed.astype(np.uint8), sub_off


def _count_group(args):
    path, a, b, j, prefixes, count_mode, symbol_bits = args
    data = np.load(os.path.join(path, "data.npy"), mmap_mode="r")
    offsets = np.load(os.path.join(path, "offsets.npy"))
    d, o = _slice_corpus(data, offsets, a, b, symbol_bits)
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
    groups = shard_bounds(offsets, workers)
    b = min(base_n, n)
    tmp = tempfile.mkdtemp(prefix="ig_oracle_")
    out = []
    try:
        np.save(os.path.join(tmp, "data.npy"), data if data.size else np.zeros(1, np.uint8))
        np.save(os.path.join(tmp, "offsets.npy"), offsets)
        ctx = mp.get_context("spawn")  # never fork a process that may hold a GPU context
        with ctx.Pool(min(workers, len(groups))) as pool:
            P = None
            for j in range(b, n + 1):
                tasks = [(tmp, a, e, j, P, count_mode, symbol_bits) for a, e in groups]
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
