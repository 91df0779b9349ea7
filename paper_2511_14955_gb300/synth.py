"""Seeded synthetic corpora shaped like the paper's workloads (inputs only).

The paper evaluates on EMBER (malware binaries), C4 (text) and 1000 Genomes
(DNA); none of those datasets is available, so these generators stand in for
them. Everything here is input generation: no n-gram is enumerated or counted.

A corpus is ``(data, offsets, symbol_bits)``:

* ``data``    - ``uint8`` array; one byte per symbol when ``symbol_bits == 8``,
  or 2-bit base codes (A,C,G,T = 0..3) packed four per byte, most significant
  bits first, when ``symbol_bits == 2``;
* ``offsets`` - ``uint64[m + 1]`` sequence boundaries in symbols,
  ``offsets[0] == 0``, non-decreasing;
* sequences are concatenated with no padding.
"""
from __future__ import annotations

import ctypes
import os
from dataclasses import dataclass, field

import numpy as np

from . import _build

MARKOV, UNIFORM, DNA = 0, 1, 2


class _Spec(ctypes.Structure):
    _fields_ = [
        ("kind", ctypes.c_uint32),
        ("markov_zipf_s", ctypes.c_double),
        ("zero_block_frac", ctypes.c_double),
        ("block", ctypes.c_uint32),
        ("n_motifs", ctypes.c_uint32),
        ("motif_len_lo", ctypes.c_uint32),
        ("motif_len_hi", ctypes.c_uint32),
        ("motif_zipf_s", ctypes.c_double),
        ("motif_rate", ctypes.c_double),
        ("dirichlet_alpha", ctypes.c_double),
        ("repeat_frac", ctypes.c_double),
        ("repeat_len_lo", ctypes.c_uint32),
        ("repeat_len_hi", ctypes.c_uint32),
        ("mutation_rate", ctypes.c_double),
    ]


_lib = None


def _load():
    global _lib
    if _lib is None:
        path = _build.build_synth()
        lib = ctypes.CDLL(str(path))
        lib.synth_model_new.restype = ctypes.c_void_p
        lib.synth_model_new.argtypes = [ctypes.POINTER(_Spec), ctypes.c_uint64]
        lib.synth_model_free.argtypes = [ctypes.c_void_p]
        lib.synth_lengths.argtypes = [ctypes.c_uint32, ctypes.c_double, ctypes.c_double,
                                      ctypes.c_uint64, ctypes.c_uint64, ctypes.c_uint64,
                                      ctypes.c_uint32, ctypes.c_void_p]
        lib.synth_fill.restype = ctypes.c_int
        lib.synth_fill.argtypes = [ctypes.c_void_p, ctypes.c_uint32, ctypes.c_void_p,
                                   ctypes.c_void_p, ctypes.c_int]
        lib.synth_philox4x32_10.argtypes = [ctypes.c_void_p, ctypes.c_void_p, ctypes.c_void_p]
        _lib = lib
    return _lib


def philox4x32_10(ctr, key):
    """Raw Philox4x32-10 block (for known-answer tests of the generator)."""
    lib = _load()
    c = np.asarray(ctr, dtype=np.uint32)
    k = np.asarray(key, dtype=np.uint32)
    out = np.zeros(4, dtype=np.uint32)
    lib.synth_philox4x32_10(c.ctypes.data, k.ctypes.data, out.ctypes.data)
    return out


@dataclass
class Model:
    kind: int = MARKOV
    markov_zipf_s: float = 1.1
    zero_block_frac: float = 0.05
    block: int = 4096
    n_motifs: int = 0
    motif_len: tuple = (16, 128)
    motif_zipf_s: float = 1.1
    motif_rate: float = 0.0
    dirichlet_alpha: float = 0.5
    repeat_frac: float = 0.0
    repeat_len: tuple = (500, 5000)
    mutation_rate: float = 0.02

    def _spec(self) -> _Spec:
        return _Spec(self.kind, self.markov_zipf_s, self.zero_block_frac, self.block,
                     self.n_motifs, self.motif_len[0], self.motif_len[1], self.motif_zipf_s,
                     self.motif_rate, self.dirichlet_alpha, self.repeat_frac,
                     self.repeat_len[0], self.repeat_len[1], self.mutation_rate)


@dataclass
class Lengths:
    dist: str = "uniform"          # "uniform" (lo..hi) or "lognormal" (median, sigma, clamp lo..hi)
    lo: int = 4096
    hi: int = 65536
    median: float = 0.0
    sigma: float = 0.0


@dataclass
class Workload:
    """A named synthetic workload: byte model, length law and run parameters."""
    name: str
    m: int
    model: Model
    lengths: Lengths
    symbol_bits: int = 8
    n: int = 4
    k: int = 1024
    candidates: int = 4096
    base_n: int = 1
    extra: dict = field(default_factory=dict)


# The five workloads: sizes, byte laws and run parameters follow the workload
# descriptions; the seeds are fixed per workload.
WORKLOADS = {
    # 64 byte sequences, lengths U[4, 64] KiB (about 2 MiB), order-1 Markov /
    # Zipf(1.1) rows, 5% zero blocks of 4 KiB; n = 4, Z = 4096, k = 1024.
    "markov_2mb": Workload(
        "markov_2mb", 64, Model(MARKOV, 1.1, 0.05, 4096),
        Lengths("uniform", 4096, 65536), 8, n=4, k=1024, candidates=4096, base_n=1),
    # 20,000 malware-like byte sequences, lognormal lengths (median 256 KiB,
    # sigma 1.0, cap 8 MiB; about 8 GB), same byte law plus 2,000 Zipf(1.1)-drawn
    # motifs of 16..128 bytes planted once per 4 KiB block; n = 8, k = 65,536,
    # Z = 262,144, base_n = 3.
    "malware_8gb": Workload(
        "malware_8gb", 20000,
        Model(MARKOV, 1.1, 0.05, 4096, n_motifs=2000, motif_len=(16, 128),
              motif_zipf_s=1.1, motif_rate=1.0),
        Lengths("lognormal", 1, 8 << 20, median=256 * 1024, sigma=1.0), 8,
        n=8, k=65536, candidates=262144, base_n=3),
    # 1,000 DNA sequences, U[1, 10] Mbp, order-3 Markov with Dirichlet(0.5)
    # rows, 1% repeat segments (500..5000 bp) with 2% point mutations, packed
    # 2 bits per base; n = 21 (also 31), k = 100,000, Z = 400,000, base_n = 12.
    "genomic_5gbp": Workload(
        "genomic_5gbp", 1000,
        Model(DNA, dirichlet_alpha=0.5, repeat_frac=0.01, repeat_len=(500, 5000),
              mutation_rate=0.02, zero_block_frac=0.0),
        Lengths("uniform", 1_000_000, 10_000_000), 2,
        n=21, k=100000, candidates=400000, base_n=12),
    # 50,000 byte sequences, lognormal lengths (median 64 KiB, sigma 1.2), a
    # uniform-random background with 10,000 substrings of 32..256 bytes drawn
    # Zipf(1.05) and planted once per 4 KiB block; n = 64, k = 262,144,
    # Z = 1,048,576, base_n = 3.
    "largen_6gb": Workload(
        "largen_6gb", 50000,
        Model(UNIFORM, zero_block_frac=0.0, block=4096, n_motifs=10000, motif_len=(32, 256),
              motif_zipf_s=1.05, motif_rate=1.0),
        Lengths("lognormal", 1, 1 << 40, median=64 * 1024, sigma=1.2), 8,
        n=64, k=262144, candidates=1048576, base_n=3),
}


def lengths_for(w: Workload, seed: int, m: int | None = None) -> np.ndarray:
    lib = _load()
    m = w.m if m is None else m
    out = np.zeros(m, dtype=np.uint64)
    L = w.lengths
    if L.dist == "uniform":
        lib.synth_lengths(0, 0.0, 0.0, L.lo, L.hi, seed, m, out.ctypes.data)
    else:
        lib.synth_lengths(1, L.median, L.sigma, L.lo, L.hi, seed, m, out.ctypes.data)
    return out


def offsets_from_lengths(lengths) -> np.ndarray:
    lengths = np.asarray(lengths, dtype=np.uint64)
    off = np.zeros(len(lengths) + 1, dtype=np.uint64)
    np.cumsum(lengths, out=off[1:])
    return off


def fill(model: Model, seed: int, offsets: np.ndarray, symbol_bits: int = 8,
         threads: int | None = None, out: np.ndarray | None = None) -> np.ndarray:
    """Generate the sequences delimited by ``offsets`` with ``model``."""
    lib = _load()
    offsets = np.ascontiguousarray(offsets, dtype=np.uint64)
    m = len(offsets) - 1
    total = int(offsets[-1])
    nbytes = total if symbol_bits == 8 else (total + 3) // 4
    if out is None:
        out = np.empty(max(nbytes, 1), dtype=np.uint8)
    assert out.dtype == np.uint8 and out.size >= nbytes and out.flags.c_contiguous
    if threads is None:
        threads = os.cpu_count() or 1
    h = lib.synth_model_new(ctypes.byref(model._spec()), seed)
    if not h:
        raise MemoryError("synth_model_new failed")
    try:
        rc = lib.synth_fill(h, m, offsets.ctypes.data, out.ctypes.data, int(threads))
    finally:
        lib.synth_model_free(h)
    if rc != 0:
        raise RuntimeError("synth_fill failed")
    return out[:nbytes] if nbytes else out[:0]


def make_corpus(name: str, seed: int = 1, m: int | None = None, threads: int | None = None,
                max_len: int | None = None, out: np.ndarray | None = None):
    """Corpus of workload ``name`` with ``m`` sequences (default: the full size).

    ``max_len`` clamps each sequence length (used to shrink a workload for
    tests while keeping its byte law). Returns ``(data, offsets, symbol_bits)``.
    """
    w = WORKLOADS[name]
    L = lengths_for(w, seed, m)
    if max_len is not None:
        L = np.minimum(L, np.uint64(max_len))
    off = offsets_from_lengths(L)
    data = fill(w.model, seed, off, w.symbol_bits, threads, out)
    return data, off, w.symbol_bits


def pack_2bit(codes) -> np.ndarray:
    """Pack base codes 0..3 four per byte, most significant bits first."""
    codes = np.asarray(codes, dtype=np.uint8)
    n = len(codes)
    pad = (-n) % 4
    c = np.concatenate([codes, np.zeros(pad, np.uint8)]).reshape(-1, 4)
    return (c[:, 0] << 6 | c[:, 1] << 4 | c[:, 2] << 2 | c[:, 3]).astype(np.uint8)


def unpack_2bit(data, total: int) -> np.ndarray:
    """Inverse of :func:`pack_2bit` for the first ``total`` bases."""
    d = np.asarray(data, dtype=np.uint8)
    out = np.stack([(d >> 6) & 3, (d >> 4) & 3, (d >> 2) & 3, d & 3], axis=1).reshape(-1)
    return out[:total].copy()
