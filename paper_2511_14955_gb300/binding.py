"""Thin ctypes binding of ``libintergrams.so`` (argument marshalling only).

Every step of the computation runs in the library's sm_103a kernels; this
module only converts arguments. PyTorch supplies device memory and streams.
If the library is missing the import of :class:`Plan` fails loudly - there is
no CPU fallback.
"""
from __future__ import annotations

import ctypes
from pathlib import Path

import numpy as np

from . import _build

IG_OK, IG_DONE = 0, 1
STATUS_NAMES = {0: "IG_OK", 1: "IG_DONE", -1: "IG_EINVAL", -2: "IG_ENOMEM", -3: "IG_ETABLE_FULL",
                -4: "IG_EOVERFLOW", -5: "IG_ETIMEOUT", -6: "IG_ECUDA", -7: "IG_ESTATE"}
COUNT_ONCE_PER_SEQUENCE = 0
COUNT_EVERY_OCCURRENCE = 1
F_HOST_INPUT = 1 << 0
F_GRAPH = 1 << 1
F_AUTOTUNE = 1 << 2
F_TIMING = 1 << 3
F_SHARDED = 1 << 7
SRV_FIFO = 1 << 0
SRV_OLDEST_FIRST = 1 << 1
SRV_LARGE_ALONE = 1 << 2
F_EXHAUSTIVE_CHECKS = 1 << 8

# every symbol include/intergrams.h declares
EXPORTS = ["intergrams_plan", "intergrams_pass", "intergrams_run", "intergrams_rewind", "intergrams_topk",
           "intergrams_stats", "intergrams_timings", "intergrams_free", "intergrams_last_error",
           "intergrams_dense_topk_static", "intergrams_plan_device_bytes", "intergrams_server_create",
           "intergrams_server_submit", "intergrams_server_wait", "intergrams_server_stats",
           "intergrams_server_destroy", "intergrams_autotune", "intergrams_features",
           "intergrams_test_fail_alloc", "intergrams_test_stall_tiles", "intergrams_prefetch",
           "intergrams_pass_scan", "intergrams_counts_export", "intergrams_counts_import",
           "intergrams_pass_select", "intergrams_shard_assign"]


class IgParams(ctypes.Structure):
    _fields_ = [(f, ctypes.c_uint32) for f in
                ("n", "k", "candidates", "base_n", "symbol_bits", "count_mode", "flags")]


class IgTuning(ctypes.Structure):
    _fields_ = [(f, ctypes.c_uint32) for f in
                ("ctas_per_sm", "threads", "words_per_thread", "smem_set_log2", "table_load_pct", "hot_log2",
                 "chain_from", "list_pct", "log_mode", "log_pct", "log_chunk_log2", "log_range_log2",
                 "dedupe_bitmap", "dense_prefix", "base_words_per_thread", "base_smem_set_log2",
                 "set_probes", "tile_buffers", "rs_depth", "tile_cache_hint", "prefetch_tiles", "spill_dedupe", "spill_min_fill", "carry_slots", "set_max_windows", "scan_variants")]


class IgPassStats(ctypes.Structure):
    _fields_ = [("j", ctypes.c_uint32), ("windows", ctypes.c_uint64), ("survivors", ctypes.c_uint64),
                ("registrations", ctypes.c_uint64), ("nonzero_selected", ctypes.c_uint64),
                ("scanned_bytes", ctypes.c_uint64)]


class IgServerConfig(ctypes.Structure):
    _fields_ = [("mem_budget", ctypes.c_uint64), ("max_active", ctypes.c_uint32), ("flags", ctypes.c_uint32),
                ("large_work", ctypes.c_uint64)]


class IgServerStats(ctypes.Structure):
    _fields_ = [("submitted", ctypes.c_uint64), ("completed", ctypes.c_uint64), ("failed", ctypes.c_uint64),
                ("active", ctypes.c_uint32), ("peak_active", ctypes.c_uint32), ("pending", ctypes.c_uint32),
                ("mem_used", ctypes.c_uint64), ("peak_mem", ctypes.c_uint64), ("mem_budget", ctypes.c_uint64)]


class IntergramsError(RuntimeError):
    def __init__(self, status: int, msg: str):
        super().__init__(f"{STATUS_NAMES.get(status, status)}: {msg}")
        self.status = status


_lib = None


def library_path() -> Path:
    return _build.LIB / "libintergrams.so"


def load(build_if_missing: bool = True):
    """Load the native library (building it first if asked and needed)."""
    global _lib
    if _lib is not None:
        return _lib
    path = library_path()
    if build_if_missing:
        path = _build.build_cuda()
    if not path.exists():
        raise RuntimeError(f"{path} is missing: the CUDA library must be built (no CPU fallback)")
    lib = ctypes.CDLL(str(path))
    P, U32 = ctypes.c_void_p, ctypes.c_uint32
    lib.intergrams_plan.restype = ctypes.c_int
    lib.intergrams_plan.argtypes = [ctypes.POINTER(IgParams), P, P, U32, P, ctypes.POINTER(IgTuning),
                                    ctypes.POINTER(ctypes.c_void_p)]
    lib.intergrams_pass.restype = ctypes.c_int
    lib.intergrams_pass.argtypes = [P, ctypes.POINTER(U32)]
    lib.intergrams_run.restype = ctypes.c_int
    lib.intergrams_run.argtypes = [P]
    lib.intergrams_rewind.restype = ctypes.c_int
    lib.intergrams_rewind.argtypes = [P]
    lib.intergrams_topk.restype = ctypes.c_int
    lib.intergrams_topk.argtypes = [P, P, P, U32, ctypes.POINTER(U32), ctypes.POINTER(U32)]
    lib.intergrams_stats.restype = ctypes.c_int
    lib.intergrams_stats.argtypes = [P, ctypes.POINTER(IgPassStats)]
    lib.intergrams_features.restype = ctypes.c_int
    lib.intergrams_features.argtypes = [P, P, P, ctypes.c_uint64, ctypes.POINTER(ctypes.c_uint64)]
    lib.intergrams_timings.restype = ctypes.c_int
    lib.intergrams_timings.argtypes = [P, P, P, U32, ctypes.POINTER(U32), ctypes.POINTER(U32)]
    lib.intergrams_free.restype = None
    lib.intergrams_free.argtypes = [P]
    lib.intergrams_dense_topk_static.restype = ctypes.c_int
    lib.intergrams_dense_topk_static.argtypes = [ctypes.POINTER(IgParams), P, P, U32, ctypes.c_uint64, P, P, P, P,
                                                 P]
    lib.intergrams_plan_device_bytes.restype = ctypes.c_int
    lib.intergrams_plan_device_bytes.argtypes = [P, ctypes.POINTER(ctypes.c_uint64)]
    lib.intergrams_server_create.restype = ctypes.c_int
    lib.intergrams_server_create.argtypes = [ctypes.POINTER(IgServerConfig), ctypes.POINTER(ctypes.c_void_p)]
    lib.intergrams_server_submit.restype = ctypes.c_int
    lib.intergrams_server_submit.argtypes = [P, ctypes.POINTER(IgParams), P, P, U32, ctypes.POINTER(IgTuning),
                                             ctypes.POINTER(ctypes.c_uint64)]
    lib.intergrams_server_wait.restype = ctypes.c_int
    lib.intergrams_server_wait.argtypes = [P, ctypes.c_uint64, ctypes.c_int64, P, P, U32, ctypes.POINTER(U32),
                                           ctypes.POINTER(ctypes.c_double)]
    lib.intergrams_server_stats.restype = ctypes.c_int
    lib.intergrams_server_stats.argtypes = [P, ctypes.POINTER(IgServerStats)]
    lib.intergrams_server_destroy.restype = None
    lib.intergrams_server_destroy.argtypes = [P]
    lib.intergrams_autotune.restype = ctypes.c_int
    lib.intergrams_autotune.argtypes = [ctypes.POINTER(IgParams), P, P, U32, P, ctypes.c_uint64,
                                        ctypes.POINTER(IgTuning), ctypes.POINTER(ctypes.c_float)]
    lib.intergrams_last_error.restype = ctypes.c_char_p
    lib.intergrams_last_error.argtypes = []
    lib.intergrams_test_fail_alloc.restype = ctypes.c_int
    lib.intergrams_test_fail_alloc.argtypes = [U32, ctypes.POINTER(ctypes.c_uint64)]
    lib.intergrams_prefetch.restype = ctypes.c_int
    lib.intergrams_prefetch.argtypes = [P, P]
    lib.intergrams_test_stall_tiles.restype = ctypes.c_int
    lib.intergrams_test_stall_tiles.argtypes = [P]
    lib.intergrams_pass_scan.restype = ctypes.c_int
    lib.intergrams_pass_scan.argtypes = [P, ctypes.POINTER(U32)]
    lib.intergrams_counts_export.restype = ctypes.c_int
    lib.intergrams_counts_export.argtypes = [P, P, ctypes.c_uint64, ctypes.POINTER(ctypes.c_uint64)]
    lib.intergrams_counts_import.restype = ctypes.c_int
    lib.intergrams_counts_import.argtypes = [P, P, ctypes.c_uint64]
    lib.intergrams_pass_select.restype = ctypes.c_int
    lib.intergrams_pass_select.argtypes = [P, ctypes.POINTER(U32)]
    lib.intergrams_shard_assign.restype = ctypes.c_int
    lib.intergrams_shard_assign.argtypes = [P, U32, U32, P, P]
    _lib = lib
    return lib


def _check(lib, st: int, what: str):
    if st not in (IG_OK, IG_DONE):
        raise IntergramsError(st, f"{what}: {lib.intergrams_last_error().decode(errors='replace')}")
    return st


def _ptr(x):
    """Device pointer of a torch tensor, or host pointer of a numpy array."""
    if x is None:
        return None
    if hasattr(x, "data_ptr"):
        return x.data_ptr()
    return np.ascontiguousarray(x).ctypes.data


class Plan:
    """One top-k n-gram job over a corpus (see include/intergrams.h).

    ``data``/``offsets`` are CUDA tensors (uint8 / int64 holding uint64
    boundaries) unless ``host_input`` is set, in which case they are numpy
    arrays and the library copies them to the device itself.
    """

    def __init__(self, data, offsets, *, n: int, k: int, candidates: int, base_n: int = 3,
                 symbol_bits: int = 8, count_mode: int = COUNT_ONCE_PER_SEQUENCE, graph: bool = False,
                 host_input: bool = False, timing: bool = False, autotune: bool = False, stream=None,
                 tuning: dict | None = None, sharded: bool = False, checks: bool = False):
        self._lib = load()
        self._h = ctypes.c_void_p(None)
        flags = ((F_GRAPH if graph else 0) | (F_HOST_INPUT if host_input else 0) | (F_TIMING if timing else 0)
                 | (F_AUTOTUNE if autotune else 0) | (F_SHARDED if sharded else 0)
                 | (F_EXHAUSTIVE_CHECKS if checks else 0))
        self.params = IgParams(n, k, candidates, base_n, symbol_bits, count_mode, flags)
        tun = IgTuning(**(tuning or {}))
        if host_input:
            self._keep = (np.ascontiguousarray(data, dtype=np.uint8),
                          np.ascontiguousarray(offsets, dtype=np.uint64))
        else:
            self._keep = (data, offsets)
        m = len(offsets) - 1
        if stream is None:
            stream_ptr = None
            try:
                import torch
                if torch.cuda.is_available():
                    stream_ptr = torch.cuda.current_stream().cuda_stream
            except ImportError:
                pass
        else:
            stream_ptr = getattr(stream, "cuda_stream", stream)
        _check(self._lib, self._lib.intergrams_plan(ctypes.byref(self.params), _ptr(self._keep[0]),
                                                    _ptr(self._keep[1]), m, stream_ptr,
                                                    ctypes.byref(tun), ctypes.byref(self._h)),
               "intergrams_plan")
        self.n = n
        self.m = m
        self.symbol_bits = symbol_bits

    def step(self):
        """Run the next pass; returns its j, or None when every pass has run."""
        j = ctypes.c_uint32(0)
        st = _check(self._lib, self._lib.intergrams_pass(self._h, ctypes.byref(j)), "intergrams_pass")
        return None if st == IG_DONE else j.value

    def run(self):
        _check(self._lib, self._lib.intergrams_run(self._h), "intergrams_run")

    def rewind(self):
        _check(self._lib, self._lib.intergrams_rewind(self._h), "intergrams_rewind")

    def prefetch(self, data=None):
        """With host input: start copying the next run's corpus (``data``, a
        numpy array of the same size, or the plan's own host buffer) into the
        plan's second device buffer; the next rewind switches to it."""
        if data is not None:
            data = np.ascontiguousarray(data, dtype=np.uint8)
            if data.nbytes != self._keep[0].nbytes:
                raise ValueError("prefetch needs a corpus of the plan's size")
            # kept alive until its copy has certainly landed: the copy queued
            # after it on the same copy stream starts only once it has
            self._next = (getattr(self, "_next", (None, None))[1], data)
        _check(self._lib, self._lib.intergrams_prefetch(self._h, None if data is None else data.ctypes.data),
               "intergrams_prefetch")

    def topk(self, capacity: int | None = None):
        """(keys, counts, j): keys is a (rows, ceil(j*bits/8)) uint8 array."""
        cap = self.params.k if capacity is None else int(capacity)
        row = (self.n * self.symbol_bits + 7) // 8
        keys = np.zeros((max(cap, 1), row), np.uint8)
        counts = np.zeros(max(cap, 1), np.uint64)
        kout, jout = ctypes.c_uint32(0), ctypes.c_uint32(0)
        _check(self._lib, self._lib.intergrams_topk(self._h, keys.ctypes.data, counts.ctypes.data, cap,
                                                    ctypes.byref(kout), ctypes.byref(jout)), "intergrams_topk")
        r, j = kout.value, jout.value
        rb = (j * self.symbol_bits + 7) // 8
        flat = keys.reshape(-1)[: r * rb].reshape(r, rb) if r else np.zeros((0, rb), np.uint8)
        return flat.copy(), counts[:r].copy(), j

    def features(self):
        """(row_ptr, cols): the Boolean sequence x top-k matrix in CSR form
        (uint64[m + 1] row starts, uint32 feature ids ascending per row)."""
        nnz = ctypes.c_uint64(0)
        _check(self._lib, self._lib.intergrams_features(self._h, None, None, 0, ctypes.byref(nnz)),
               "intergrams_features")
        row_ptr = np.zeros(self.m + 1, np.uint64)
        cols = np.zeros(max(nnz.value, 1), np.uint32)
        _check(self._lib, self._lib.intergrams_features(self._h, row_ptr.ctypes.data, cols.ctypes.data, nnz.value,
                                                        ctypes.byref(nnz)), "intergrams_features")
        return row_ptr, cols[: nnz.value].copy()

    def stats(self) -> dict:
        s = IgPassStats()
        _check(self._lib, self._lib.intergrams_stats(self._h, ctypes.byref(s)), "intergrams_stats")
        return {f: getattr(s, f) for f, _ in IgPassStats._fields_}

    def timings(self):
        """Per-pass scan-kernel and pass durations (ms) of the latest run, and
        the number of kernels launched since the last rewind."""
        cap = 128
        scan = np.zeros(cap, np.float32)
        pas = np.zeros(cap, np.float32)
        npass, kern = ctypes.c_uint32(0), ctypes.c_uint32(0)
        _check(self._lib, self._lib.intergrams_timings(self._h, scan.ctypes.data, pas.ctypes.data, cap,
                                                       ctypes.byref(npass), ctypes.byref(kern)),
               "intergrams_timings")
        r = npass.value
        return scan[:r].copy(), pas[:r].copy(), kern.value

    # sharded passes (include/intergrams.h): scan, export, (caller sums), import, select
    def pass_scan(self):
        """Scan of the next pass only; its j, or None when every pass has run."""
        j = ctypes.c_uint32(0)
        st = _check(self._lib, self._lib.intergrams_pass_scan(self._h, ctypes.byref(j)), "intergrams_pass_scan")
        return None if st == IG_DONE else j.value

    def counts_export(self, out):
        """The pending pass's counts into ``out`` (a CUDA uint32/int32 tensor
        with room for them); returns the number of slots."""
        n = ctypes.c_uint64(0)
        _check(self._lib, self._lib.intergrams_counts_export(self._h, _ptr(out), out.numel(), ctypes.byref(n)),
               "intergrams_counts_export")
        return n.value

    def counts_slots(self):
        """Number of counters of the pending pass."""
        n = ctypes.c_uint64(0)
        self._lib.intergrams_counts_export(self._h, None, 0, ctypes.byref(n))
        return n.value

    def counts_import(self, counts):
        _check(self._lib, self._lib.intergrams_counts_import(self._h, _ptr(counts), counts.numel()),
               "intergrams_counts_import")

    def pass_select(self):
        j = ctypes.c_uint32(0)
        _check(self._lib, self._lib.intergrams_pass_select(self._h, ctypes.byref(j)), "intergrams_pass_select")
        return j.value

    def test_stall_tiles(self):
        """Test hook: later corpus scans wait for tiles that are never sent,
        so their passes raise IG_ETIMEOUT after about a second."""
        _check(self._lib, self._lib.intergrams_test_stall_tiles(self._h), "intergrams_test_stall_tiles")

    def close(self):
        if self._h and self._h.value:
            self._lib.intergrams_free(self._h)
            self._h = ctypes.c_void_p(None)

    def __enter__(self):
        return self

    def __exit__(self, *exc):
        self.close()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


def test_fail_alloc(nth: int) -> int:
    """Test hook: the nth device allocation of the library from now on fails
    as out of memory (0 disarms). Returns the device allocations held now."""
    lib = load()
    live = ctypes.c_uint64(0)
    lib.intergrams_test_fail_alloc(int(nth), ctypes.byref(live))
    return live.value


def dense_topk_static(data, offsets, *, n: int, k: int, symbol_bits: int = 8,
                      count_mode: int = COUNT_ONCE_PER_SEQUENCE, total_symbols: int, stream=None,
                      keys_out=None, counts_out=None, rows_out=None, status_out=None):
    """Allocation-free exact top-k of short n-grams (intergrams_dense_topk_static).

    ``data``/``offsets`` are CUDA tensors; ``keys_out`` (uint8, k * row bytes),
    ``counts_out`` (int64, k), ``rows_out`` (int32, 1) and ``status_out``
    (int32, 1) are caller-owned CUDA tensors. The library allocates nothing;
    the work is enqueued on ``stream`` (default: torch's current stream) and
    not synchronised: ``status_out`` holds IG_OK or the device-side failure
    (then ``rows_out`` is 0) once the stream has reached it.
    """
    lib = load()
    m = len(offsets) - 1
    params = IgParams(n, k, k, n, symbol_bits, count_mode, 0)
    if stream is None:
        import torch
        stream_ptr = torch.cuda.current_stream().cuda_stream
    else:
        stream_ptr = getattr(stream, "cuda_stream", stream)
    st = lib.intergrams_dense_topk_static(ctypes.byref(params), _ptr(data), _ptr(offsets), m, int(total_symbols),
                                          stream_ptr, _ptr(keys_out), _ptr(counts_out), _ptr(rows_out),
                                          _ptr(status_out))
    _check(lib, st, "intergrams_dense_topk_static")


def shard_assign(offsets, nshards: int):
    """Byte-balanced greedy split of the sequences (intergrams_shard_assign):
    (shard of each sequence uint32[m], symbols per shard uint64[nshards])."""
    lib = load(build_if_missing=False) if _build.LIB.joinpath("libintergrams.so").exists() else load()
    off = np.ascontiguousarray(np.asarray(offsets, dtype=np.uint64))
    m = len(off) - 1
    out = np.zeros(max(m, 1), np.uint32)
    loads = np.zeros(max(nshards, 1), np.uint64)
    _check(lib, lib.intergrams_shard_assign(off.ctypes.data, m, nshards, out.ctypes.data, loads.ctypes.data),
           "intergrams_shard_assign")
    return out[:m].copy(), loads[:nshards].copy()


def test_stall_next_static_call():
    """Test hook: the next dense_topk_static call's scan waits for tiles that
    are never sent, so its status word reports IG_ETIMEOUT after about a
    second (intergrams_test_stall_tiles with no plan)."""
    lib = load()
    _check(lib, lib.intergrams_test_stall_tiles(None), "intergrams_test_stall_tiles")


class Server:
    """Continuous-batching job server (intergrams_server_*): submit jobs whose
    corpora are CUDA tensors, wait for their top-k. Marshalling only."""

    def __init__(self, mem_budget: int = 0, max_active: int = 8, fifo: bool = False, policy: str | None = None,
                 large_work: int = 0):
        """policy: "least_work_first" (default), "oldest_first", "fifo", or
        either of the first two with "+large_alone"."""
        self._lib = load()
        self._h = ctypes.c_void_p(None)
        policy = policy or ("fifo" if fifo else "least_work_first")
        flags = {"least_work_first": 0, "oldest_first": SRV_OLDEST_FIRST, "fifo": SRV_FIFO,
                 "least_work_first+large_alone": SRV_LARGE_ALONE,
                 "oldest_first+large_alone": SRV_OLDEST_FIRST | SRV_LARGE_ALONE}[policy]
        cfg = IgServerConfig(int(mem_budget), int(max_active), flags, int(large_work))
        _check(self._lib, self._lib.intergrams_server_create(ctypes.byref(cfg), ctypes.byref(self._h)),
               "intergrams_server_create")
        self._keep = {}
        self._meta = {}

    def submit(self, data, offsets, *, n: int, k: int, candidates: int, base_n: int = 3, symbol_bits: int = 8,
               count_mode: int = COUNT_ONCE_PER_SEQUENCE, tuning: dict | None = None) -> int:
        off = np.ascontiguousarray(offsets, dtype=np.uint64)
        params = IgParams(n, k, candidates, base_n, symbol_bits, count_mode, 0)
        tun = IgTuning(**(tuning or {}))
        jid = ctypes.c_uint64(0)
        _check(self._lib, self._lib.intergrams_server_submit(self._h, ctypes.byref(params), _ptr(data),
                                                             off.ctypes.data, len(off) - 1, ctypes.byref(tun),
                                                             ctypes.byref(jid)), "intergrams_server_submit")
        self._keep[jid.value] = data
        self._meta[jid.value] = (n, k, symbol_bits)
        return jid.value

    def wait(self, job_id: int, timeout_s: float | None = None):
        """(keys, counts, latency_s) of a finished job."""
        n, k, bits = self._meta.pop(job_id)
        row = (n * bits + 7) // 8
        keys = np.zeros((max(k, 1), row), np.uint8)
        counts = np.zeros(max(k, 1), np.uint64)
        kout, lat = ctypes.c_uint32(0), ctypes.c_double(0.0)
        tmo = -1 if timeout_s is None else int(timeout_s * 1e6)
        st = self._lib.intergrams_server_wait(self._h, job_id, tmo, keys.ctypes.data, counts.ctypes.data, k,
                                              ctypes.byref(kout), ctypes.byref(lat))
        self._keep.pop(job_id, None)
        _check(self._lib, st, "intergrams_server_wait")
        r = kout.value
        return keys[:r].copy(), counts[:r].copy(), lat.value

    def stats(self) -> dict:
        s = IgServerStats()
        _check(self._lib, self._lib.intergrams_server_stats(self._h, ctypes.byref(s)), "intergrams_server_stats")
        return {f: getattr(s, f) for f, _ in IgServerStats._fields_}

    def close(self):
        if self._h and self._h.value:
            self._lib.intergrams_server_destroy(self._h)
            self._h = ctypes.c_void_p(None)

    def __enter__(self):
        return self

    def __exit__(self, *exc):
        self.close()


def autotune(data, offsets, *, n: int, k: int, candidates: int, base_n: int = 3, symbol_bits: int = 8,
             count_mode: int = COUNT_ONCE_PER_SEQUENCE, sample_bytes: int = 0, stream=None):
    """intergrams_autotune: (best tuning dict, its job time in ms on the sample)."""
    lib = load()
    params = IgParams(n, k, candidates, base_n, symbol_bits, count_mode, 0)
    out = IgTuning()
    best = ctypes.c_float(0.0)
    if stream is None:
        import torch
        stream_ptr = torch.cuda.current_stream().cuda_stream
    else:
        stream_ptr = getattr(stream, "cuda_stream", stream)
    _check(lib, lib.intergrams_autotune(ctypes.byref(params), _ptr(data), _ptr(offsets), len(offsets) - 1,
                                        stream_ptr, int(sample_bytes), ctypes.byref(out), ctypes.byref(best)),
           "intergrams_autotune")
    return {f: getattr(out, f) for f, _ in IgTuning._fields_}, best.value
