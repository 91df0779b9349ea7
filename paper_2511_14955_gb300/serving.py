"""Poisson job stream against the continuous-batching server.

Jobs arrive at exponential inter-arrival times; each names a corpus (drawn
from a seeded pool of device-resident corpora whose total sizes follow the
workload's lognormal law), n and k. The client submits each job at its
arrival time; the server (native, ``intergrams_server_*``) admits, batches
and runs them. Latency is measured by the server from submission to
completion (results ready on the host). Only marshalling and timing live
here; all computation runs in the library's kernels.
"""
from __future__ import annotations

import threading
import time
from dataclasses import dataclass

import numpy as np

from . import binding, synth


@dataclass
class Job:
    arrival: float      # seconds after the stream starts
    corpus: int         # index into the pool
    n: int
    k: int


def make_pool(n_corpora: int, seed: int, median_bytes: float = 64e6, sigma: float = np.log(32) / 3,
              lo_bytes: int = 1 << 20, hi_bytes: int = 2 << 30, device="cuda"):
    """Corpora of the 2 MiB workload's byte law (order-1 Markov, Zipf(1.1)
    rows, zero blocks), sequences U[4, 64] KiB, total sizes lognormal
    (median 64 MB, sigma ln(32)/3) clamped to [lo, hi]."""
    import torch
    w = synth.WORKLOADS["markov_2mb"]
    rng = np.random.default_rng(seed)
    pool = []
    for i in range(n_corpora):
        size = float(np.clip(np.exp(np.log(median_bytes) + sigma * rng.standard_normal()), lo_bytes, hi_bytes))
        lens = []
        tot = 0
        while tot < size:
            L = int(rng.integers(4096, 65536 + 1))
            lens.append(L)
            tot += L
        off = synth.offsets_from_lengths(lens)
        data = synth.fill(w.model, seed * 1000 + i, off, 8)
        pool.append((torch.from_numpy(data).to(device), off))
    return pool


def job_stream(n_jobs: int, rate: float, n_corpora: int, seed: int, ns=(4, 8, 16), ks=(1024, 16384, 262144)):
    rng = np.random.default_rng(seed)
    t = 0.0
    jobs = []
    for _ in range(n_jobs):
        t += rng.exponential(1.0 / rate)
        jobs.append(Job(t, int(rng.integers(0, n_corpora)), int(rng.choice(ns)), int(rng.choice(ks))))
    return jobs


def run_stream(pool, jobs, *, max_active: int, mem_budget: int = 0, z_factor: int = 4, base_n: int = 3,
               tuning: dict | None = None, keep_results: bool = False, fifo: bool = False,
               policy: str | None = None, large_work: int = 0):
    """Submit every job at its arrival time; returns latency and throughput
    figures. ``policy``: "least_work_first" (the server's default),
    "oldest_first" or "fifo" (arrival order on default-priority streams, the
    one-job-per-launch baseline; also ``fifo=True``)."""
    results = {}
    lat = [None] * len(jobs)
    policy = policy or ("fifo" if fifo else "least_work_first")
    with binding.Server(mem_budget=mem_budget, max_active=max_active, policy=policy, large_work=large_work) as sv:
        ids = [None] * len(jobs)
        ready = threading.Event()
        errors = []

        def waiter():
            ready.wait()
            for i in range(len(jobs)):
                while ids[i] is None:
                    time.sleep(0.0005)
                try:
                    keys, counts, latency = sv.wait(ids[i])
                    lat[i] = latency
                    if keep_results:
                        results[i] = (keys, counts)
                except Exception as e:  # noqa: BLE001 - reported to the caller
                    errors.append((i, e))

        th = threading.Thread(target=waiter, daemon=True)
        th.start()
        t0 = time.perf_counter()
        ready.set()
        for i, jb in enumerate(jobs):
            now = time.perf_counter() - t0
            if jb.arrival > now:
                time.sleep(jb.arrival - now)
            data, off = pool[jb.corpus]
            ids[i] = sv.submit(data, off, n=jb.n, k=jb.k, candidates=z_factor * jb.k, base_n=base_n,
                               tuning=tuning)
        th.join()
        makespan = time.perf_counter() - t0
        stats = sv.stats()
    if errors:
        raise RuntimeError(f"{len(errors)} jobs failed, first: {errors[0]}")
    scanned = sum(int(pool[jb.corpus][1][-1]) * (jb.n - min(base_n, jb.n) + 1) for jb in jobs)
    lat_ms = np.array(lat) * 1e3
    out = {"jobs": len(jobs), "max_active": max_active, "policy": policy,
           "p50_ms": float(np.percentile(lat_ms, 50)),
           "p99_ms": float(np.percentile(lat_ms, 99)), "mean_ms": float(lat_ms.mean()),
           "makespan_s": makespan, "scanned_gb": scanned / 1e9, "gbps": scanned / makespan / 1e9,
           "peak_active": stats["peak_active"], "peak_mem_gb": stats["peak_mem"] / 1e9}
    return (out, results) if keep_results else out
