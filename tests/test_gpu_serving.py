"""Continuous-batching server: every job's result is the same alone and in
the mix (exactly: all counts are integers), admission respects the memory
budget, and max_active = 1 runs one job at a time."""
import numpy as np
import pytest

torch = pytest.importorskip("torch")

from paper_2511_14955_gb300 import binding as B  # noqa: E402
from paper_2511_14955_gb300 import serving  # noqa: E402

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def pool():
    return serving.make_pool(6, seed=21, median_bytes=1.5e6, sigma=0.6, lo_bytes=200_000, hi_bytes=4_000_000)


def alone(pool, jb, z_factor=4, base_n=3):
    data, off = pool[jb.corpus]
    o = torch.from_numpy(off.view(np.int64).copy()).cuda()
    with B.Plan(data, o, n=jb.n, k=jb.k, candidates=z_factor * jb.k, base_n=base_n) as pl:
        pl.run()
        keys, counts, _ = pl.topk()
    return keys, counts


def test_each_result_is_the_same_alone_and_in_the_mix(pool):
    jobs = serving.job_stream(14, rate=400.0, n_corpora=len(pool), seed=5, ns=(4, 8, 16), ks=(64, 512))
    summary, results = serving.run_stream(pool, jobs, max_active=5, keep_results=True)
    assert summary["peak_active"] >= 2          # jobs really overlapped
    for i, jb in enumerate(jobs):
        ek, ec = alone(pool, jb)
        gk, gc = results[i]
        assert np.array_equal(gc, ec) and np.array_equal(gk, ek), f"job {i} differs in the mix"


def test_admission_respects_the_memory_budget(pool):
    jobs = serving.job_stream(8, rate=1000.0, n_corpora=len(pool), seed=7, ns=(8,), ks=(512,))
    # size one job with a dry-run plan, allow about two at once
    data, off = pool[0]
    need = []
    for jb in jobs:
        d, o = pool[jb.corpus]
        sv_bytes = _dry_bytes(d, o, jb)
        need.append(sv_bytes)
    budget = int(max(need) * 2.2)
    summary, results = serving.run_stream(pool, jobs, max_active=8, mem_budget=budget, keep_results=True)
    assert summary["peak_mem_gb"] * 1e9 <= budget
    for i, jb in enumerate(jobs):
        ek, ec = alone(pool, jb)
        assert np.array_equal(results[i][1], ec) and np.array_equal(results[i][0], ek)


def _dry_bytes(data, off, jb):
    import ctypes
    lib = B.load()
    params = B.IgParams(jb.n, jb.k, 4 * jb.k, 3, 8, 0, (1 << 4) | (1 << 6))   # OFFSETS_HOST | DRY_RUN
    h = ctypes.c_void_p(None)
    o = np.ascontiguousarray(off, dtype=np.uint64)
    assert lib.intergrams_plan(ctypes.byref(params), data.data_ptr(), o.ctypes.data, len(o) - 1, None, None,
                               ctypes.byref(h)) == 0
    b = ctypes.c_uint64(0)
    lib.intergrams_plan_device_bytes(h, ctypes.byref(b))
    lib.intergrams_free(h)
    return b.value


def test_one_job_per_launch_mode(pool):
    jobs = serving.job_stream(5, rate=1000.0, n_corpora=len(pool), seed=9, ns=(4, 8), ks=(64,))
    summary = serving.run_stream(pool, jobs, max_active=1)
    assert summary["peak_active"] == 1
    assert summary["jobs"] == 5 and summary["p99_ms"] >= summary["p50_ms"]


def test_job_larger_than_budget_is_rejected(pool):
    data, off = pool[0]
    with B.Server(mem_budget=1 << 20, max_active=2) as sv:
        with pytest.raises(B.IntergramsError) as ei:
            sv.submit(data, off, n=8, k=512, candidates=2048)
        assert ei.value.status == -2


def test_least_work_first_admits_the_small_job_ahead():
    """With one slot busy, a large job and then a small job queue up: the
    default policy admits the small one first, arrival order the large one;
    results are the same either way."""
    import time
    big = serving.make_pool(1, seed=41, median_bytes=60e6, sigma=0.01, lo_bytes=50_000_000, hi_bytes=70_000_000)[0]
    small = serving.make_pool(1, seed=42, median_bytes=3e5, sigma=0.01, lo_bytes=200_000, hi_bytes=400_000)[0]
    order = {}
    rows = {}
    for fifo in (False, True):
        with B.Server(max_active=1, fifo=fifo) as sv:
            first = sv.submit(*big, n=16, k=1024, candidates=4096)      # occupies the slot
            t_b = time.perf_counter()
            b = sv.submit(*big, n=8, k=1024, candidates=4096)
            t_s = time.perf_counter()
            s = sv.submit(*small, n=8, k=1024, candidates=4096)
            done = {}
            for name, jid, t in (("small", s, t_s), ("big", b, t_b), ("first", first, 0.0)):
                keys, counts, lat = sv.wait(jid)
                rows[(fifo, name)] = (keys.tobytes(), counts.tolist())
                done[name] = lat + t                  # completion on the perf_counter clock
            order[fifo] = done["small"] < done["big"]
    assert order[False] and not order[True]
    assert rows[(False, "small")] == rows[(True, "small")] and rows[(False, "big")] == rows[(True, "big")]


def test_served_job_grows_its_survivor_lists(pool):
    """A served job whose survivor lists are far too small: the server grows
    them, runs the job again and returns the exact rows."""
    data, off = pool[0]
    want = alone(pool, serving.Job(0.0, 0, 8, 256))
    with B.Server(max_active=2) as sv:
        jid = sv.submit(data, off, n=8, k=256, candidates=1024, base_n=3, tuning=dict(chain_from=5, list_pct=1))
        keys, counts, _ = sv.wait(jid, timeout_s=120)
    assert np.array_equal(counts, want[1]) and np.array_equal(keys, want[0])


def test_large_jobs_run_alone(pool):
    """IG_SRV_LARGE_ALONE with every job counted as large (a 1-byte
    threshold): no two jobs ever run together, under either admission order,
    and every result is exact."""
    jobs = serving.job_stream(10, rate=2000.0, n_corpora=len(pool), seed=17, ns=(4, 8), ks=(64, 512))
    for policy in ("oldest_first+large_alone", "least_work_first+large_alone"):
        summary, results = serving.run_stream(pool, jobs, max_active=8, policy=policy, large_work=1,
                                              keep_results=True)
        assert summary["peak_active"] == 1
        for i, jb in enumerate(jobs):
            ek, ec = alone(pool, jb)
            assert np.array_equal(results[i][1], ec) and np.array_equal(results[i][0], ek)
    # with the default threshold these small jobs overlap
    summary = serving.run_stream(pool, jobs, max_active=8, policy="oldest_first+large_alone")
    assert summary["peak_active"] >= 2
