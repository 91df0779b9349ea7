"""Failure paths made on the host (GPU; nothing here faults, traps or hangs
the device):

* every device allocation of a plan, of the feature matrix and of a served
  job made to fail in turn: the call returns IG_ENOMEM, nothing it had
  allocated stays allocated, and the same call succeeds once disarmed with
  results equal to the oracle's;
* the scan's bounded tile wait made to run out (its copies are never issued):
  the pass returns IG_ETIMEOUT after about a second, and the device then
  runs a fresh plan bit-exactly.
"""
import time

import numpy as np
import pytest

torch = pytest.importorskip("torch")

from oracle import oracle as O  # noqa: E402
from paper_2511_14955_gb300 import binding as B  # noqa: E402
from paper_2511_14955_gb300 import synth  # noqa: E402

pytestmark = pytest.mark.gpu

IG_ENOMEM, IG_ETIMEOUT, IG_ESTATE = -2, -5, -7


@pytest.fixture(scope="module")
def small():
    data, off, _ = synth.make_corpus("malware_8gb", seed=4, m=24, max_len=1 << 16)
    d = torch.from_numpy(data).cuda()
    o = torch.from_numpy(off.view(np.int64)).cuda()
    ek, ec = O.intergrams(data, off, 6, 256, 1024, base_n=3)
    return data, off, d, o, ek, ec


@pytest.fixture(autouse=True)
def disarm():
    B.test_fail_alloc(0)
    yield
    B.test_fail_alloc(0)


@pytest.mark.parametrize("graph", [False, True])
def test_each_plan_allocation_failing_releases_everything(small, graph):
    data, off, d, o, ek, ec = small
    base = B.test_fail_alloc(0)
    failures = 0
    for nth in range(1, 200):
        B.test_fail_alloc(nth)
        try:
            pl = B.Plan(d, o, n=6, k=256, candidates=1024, base_n=3, graph=graph)
        except B.IntergramsError as e:
            assert e.status == IG_ENOMEM, e
            failures += 1
            assert B.test_fail_alloc(0) == base, f"allocation {nth} failing left buffers allocated"
            continue
        B.test_fail_alloc(0)
        with pl:
            pl.run()
            gk, gc, _ = pl.topk()
        assert np.array_equal(gk, ek) and np.array_equal(gc, ec)
        break
    else:
        pytest.fail("the plan never succeeded")
    assert failures >= 10  # the plan makes many allocations; each one failed in turn
    assert B.test_fail_alloc(0) == base


def test_feature_matrix_allocation_failing(small):
    data, off, d, o, ek, _ = small
    base = B.test_fail_alloc(0)
    with B.Plan(d, o, n=6, k=256, candidates=1024, base_n=3) as pl:
        pl.run()
        held = B.test_fail_alloc(0)
        failures = 0
        for nth in range(1, 12):
            B.test_fail_alloc(nth)
            try:
                row_ptr, cols = pl.features()
            except B.IntergramsError as e:
                assert e.status == IG_ENOMEM, e
                failures += 1
                continue
            break
        B.test_fail_alloc(0)
        assert failures >= 1
        row_ptr, cols = pl.features()
        er, ecols = O.features(data, off, ek)
        assert np.array_equal(row_ptr, er) and np.array_equal(cols, ecols)
        assert B.test_fail_alloc(0) >= held
    assert B.test_fail_alloc(0) == base


def test_served_job_allocation_failing(small):
    """A job whose plan cannot allocate fails alone; the server goes on."""
    data, off, d, o, ek, ec = small
    with B.Server() as sv:
        B.test_fail_alloc(3)
        bad = sv.submit(d, off, n=6, k=256, candidates=1024, base_n=3)
        with pytest.raises(B.IntergramsError) as ei:
            sv.wait(bad, timeout_s=60)
        assert ei.value.status == IG_ENOMEM
        B.test_fail_alloc(0)
        good = sv.submit(d, off, n=6, k=256, candidates=1024, base_n=3)
        gk, gc, _ = sv.wait(good, timeout_s=60)
        assert np.array_equal(gk, ek) and np.array_equal(gc, ec)
        st = sv.stats()
        assert st["failed"] == 1 and st["completed"] >= 1


@pytest.mark.parametrize("first_pass", [True, False])
def test_tile_wait_runs_out_then_device_is_usable(small, first_pass):
    data, off, d, o, ek, ec = small
    pl = B.Plan(d, o, n=6, k=256, candidates=1024, base_n=3)
    try:
        if not first_pass:
            assert pl.step() == 3          # the base pass runs normally
        pl.test_stall_tiles()
        t0 = time.perf_counter()
        with pytest.raises(B.IntergramsError) as ei:
            pl.step()
        dt = time.perf_counter() - t0
        assert ei.value.status == IG_ETIMEOUT
        assert 0.5 < dt < 60.0, dt            # each CTA gave up after its ~1 s wait
    finally:
        pl.close()
    with B.Plan(d, o, n=6, k=256, candidates=1024, base_n=3) as pl2:
        pl2.run()
        gk, gc, _ = pl2.topk()
    assert np.array_equal(gk, ek) and np.array_equal(gc, ec)


def test_stall_hook_refuses_graph_plans(small):
    _, _, d, o, _, _ = small
    with B.Plan(d, o, n=6, k=256, candidates=1024, base_n=3, graph=True) as pl:
        with pytest.raises(B.IntergramsError) as ei:
            pl.test_stall_tiles()
        assert ei.value.status == IG_ESTATE
