"""The allocation-free entry point (intergrams_dense_topk_static).

It exists for callers that cannot allocate device memory when they need an
answer - code inside a memory pool that owns the device budget, hot paths
with a no-allocation contract, embedders that forbid cudaMalloc after
start-up. Its tables live in a fixed device array inside the library. Here
it is called through the C ABI twice in a row, on different inputs, and each
result must equal the planned path's (intergrams_plan/run/topk with
n = base_n) exactly: all counts are integers, so the tolerance is zero.
A failure the device reports (a tile wait that ran out, made to happen by a
test hook on the host) comes back through the call's status word.
"""
import time

import numpy as np
import pytest

torch = pytest.importorskip("torch")

from paper_2511_14955_gb300 import binding as B  # noqa: E402
from paper_2511_14955_gb300 import synth  # noqa: E402

pytestmark = pytest.mark.gpu

IG_EINVAL, IG_ETIMEOUT = -1, -5


def planned(d, o, n, k, bits, mode):
    with B.Plan(d, o, n=n, k=k, candidates=k, base_n=n, symbol_bits=bits, count_mode=mode) as pl:
        pl.run()
        keys, counts, _ = pl.topk()
    return keys, counts


def static_call(d, o, total, n, k, bits, mode):
    rb = (n * bits + 7) // 8
    keys = torch.full((k * rb,), 0xAB, dtype=torch.uint8, device="cuda")
    counts = torch.full((k,), -1, dtype=torch.int64, device="cuda")
    rows = torch.full((1,), -1, dtype=torch.int32, device="cuda")
    status = torch.full((1,), 77, dtype=torch.int32, device="cuda")
    B.dense_topk_static(d, o, n=n, k=k, symbol_bits=bits, count_mode=mode, total_symbols=total,
                        keys_out=keys, counts_out=counts, rows_out=rows, status_out=status)
    torch.cuda.synchronize()
    r = int(rows.item())
    return keys[: r * rb].cpu().numpy().reshape(r, rb), counts[:r].cpu().numpy().view(np.uint64), int(status.item())


CASES = [
    # (corpus, n, k, symbol_bits, count_mode)
    (lambda: synth.make_corpus("malware_8gb", m=30, max_len=200_000, seed=11), 2, 4000, 8, 0),
    (lambda: synth.make_corpus("genomic_5gbp", m=4, max_len=300_001, seed=12), 8, 20000, 2, 1),
]


def test_two_calls_in_a_row_match_the_planned_path():
    for make, n, k, bits, mode in CASES:
        data, off, _ = make()
        d = torch.from_numpy(np.array(data, copy=True)).cuda()
        o = torch.from_numpy(off.view(np.int64).copy()).cuda()
        total = int(off[-1])
        ek, ec = planned(d, o, n, k, bits, mode)
        gk, gc, st = static_call(d, o, total, n, k, bits, mode)
        assert st == 0
        assert len(ec) > 0
        assert np.array_equal(gc, ec)
        assert np.array_equal(gk, ek)


def test_device_failure_is_reported_then_next_call_is_exact():
    data, off, _ = synth.make_corpus("malware_8gb", m=12, max_len=100_000, seed=13)
    d = torch.from_numpy(np.array(data, copy=True)).cuda()
    o = torch.from_numpy(off.view(np.int64).copy()).cuda()
    total = int(off[-1])
    ek, ec = planned(d, o, 2, 1000, 8, 0)
    B.test_stall_next_static_call()
    t0 = time.perf_counter()
    gk, gc, st = static_call(d, o, total, 2, 1000, 8, 0)
    dt = time.perf_counter() - t0
    assert st == IG_ETIMEOUT and len(gc) == 0
    assert 0.5 < dt < 60.0, dt  # each CTA gave up after its ~1 s wait
    # the hook fires once: the next call is exact again (epochs carried over)
    for _ in range(2):
        gk, gc, st = static_call(d, o, total, 2, 1000, 8, 0)
        assert st == 0 and np.array_equal(gk, ek) and np.array_equal(gc, ec)


def test_sizes_beyond_the_scratch_are_rejected():
    data, off, _ = synth.make_corpus("markov_2mb", m=2)
    d = torch.from_numpy(np.array(data, copy=True)).cuda()
    o = torch.from_numpy(off.view(np.int64).copy()).cuda()
    out = torch.zeros(16, dtype=torch.uint8, device="cuda")
    cnt = torch.zeros(4, dtype=torch.int64, device="cuda")
    rows = torch.zeros(1, dtype=torch.int32, device="cuda")
    status = torch.zeros(1, dtype=torch.int32, device="cuda")
    for n, k, mode, total in ((3, 4, 0, int(off[-1])), (2, 70000, 0, int(off[-1])), (2, 4, 1, 1 << 32)):
        with pytest.raises(B.IntergramsError) as ei:
            B.dense_topk_static(d, o, n=n, k=k, count_mode=mode, total_symbols=total, keys_out=out,
                                counts_out=cnt, rows_out=rows, status_out=status)
        assert ei.value.status == IG_EINVAL
