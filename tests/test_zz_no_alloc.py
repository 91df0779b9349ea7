"""The allocation-free entry point (intergrams_dense_topk_static).

It exists for callers that cannot allocate device memory when they need an
answer - code inside a memory pool that owns the device budget, hot paths
with a no-allocation contract, embedders that forbid cudaMalloc after
start-up. Its tables live in a fixed device array inside the library. Here
it is called through the C ABI twice in a row, on different inputs, and each
result must equal the planned path's (intergrams_plan/run/topk with
n = base_n) exactly: all counts are integers, so the tolerance is zero.
"""
import numpy as np
import pytest

torch = pytest.importorskip("torch")

from paper_2511_14955_gb300 import binding as B  # noqa: E402
from paper_2511_14955_gb300 import synth  # noqa: E402

pytestmark = pytest.mark.gpu


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
    B.dense_topk_static(d, o, n=n, k=k, symbol_bits=bits, count_mode=mode, total_symbols=total,
                        keys_out=keys, counts_out=counts, rows_out=rows)
    torch.cuda.synchronize()
    r = int(rows.item())
    return keys[: r * rb].cpu().numpy().reshape(r, rb), counts[:r].cpu().numpy().view(np.uint64)


def test_two_calls_in_a_row_match_the_planned_path():
    cases = [
        # (corpus, n, k, symbol_bits, count_mode)
        (synth.make_corpus("malware_8gb", m=30, max_len=200_000, seed=11), 2, 4000, 8, 0),
        (synth.make_corpus("genomic_5gbp", m=4, max_len=300_001, seed=12), 8, 20000, 2, 1),
    ]
    for (data, off, bits), n, k, bits_, mode in cases:
        d = torch.from_numpy(np.array(data, copy=True)).cuda()
        o = torch.from_numpy(off.view(np.int64).copy()).cuda()
        total = int(off[-1])
        ek, ec = planned(d, o, n, k, bits_, mode)
        gk, gc = static_call(d, o, total, n, k, bits_, mode)
        assert len(ec) > 0
        assert np.array_equal(gc, ec)
        assert np.array_equal(gk, ek)


def test_sizes_beyond_the_scratch_are_rejected():
    data, off, _ = synth.make_corpus("markov_2mb", m=2)
    d = torch.from_numpy(np.array(data, copy=True)).cuda()
    o = torch.from_numpy(off.view(np.int64).copy()).cuda()
    out = torch.zeros(16, dtype=torch.uint8, device="cuda")
    cnt = torch.zeros(4, dtype=torch.int64, device="cuda")
    rows = torch.zeros(1, dtype=torch.int32, device="cuda")
    for n, k in ((3, 4), (2, 70000)):
        with pytest.raises(B.IntergramsError) as ei:
            B.dense_topk_static(d, o, n=n, k=k, total_symbols=int(off[-1]), keys_out=out, counts_out=cnt,
                                rows_out=rows)
        assert ei.value.status == -1
