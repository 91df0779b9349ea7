"""Full-size workloads in the benchmark's launch configuration (autotuned
knobs, the job as one CUDA graph). The oracle cannot redo these jobs in
seconds, so it checks what it can compute one by one: the exact count of a
sample of output rows (Eq. 2 counts by definition, over the whole corpus),
and properties that hold at any size - rank order by (count desc, bytes asc),
no duplicate rows, counts bounded by the number of sequences."""
import numpy as np
import pytest

torch = pytest.importorskip("torch")

from oracle import oracle as O  # noqa: E402
from paper_2511_14955_gb300 import binding as B  # noqa: E402
from paper_2511_14955_gb300 import synth  # noqa: E402

pytestmark = pytest.mark.gpu


def run_full(name, n=None, step=False):
    w = synth.WORKLOADS[name]
    data, off, bits = synth.make_corpus(name)
    d = torch.from_numpy(data).cuda()
    o = torch.from_numpy(off.view(np.int64)).cuda()
    n = n or w.n
    base_rows = None
    with B.Plan(d, o, n=n, k=w.k, candidates=w.candidates, base_n=w.base_n, symbol_bits=bits,
                graph=not step, autotune=True) as pl:
        if step:
            while True:
                j = pl.step()
                if j is None:
                    break
                if j == w.base_n:
                    base_rows = pl.topk()
        else:
            pl.run()
        keys, counts, j = pl.topk()
    del d, o
    torch.cuda.empty_cache()
    return data, off, bits, keys, counts, j, base_rows


def codes(rows, n, bits):
    if bits == 8:
        return rows
    return np.stack([synth.unpack_2bit(r, n) for r in rows])


def check_properties(keys, counts, m):
    assert counts.max() <= m and counts.min() >= 1
    order = [(-int(c), bytes(k)) for k, c in zip(keys, counts)]
    assert order == sorted(order)
    assert len({bytes(k) for k in keys}) == len(keys)


def sample_idx(r, nsample=40):
    return np.unique(np.concatenate([np.arange(min(8, r)), np.linspace(0, r - 1, nsample).astype(int)]))


def test_malware_8gb_full_size():
    w = synth.WORKLOADS["malware_8gb"]
    data, off, bits, keys, counts, j, base = run_full("malware_8gb", step=True)
    assert j == 8 and len(counts) == w.k
    check_properties(keys, counts, w.m)
    idx = sample_idx(len(counts))
    assert np.array_equal(O.count_keys(data, off, keys[idx]), counts[idx])
    bk, bc, bj = base
    assert bj == 3 and len(bc) == w.k
    check_properties(bk, bc, w.m)
    bidx = sample_idx(len(bc), 24)
    assert np.array_equal(O.count_keys(data, off, bk[bidx]), bc[bidx])


def test_malware_8gb_graph_matches_stepwise():
    """The graph launch the benchmark times returns the same rows as pass-by-pass launches."""
    w = synth.WORKLOADS["malware_8gb"]
    data, off, bits = synth.make_corpus("malware_8gb", m=3000)
    d = torch.from_numpy(data).cuda()
    o = torch.from_numpy(off.view(np.int64)).cuda()
    outs = []
    for graph in (True, False):
        with B.Plan(d, o, n=w.n, k=w.k, candidates=w.candidates, base_n=w.base_n, graph=graph,
                    autotune=True) as pl:
            pl.run()
            outs.append(pl.topk())
    assert np.array_equal(outs[0][0], outs[1][0]) and np.array_equal(outs[0][1], outs[1][1])


@pytest.mark.parametrize("n", [21, 31])
def test_genomic_full_size(n):
    w = synth.WORKLOADS["genomic_5gbp"]
    data, off, bits, keys, counts, j, _ = run_full("genomic_5gbp", n=n)
    assert j == n and len(counts) == w.k
    check_properties(keys, counts, w.m)
    idx = sample_idx(len(counts), 24)
    got = O.count_keys(data, off, codes(keys[idx], n, 2), symbol_bits=2)
    assert np.array_equal(got, counts[idx])


def test_largen_full_size():
    w = synth.WORKLOADS["largen_6gb"]
    data, off, bits, keys, counts, j, _ = run_full("largen_6gb")
    assert j == 64 and len(counts) == w.k
    check_properties(keys, counts, w.m)
    idx = sample_idx(len(counts), 24)
    assert np.array_equal(O.count_keys(data, off, keys[idx]), counts[idx])


def test_malware_8gb_feature_matrix():
    """Fig. 1's Boolean matrix of the 8.8 GB job: the column sums are the
    top-k's Eq. 2 counts, rows are sorted and distinct, and sampled rows
    equal the oracle's matrix of those sequences."""
    w = synth.WORKLOADS["malware_8gb"]
    data, off, bits = synth.make_corpus("malware_8gb")
    d = torch.from_numpy(data).cuda()
    o = torch.from_numpy(off.view(np.int64)).cuda()
    with B.Plan(d, o, n=w.n, k=w.k, candidates=w.candidates, base_n=w.base_n, graph=True, autotune=True) as pl:
        pl.run()
        keys, counts, _ = pl.topk()
        row_ptr, cols = pl.features()
    del d, o
    torch.cuda.empty_cache()
    assert row_ptr[0] == 0 and row_ptr[-1] == len(cols) and np.all(np.diff(row_ptr.astype(np.int64)) >= 0)
    assert np.array_equal(np.bincount(cols, minlength=len(keys)), counts)
    rng = np.random.default_rng(5)
    for i in rng.choice(w.m, size=12, replace=False):
        a, b = int(off[i]), int(off[i + 1])
        row = cols[row_ptr[i]:row_ptr[i + 1]]
        assert np.all(np.diff(row.astype(np.int64)) > 0)
        er, ec = O.features(data[a:b], np.array([0, b - a], np.uint64), keys)
        assert np.array_equal(row, ec), i
