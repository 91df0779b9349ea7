"""Element-wise parity at the headline parameters, on sequences as long as
the full malware-like workload's.

The corpus follows the 8.8 GB workload's byte law (order-1 Markov bytes with
Zipf rows, zero blocks, planted motifs) with its lognormal lengths, about
230 MB in all, and five sequences of 4 to 8 MiB (the workload's cap). The
job is the benchmark's: n = 8, k = 65,536, Z = 262,144, base 3, autotuned
knobs. So the paths the full-size job takes - rank/select over the 67M
candidate slots with 16-bit counters, the Eq. 2 spill lists of multi-MiB
sequences partitioned twice, the autotuned tile and set sizes - are compared
with the oracle row for row: after every pass j = 3..8 (pass by pass) and
for the job captured as one CUDA graph, under Eq. 2 and Eq. 1. The oracle is
Algorithm 3 run over groups of whole sequences on every host core
(``oracle/sharded.py``, pinned against the single-threaded oracle). All
counts are integers: keys and counts must be equal, tolerance zero.
"""
import numpy as np
import pytest

torch = pytest.importorskip("torch")

from oracle import sharded  # noqa: E402
from paper_2511_14955_gb300 import binding as B  # noqa: E402
from paper_2511_14955_gb300 import synth  # noqa: E402

pytestmark = pytest.mark.gpu

N, K, Z, BASE = 8, 65536, 262144, 3
LONG = [8 << 20, 7 << 20, 6 << 20, 5 << 20, 4 << 20]


def headline_corpus(seed=21, short_bytes=200_000_000):
    w = synth.WORKLOADS["malware_8gb"]
    L = synth.lengths_for(w, seed).astype(np.int64)
    L = L[np.cumsum(L) <= short_bytes]
    L = np.concatenate([L[:40], np.array(LONG, np.int64), L[40:]]).astype(np.uint64)
    off = synth.offsets_from_lengths(L)
    return synth.fill(w.model, seed, off, 8), off


@pytest.fixture(scope="module")
def corpus():
    data, off = headline_corpus()
    assert (np.diff(off.astype(np.int64)) >= 4 << 20).sum() >= len(LONG) and len(off) - 1 >= 200
    return data, off


@pytest.fixture(scope="module")
def expected():
    """Oracle rows after every pass, per count mode (computed once; the pool
    is started with spawn)."""
    cache = {}

    def get(data, off, mode):
        if mode not in cache:
            cache[mode] = {j: (k, c) for j, k, c in
                           sharded.intergrams(data, off, N, K, Z, base_n=BASE, count_mode=mode, per_pass=True)}
        return cache[mode]
    return get


@pytest.mark.parametrize("mode", [0, 1])
def test_every_pass_and_the_graph_job_match_the_oracle(corpus, expected, mode):
    data, off = corpus
    want = expected(data, off, mode)
    d = torch.from_numpy(data).cuda()
    o = torch.from_numpy(off.view(np.int64)).cuda()
    try:
        # pass by pass, autotuned knobs: the top-k after every pass
        with B.Plan(d, o, n=N, k=K, candidates=Z, base_n=BASE, count_mode=mode, autotune=True) as pl:
            seen = []
            while (j := pl.step()) is not None:
                keys, counts, jj = pl.topk()
                ek, ec = want[j]
                assert jj == j and len(counts) == len(ec) == K, (j, len(counts), len(ec))
                assert np.array_equal(counts, ec), f"pass {j}: counts differ"
                assert np.array_equal(keys, ek), f"pass {j}: keys differ"
                seen.append(j)
            assert seen == list(range(BASE, N + 1))
        # the benchmark's launch: the whole job as one CUDA graph
        with B.Plan(d, o, n=N, k=K, candidates=Z, base_n=BASE, count_mode=mode, autotune=True, graph=True) as pl:
            for _ in range(2):  # replayed after a rewind
                pl.rewind()
                pl.run()
                keys, counts, j = pl.topk()
                ek, ec = want[N]
                assert j == N and np.array_equal(counts, ec) and np.array_equal(keys, ek)
    finally:
        del d, o
        torch.cuda.empty_cache()
