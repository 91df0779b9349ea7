"""The byte-balanced greedy split of a corpus into shards (host code of the
C ABI, no GPU): every sequence in exactly one shard, longest first to the
lightest shard, and the largest shard exceeds the smallest by at most one
sequence's length."""
import numpy as np
import pytest

from paper_2511_14955_gb300 import binding as B


def greedy(L, g):
    """The same rule written out in Python."""
    load = [0] * g
    out = [0] * len(L)
    for i in sorted(range(len(L)), key=lambda i: (-L[i], i)):
        s = min(range(g), key=lambda x: (load[x], x))
        out[i] = s
        load[s] += L[i]
    return out, load


@pytest.mark.parametrize("seed", range(6))
def test_assign_matches_the_greedy_rule(seed):
    rng = np.random.default_rng(seed)
    L = rng.integers(0, 5000, size=int(rng.integers(1, 300)))
    L[rng.random(len(L)) < 0.1] = 0
    off = np.concatenate([[0], np.cumsum(L)]).astype(np.uint64)
    for g in (1, 2, 3, 8, 400):
        shard, loads = B.shard_assign(off, g)
        want, wload = greedy([int(x) for x in L], g)
        assert shard.tolist() == want and loads.tolist() == wload
        assert int(loads.sum()) == int(L.sum())
        assert int(loads.max()) - int(loads.min()) <= int(L.max())


def test_assign_rejects_bad_input():
    with pytest.raises(B.IntergramsError):
        B.shard_assign(np.array([0, 5, 3], np.uint64), 2)
    with pytest.raises(B.IntergramsError):
        B.shard_assign(np.array([0, 5], np.uint64), 0)
