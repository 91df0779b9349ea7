"""Input pipelining with host input (GPU): intergrams_prefetch copies the
next run's corpus into the plan's second device buffer while the current
run computes; the next rewind switches buffers. Every run must equal the
oracle on the corpus it was given, pass by pass or as a graph, and a plain
rewind still re-reads the plan's host buffer."""
import numpy as np
import pytest

torch = pytest.importorskip("torch")

from oracle import oracle as O  # noqa: E402
from paper_2511_14955_gb300 import binding as B  # noqa: E402
from paper_2511_14955_gb300 import synth  # noqa: E402

pytestmark = pytest.mark.gpu

IG_ESTATE = -7
N, K, Z, BASE = 5, 300, 1200, 2


def job(pl):
    pl.run()
    k, c, _ = pl.topk()
    return k, c


@pytest.mark.parametrize("graph", [False, True])
def test_prefetch_alternates_buffers(graph):
    a, off, _ = synth.make_corpus("markov_2mb", seed=6, m=12, max_len=20000)
    b = np.ascontiguousarray(a ^ np.uint8(0x5A))
    c = np.ascontiguousarray(np.roll(a, 777))
    want = {name: O.intergrams(x, off, N, K, Z, base_n=BASE) for name, x in (("a", a), ("b", b), ("c", c))}
    host = a.copy()
    with B.Plan(host, off, n=N, k=K, candidates=Z, base_n=BASE, host_input=True, graph=graph) as pl:
        order = []
        got = job(pl)
        order.append(("a", got))
        for name, x in (("b", b), ("c", c), ("a", None), ("b", b)):
            pl.prefetch(x)                     # None: the plan's own host buffer (a)
            with pytest.raises(B.IntergramsError) as ei:
                pl.prefetch(x)                 # one pending prefetch at a time
            assert ei.value.status == IG_ESTATE
            pl.rewind()
            order.append((name, job(pl)))
        host[:] = c                            # a plain rewind re-reads the plan's buffer
        pl.rewind()
        order.append(("c", job(pl)))
    for name, (gk, gc) in order:
        ek, ec = want[name]
        assert np.array_equal(gk, ek) and np.array_equal(gc, ec), name


def test_prefetch_needs_host_input():
    a, off, _ = synth.make_corpus("markov_2mb", seed=6, m=4, max_len=5000)
    d = torch.from_numpy(a).cuda()
    o = torch.from_numpy(off.view(np.int64)).cuda()
    with B.Plan(d, o, n=N, k=K, candidates=Z, base_n=BASE) as pl:
        with pytest.raises(B.IntergramsError) as ei:
            pl.prefetch()
        assert ei.value.status == IG_ESTATE
    with B.Plan(a, off, n=N, k=K, candidates=Z, base_n=BASE, host_input=True) as pl:
        with pytest.raises(ValueError):
            pl.prefetch(a[:-1])
