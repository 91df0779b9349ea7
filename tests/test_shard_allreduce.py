"""The sharded form of Algorithm 3 on CPU ranks (gloo, world size 2).

Sequences are independent under Eq. 1 and Eq. 2, so a corpus split by
sequences across ranks counts each pass as the sum of the shards' counts.
Each rank counts its shard (the oracle's exhaustive counts), one sum
all-reduce per pass combines them, and every rank then applies the same
deterministic top-Z (count descending, symbols ascending) to the summed
counts of the j-grams whose prefix is in P^(j-1). The test checks that both
ranks select the same P^(j) at every pass and that the final top-k equals
the oracle's Intergrams run on the whole corpus.
"""
import os

import numpy as np
import pytest

torch = pytest.importorskip("torch")
import torch.distributed as dist  # noqa: E402
import torch.multiprocessing as mp  # noqa: E402

SIGMA = 4  # symbols 0..3 stored one per byte, so a j-gram indexes a dense array of 4^j counts


def corpus(m, seed):
    rng = np.random.default_rng(seed)
    P = rng.dirichlet(np.full(SIGMA, 0.4), size=SIGMA)
    seqs = []
    for _ in range(m):
        L = int(rng.integers(0, 400))
        s = np.zeros(L, np.uint8)
        for i in range(1, L):
            s[i] = rng.choice(SIGMA, p=P[s[i - 1]])
        seqs.append(s)
    off = np.zeros(m + 1, np.uint64)
    off[1:] = np.cumsum([len(s) for s in seqs])
    data = np.concatenate(seqs) if sum(len(s) for s in seqs) else np.zeros(0, np.uint8)
    return data, off


def shard(data, off, rank, world):
    idx = list(range(rank, len(off) - 1, world))
    parts = [data[int(off[i]):int(off[i + 1])] for i in idx]
    o = np.zeros(len(idx) + 1, np.uint64)
    o[1:] = np.cumsum([len(p) for p in parts]) if idx else []
    d = np.concatenate(parts) if parts and sum(len(p) for p in parts) else np.zeros(0, np.uint8)
    return d, o


def gram_index(rows):
    j = rows.shape[1]
    return (rows.astype(np.int64) * (SIGMA ** np.arange(j - 1, -1, -1, dtype=np.int64))).sum(axis=1)


def top(counts, allowed, t):
    """Top-t nonzero allowed slots by (count desc, index asc) = (count desc, symbols asc)."""
    idx = np.nonzero((counts > 0) & allowed)[0]
    order = np.lexsort((idx, -counts[idx]))
    return idx[order[:t]]


def _worker(rank, world, port, m, seed, n, k, Z, mode, out):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank), WORLD_SIZE=str(world))
    from oracle import oracle as O
    dist.init_process_group("gloo", rank=rank, world_size=world)
    data, off = corpus(m, seed)
    d, o = shard(data, off, rank, world)
    prev = None
    same = True
    for j in range(1, n + 1):
        local = np.zeros(SIGMA ** j, np.int64)
        if len(o) > 1:
            keys, c = O.exhaustive(d, o, j, SIGMA ** j, count_mode=mode)
            local[gram_index(keys)] = c.astype(np.int64)
        t = torch.from_numpy(local)
        dist.all_reduce(t, op=dist.ReduceOp.SUM)          # the one exchange of the pass
        counts = t.numpy()
        allowed = np.ones(len(counts), bool) if prev is None else np.isin(np.arange(len(counts)) // SIGMA, prev)
        sel = top(counts, allowed, k if j == n else Z)
        # every rank must have selected the same set
        pad = np.full(Z, -1, np.int64)
        pad[:len(sel)] = sel
        g = [torch.zeros(Z, dtype=torch.int64) for _ in range(world)]
        dist.all_gather(g, torch.from_numpy(pad))
        same &= all(torch.equal(g[0], x) for x in g)
        prev = sel
    out[rank] = (same, [int(x) for x in prev], [int(counts[x]) for x in prev])
    dist.destroy_process_group()


@pytest.mark.parametrize("mode", [0, 1])
@pytest.mark.parametrize("m,seed", [(11, 5), (3, 8), (1, 2)])
def test_sharded_passes_equal_single_corpus(mode, m, seed):
    from oracle import oracle as O
    n, k, Z = 5, 12, 40
    ctx = mp.get_context("spawn")
    mgr = ctx.Manager()
    out = mgr.dict()
    port = 29700 + (os.getpid() + 7 * m + mode) % 800
    procs = [ctx.Process(target=_worker, args=(r, 2, port, m, seed, n, k, Z, mode, out)) for r in range(2)]
    for p in procs:
        p.start()
    for p in procs:
        p.join(180)
        assert p.exitcode == 0
    data, off = corpus(m, seed)
    ek, ec = O.intergrams(data, off, n, k, Z, base_n=1, count_mode=mode)
    for r in range(2):
        same, sel, cnt = out[r]
        assert same
        assert sel == [int(x) for x in gram_index(ek)] and cnt == [int(x) for x in ec]
