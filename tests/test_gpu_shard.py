"""Sharded passes through the C ABI (intergrams_pass_scan, _counts_export,
_counts_import, _pass_select; intergrams_shard_assign), and the exhaustive
device checks (IG_F_EXHAUSTIVE_CHECKS).

Two processes share the GPU, each with one byte-balanced shard of the same
corpus (whole sequences); after every pass's scan they sum their exported
counts with one gloo all-reduce on host memory and import the sums. Every
pass's top-k must equal the oracle's run on the whole corpus (Algorithm 3,
Sec. 7; Eq. 1 and Eq. 2 counts of independent sequences add up, Sec. 2), on
both ranks. The processes never wait on each other on the GPU: the only
exchange is the host all-reduce between a pass's scan and its selection."""
import os

import numpy as np
import pytest

torch = pytest.importorskip("torch")

from oracle import oracle as O  # noqa: E402
from paper_2511_14955_gb300 import binding as B  # noqa: E402
from paper_2511_14955_gb300 import synth  # noqa: E402

pytestmark = pytest.mark.gpu
IG_ESTATE = -7


def corpus():
    data, off, _ = synth.make_corpus("malware_8gb", m=23, max_len=150_000, seed=31)
    return data, off


def shard_of(data, off, rank, world):
    shard, _ = B.shard_assign(off, world)
    idx = np.flatnonzero(shard == rank)
    L = np.diff(off.astype(np.int64))[idx]
    sub = np.zeros(len(idx) + 1, np.uint64)
    sub[1:] = np.cumsum(L)
    parts = [data[int(off[i]):int(off[i + 1])] for i in idx]
    return (np.concatenate(parts) if parts else np.zeros(1, np.uint8)), sub


def run_sharded(rank, world, port, mode, out):
    import torch.distributed as dist
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    torch.cuda.set_device(0)
    data, off = corpus()
    d, o = shard_of(data, off, rank, world)
    dd = torch.from_numpy(d).cuda()
    oo = torch.from_numpy(o.view(np.int64)).cuda()
    rows = {}
    with B.Plan(dd, oo, n=6, k=500, candidates=3000, base_n=2, count_mode=mode, sharded=True, checks=True) as pl:
        while (j := pl.pass_scan()) is not None:
            buf = torch.empty(pl.counts_slots(), dtype=torch.int32, device="cuda")
            pl.counts_export(buf)
            torch.cuda.synchronize()
            host = buf.cpu()
            dist.all_reduce(host, op=dist.ReduceOp.SUM)  # the one exchange of the pass
            buf.copy_(host.cuda())
            pl.counts_import(buf)
            assert pl.pass_select() == j
            keys, counts, _ = pl.topk()
            rows[j] = (keys.tobytes(), counts.tolist())
    out[rank] = rows
    dist.destroy_process_group()


@pytest.mark.parametrize("mode", [0, 1])
def test_two_shards_with_one_allreduce_per_pass_match_the_whole_corpus(mode):
    import torch.multiprocessing as mp
    ctx = mp.get_context("spawn")
    mgr = ctx.Manager()
    out = mgr.dict()
    port = 29700 + os.getpid() % 500 + 7 * mode
    procs = [ctx.Process(target=run_sharded, args=(r, 2, port, mode, out)) for r in range(2)]
    for p in procs:
        p.start()
    for p in procs:
        p.join(300)
        assert p.exitcode == 0
    data, off = corpus()
    assert out[0] == out[1]
    for j in range(2, 7):
        ek, ec = O.intergrams(data, off, 6, 500, 3000, base_n=2, count_mode=mode, stop_j=j)
        keys, counts = out[0][j]
        assert counts == ec.tolist(), j
        assert keys == ek.tobytes(), j


def test_one_shard_equals_the_plain_plan_and_checks_pass():
    data, off = corpus()
    d = torch.from_numpy(data).cuda()
    o = torch.from_numpy(off.view(np.int64)).cuda()
    with B.Plan(d, o, n=8, k=400, candidates=2000, base_n=3) as pl:
        pl.run()
        ek, ec, _ = pl.topk()
    with B.Plan(d, o, n=8, k=400, candidates=2000, base_n=3, sharded=True, checks=True) as pl:
        while pl.pass_scan() is not None:
            pl.pass_select()  # nothing exchanged: one shard
        gk, gc, _ = pl.topk()
    assert np.array_equal(gk, ek) and np.array_equal(gc, ec)
    # the device checks on a plain plan, both modes
    for mode in (0, 1):
        with B.Plan(d, o, n=8, k=400, candidates=2000, base_n=3, count_mode=mode, checks=True) as pl:
            pl.run()
            keys, counts, _ = pl.topk()
        want = O.intergrams(data, off, 8, 400, 2000, base_n=3, count_mode=mode)
        assert np.array_equal(keys, want[0]) and np.array_equal(counts, want[1])


def test_checks_catch_a_planted_count():
    """A count planted on the host through the import: a 4-gram counted above
    its 3-gram prefix (the least frequent candidate's row, whether the pass
    counts rows by rank or by byte-order id) ends the pass with IG_ESTATE
    (no device fault)."""
    data, off = corpus()
    d = torch.from_numpy(data).cuda()
    o = torch.from_numpy(off.view(np.int64)).cuda()
    with B.Plan(d, o, n=5, k=500, candidates=500, base_n=3, sharded=True, checks=True) as pl:
        pl.pass_scan()
        pl.pass_select()                        # the base pass, untouched: P^(3)
        keys, counts, _ = pl.topk()             # all of P^(3), by (count desc, bytes asc)
        c_min = int(counts[-1])                 # (imported counts are not held to the shard's m)
        rank = len(counts) - 1                  # its counter row if the next pass counts by rank
        ident = sorted(bytes(k) for k in keys).index(bytes(keys[-1]))  # ... or by byte-order id
        pl.pass_scan()
        buf = torch.empty(pl.counts_slots(), dtype=torch.int32, device="cuda")
        pl.counts_export(buf)
        for row in {rank, ident}:               # a 4-gram of that 3-gram above the 3-gram's count
            buf[row * 256] = c_min + 1
        pl.counts_import(buf)
        with pytest.raises(B.IntergramsError) as ei:
            pl.pass_select()
        assert ei.value.status == IG_ESTATE


def test_split_pass_on_16_bit_counters_and_dna():
    """The split pass (scan, export, import, select) on plans whose counters
    are 16-bit (not sharded: exported widened to 32 bits, imported narrowed
    back) and on 2-bit DNA with chain passes: the same rows as the plain
    plan."""
    cases = [(corpus(), dict(n=8, k=300, candidates=1200, base_n=3, symbol_bits=8)),
             (synth.make_corpus("genomic_5gbp", m=4, max_len=40_000, seed=33)[:2],
              dict(n=40, k=200, candidates=800, base_n=10, symbol_bits=2))]
    for (data, off), p in cases:
        d = torch.from_numpy(np.ascontiguousarray(data)).cuda()
        o = torch.from_numpy(off.view(np.int64).copy()).cuda()
        with B.Plan(d, o, **p) as pl:
            pl.run()
            ek, ec, _ = pl.topk()
        for mode_flags in (dict(), dict(sharded=True, checks=True)):
            with B.Plan(d, o, **p, **mode_flags) as pl:
                while pl.pass_scan() is not None:
                    buf = torch.empty(pl.counts_slots(), dtype=torch.int32, device="cuda")
                    pl.counts_export(buf)
                    pl.counts_import(buf.clone())
                    pl.pass_select()
                gk, gc, _ = pl.topk()
            assert np.array_equal(gk, ek) and np.array_equal(gc, ec), (p, mode_flags)


def test_split_pass_calls_out_of_order_are_refused():
    data, off = corpus()
    d = torch.from_numpy(data).cuda()
    o = torch.from_numpy(off.view(np.int64)).cuda()
    buf = torch.empty(1 << 24, dtype=torch.int32, device="cuda")
    with B.Plan(d, o, n=5, k=100, candidates=400, base_n=3) as pl:
        with pytest.raises(B.IntergramsError) as ei:
            pl.counts_export(buf)
        assert ei.value.status == IG_ESTATE
        with pytest.raises(B.IntergramsError) as ei:
            pl.pass_select()
        assert ei.value.status == IG_ESTATE
        pl.pass_scan()
        with pytest.raises(B.IntergramsError) as ei:
            pl.pass_scan()                       # the first scan waits for its selection
        assert ei.value.status == IG_ESTATE
        with pytest.raises(B.IntergramsError) as ei:
            pl.step()                            # so does a whole pass
        assert ei.value.status == IG_ESTATE
        with pytest.raises(B.IntergramsError) as ei:
            pl.counts_import(buf[:5])            # wrong length
        assert ei.value.status == -1
        pl.pass_select()
    with B.Plan(d, o, n=5, k=100, candidates=400, base_n=3, graph=True) as pl:
        with pytest.raises(B.IntergramsError) as ei:
            pl.pass_scan()                       # graph plans run whole jobs
        assert ei.value.status == IG_ESTATE
