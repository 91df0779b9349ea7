"""GPU path vs the CPU oracle: bit-exact keys and counts (all integer work).

Every test calls the CUDA library through its C ABI (paper_2511_14955_gb300
.binding) and compares with oracle/ on the same seeded inputs.
"""
import numpy as np
import pytest

torch = pytest.importorskip("torch")

from oracle import oracle as O  # noqa: E402
from paper_2511_14955_gb300 import binding as B  # noqa: E402
from paper_2511_14955_gb300 import synth  # noqa: E402

pytestmark = pytest.mark.gpu


def dev(data, off):
    d = torch.from_numpy(np.array(data, copy=True)).cuda() if len(data) else torch.zeros(1, dtype=torch.uint8).cuda()
    o = torch.from_numpy(np.ascontiguousarray(off).view(np.int64)).cuda()
    return d, o


def oracle_rows(keys, symbol_bits):
    """Oracle symbol codes -> the library's packed row format."""
    if symbol_bits == 8:
        return keys
    return np.stack([synth.pack_2bit(r) for r in keys]) if len(keys) else keys[:, : (keys.shape[1] + 3) // 4]


def dedupe_variants(mode, tuning):
    """Under Eq. 2 a pass dedupes by bit vector when its slot space is small,
    else by the shared-memory set with spill lists: run both unless the
    tuning picks one."""
    tuning = dict(tuning or {})
    if mode != O.EQ2_ONCE_PER_SEQUENCE or "dedupe_bitmap" in tuning:
        return [tuning]
    return [tuning, dict(tuning, dedupe_bitmap=1)]


def check_all_passes(data, off, *, n, k, Z, base_n, mode=0, symbol_bits=8, tuning=None, graph=False):
    b = min(base_n, n)
    expect = {}
    for tun in dedupe_variants(mode, tuning):
        d, o = dev(data, off)
        pl = B.Plan(d, o, n=n, k=k, candidates=Z, base_n=base_n, symbol_bits=symbol_bits, count_mode=mode,
                    tuning=tun, graph=graph)
        seen = []
        while True:
            j = pl.step()
            if j is None:
                break
            seen.append(j)
            gk, gc, gj = pl.topk()
            if j not in expect:
                ek, ec = O.intergrams(data, off, n, k, Z, base_n=base_n, count_mode=mode,
                                      symbol_bits=symbol_bits, stop_j=j)
                surv = None
                if mode == O.EQ1_EVERY_OCCURRENCE:
                    _, _, surv = O.intergrams(data, off, n, 1, Z, base_n=base_n, count_mode=mode,
                                              symbol_bits=symbol_bits, stop_j=j, want_survivors=True)
                expect[j] = (oracle_rows(ek, symbol_bits), ec, surv)
            ek, ec, surv = expect[j]
            assert gj == j
            assert gk.shape == ek.shape, (tun, j, gk.shape, ek.shape)
            assert np.array_equal(gc, ec), f"counts differ at pass {j} ({tun})"
            assert np.array_equal(gk, ek), f"keys differ at pass {j} ({tun})"
            if surv is not None:
                assert pl.stats()["survivors"] == surv
        assert seen == list(range(b, n + 1))
        pl.close()


@pytest.mark.parametrize("mode", [0, 1])
def test_markov_2mb_every_pass(mode):
    """The 2 MiB Markov workload: n = 4, Z = 4096, k = 1024, base 1; top-k after every pass."""
    data, off, _ = synth.make_corpus("markov_2mb")
    check_all_passes(data, off, n=4, k=1024, Z=4096, base_n=1, mode=mode)


@pytest.mark.parametrize("base_n", [1, 3])
def test_malware_like_reduced(base_n):
    """Malware-like byte law (motifs + zero blocks), reduced to 60 sequences of <= 32 KiB, n = 8."""
    data, off, _ = synth.make_corpus("malware_8gb", m=60, max_len=32 * 1024)
    check_all_passes(data, off, n=8, k=512, Z=2048, base_n=base_n)


def test_largen_background_reduced():
    data, off, _ = synth.make_corpus("largen_6gb", m=60, max_len=40000)
    check_all_passes(data, off, n=8, k=300, Z=1500, base_n=2)


@pytest.mark.parametrize("mode", [0, 1])
def test_dna_reduced(mode):
    """2-bit packed DNA at arbitrary base offsets; k-mers up to 32 bases."""
    data, off, bits = synth.make_corpus("genomic_5gbp", m=5, max_len=30011)
    check_all_passes(data, off, n=16, k=400, Z=1600, base_n=8, mode=mode, symbol_bits=2)
    check_all_passes(data, off, n=32, k=50, Z=300, base_n=12, mode=mode, symbol_bits=2)


@pytest.mark.parametrize("tuning", [
    dict(threads=256, words_per_thread=1, smem_set_log2=8, ctas_per_sm=4),   # tiny tiles, heavy spill
    dict(threads=1024, words_per_thread=7, smem_set_log2=14, ctas_per_sm=1),
    dict(threads=512, words_per_thread=3, smem_set_log2=10, table_load_pct=50, hot_log2=6),
    dict(threads=512, words_per_thread=5, smem_set_log2=12, hot_log2=13),
    dict(dense_prefix=1, words_per_thread=3),                                 # probe table in pass base + 1
    dict(dense_prefix=2, threads=512),                                        # dense map in pass base + 1
    dict(dense_prefix=3, hot_log2=7),                                         # window runs + probe table
    dict(dense_prefix=4),                                                     # rank/select in passes base + 1, + 2
    dict(dense_prefix=4, rs_depth=4, words_per_thread=3),                     # four rank/select levels
    dict(dense_prefix=4, rs_depth=1, hot_log2=8),
    dict(words_per_thread=3, smem_set_log2=13, base_words_per_thread=7, base_smem_set_log2=15),  # base knobs
    dict(set_probes=1, smem_set_log2=11),                                     # one-probe set, many spills
    dict(set_probes=8),
    dict(tile_cache_hint=1, tile_buffers=1),                                  # plain tile copies, one buffer
    dict(prefetch_tiles=4),                                                   # tiles prefetched into L2
    dict(spill_dedupe=1, smem_set_log2=10),                                   # spills by hash partition
    dict(spill_min_fill=1, smem_set_log2=10),                                 # spills by bit vector, always
    dict(dense_prefix=4, rs_depth=3, carry_slots=2),                          # carried slots
    dict(chain_from=6),                                                       # no chain passes
    dict(scan_variants=1, dedupe_bitmap=1),                                   # general kernel only
    dict(dedupe_bitmap=1, rs_depth=1),                                        # one-level variant
])
def test_results_do_not_depend_on_tuning(tuning):
    data, off, _ = synth.make_corpus("markov_2mb", seed=2)
    check_all_passes(data, off, n=5, k=700, Z=3000, base_n=2, tuning=tuning)


def test_plans_with_different_shared_memory_coexist():
    """The scan kernels' shared-memory limits belong to the kernels, not to a
    plan: a plan made later with small tiles and sets must leave a live plan
    that needs more shared memory runnable, and both stay bit-exact."""
    data, off, _ = synth.make_corpus("markov_2mb", m=16, seed=12)
    big = dict(threads=1024, words_per_thread=7, smem_set_log2=14, ctas_per_sm=1, dedupe_bitmap=1)
    small = dict(threads=256, words_per_thread=1, smem_set_log2=8, ctas_per_sm=4, dedupe_bitmap=1)
    ek, ec = O.intergrams(data, off, 5, 100, 400, base_n=2)
    d, o = dev(data, off)
    plans = [B.Plan(d, o, n=5, k=100, candidates=400, base_n=2, tuning=t) for t in (big, small)]
    for pl in plans:  # the large plan runs after the small one was made
        pl.run()
        gk, gc, gj = pl.topk()
        assert gj == 5
        assert np.array_equal(gc, ec) and np.array_equal(gk, ek)
    for pl in plans:
        pl.close()


def check_passes(data, off, *, n, k, Z, base_n, js, mode=0, symbol_bits=8, tuning=None):
    """Run every pass; compare with the oracle after the passes in `js`."""
    expect = {}
    for tun in dedupe_variants(mode, tuning):
        d, o = dev(data, off)
        pl = B.Plan(d, o, n=n, k=k, candidates=Z, base_n=base_n, symbol_bits=symbol_bits, count_mode=mode,
                    tuning=tun)
        while True:
            j = pl.step()
            if j is None:
                break
            if j in js:
                gk, gc, gj = pl.topk()
                if j not in expect:
                    ek, ec = O.intergrams(data, off, n, k, Z, base_n=base_n, count_mode=mode,
                                          symbol_bits=symbol_bits, stop_j=j)
                    expect[j] = (oracle_rows(ek, symbol_bits), ec)
                ek, ec = expect[j]
                assert gk.shape == ek.shape, (tun, j, gk.shape, ek.shape)
                assert np.array_equal(gc, ec), f"counts differ at pass {j} ({tun})"
                assert np.array_equal(gk, ek), f"keys differ at pass {j} ({tun})"
        pl.close()


@pytest.mark.parametrize("mode", [0, 1])
def test_long_byte_keys(mode):
    """n = 16 and n = 64 bytes: passes whose (j-1)-gram exceeds 64 bits run from survivor lists."""
    data, off, _ = synth.make_corpus("largen_6gb", m=24, max_len=12000, seed=4)
    check_passes(data, off, n=16, k=200, Z=800, base_n=3, js={3, 8, 9, 10, 11, 16}, mode=mode)
    check_passes(data, off, n=64, k=150, Z=600, base_n=2, js={9, 10, 33, 64}, mode=mode)


def test_long_dna_keys():
    data, off, _ = synth.make_corpus("genomic_5gbp", m=3, max_len=20011, seed=6)
    check_passes(data, off, n=48, k=100, Z=400, base_n=10, js={32, 33, 34, 35, 48}, symbol_bits=2)


@pytest.mark.parametrize("mode", [0, 1])
def test_chain_mode_with_short_keys(mode):
    """Chain passes from pass base+2 on (short keys), against every pass of the oracle."""
    data, off, _ = synth.make_corpus("malware_8gb", m=30, max_len=40000, seed=8)
    check_all_passes(data, off, n=8, k=300, Z=1200, base_n=2, mode=mode, tuning=dict(chain_from=4))


@pytest.mark.parametrize("mode", [0, 1])
def test_chain_passes_after_rank_select_passes(mode):
    """Rank/select passes (counting in byte-order ids) followed by passes run from survivor lists."""
    data, off, _ = synth.make_corpus("malware_8gb", m=30, max_len=40000, seed=12)
    check_all_passes(data, off, n=8, k=300, Z=1200, base_n=2, mode=mode,
                     tuning=dict(chain_from=5, dense_prefix=4, rs_depth=3))


@pytest.mark.parametrize("graph", [False, True])
def test_survivor_lists_grow_and_the_job_replays(graph):
    """Survivor lists far too small for the job: the plan grows them to what
    the passes asked for and replays, so the result is exact (pass by pass
    and as one captured graph, which is captured again for the new lists)."""
    data, off, _ = synth.make_corpus("markov_2mb", m=10, seed=3)
    d, o = dev(data, off)
    ek, ec = O.intergrams(data, off, 6, 10, 4000, base_n=1)
    with B.Plan(d, o, n=6, k=10, candidates=4000, base_n=1, graph=graph,
                tuning=dict(chain_from=3, list_pct=1)) as pl:
        for _ in range(2):
            pl.rewind()
            pl.run()
            keys, counts, _ = pl.topk()
            assert np.array_equal(keys, ek) and np.array_equal(counts, ec)
    with B.Plan(d, o, n=6, k=10, candidates=4000, base_n=1, tuning=dict(chain_from=3, list_pct=1)) as pl:
        for j in range(1, 7):
            assert pl.step() == j
            keys, counts, _ = pl.topk()
            wk, wc = O.intergrams(data, off, 6, 10, 4000, base_n=1, stop_j=j)
            assert np.array_equal(keys, wk) and np.array_equal(counts, wc), j


def test_list_growth_failing_is_reported():
    """No memory for the larger lists (the growth allocation made to fail on
    the host): IG_ETABLE_FULL, the plan refuses further passes, and nothing
    leaks once it is freed."""
    data, off, _ = synth.make_corpus("markov_2mb", m=10, seed=3)
    d, o = dev(data, off)
    live0 = B.test_fail_alloc(0)
    pl = B.Plan(d, o, n=6, k=10, candidates=4000, base_n=1, tuning=dict(chain_from=3, list_pct=1))
    B.test_fail_alloc(1)                 # the next allocation: the first grown list
    try:
        with pytest.raises(B.IntergramsError) as ei:
            pl.run()
        assert ei.value.status == -3
        B.test_fail_alloc(0)
        with pytest.raises(B.IntergramsError) as ei:
            pl.rewind()
            pl.run()
        assert ei.value.status == -7
    finally:
        B.test_fail_alloc(0)
        pl.close()
    assert B.test_fail_alloc(0) == live0


def test_edge_cases():
    rng = np.random.default_rng(0)
    cases = [
        [],                                     # no sequences
        [b""],                                  # one empty sequence
        [b"ab", b"", b"c"],                     # all shorter than n
        [b"\x00" * 5000],                       # one zero run: a single n-gram
        [bytes(rng.integers(0, 2, 3000).astype(np.uint8)) for _ in range(7)],   # binary alphabet
        [b"abcd" * 100, b"abcd" * 3, b"dcba"],  # ties
    ]
    for seqs in cases:
        lens = [len(s) for s in seqs]
        off = np.zeros(len(seqs) + 1, np.uint64)
        off[1:] = np.cumsum(lens) if seqs else []
        data = np.frombuffer(b"".join(seqs), np.uint8) if sum(lens) else np.zeros(0, np.uint8)
        for mode in (0, 1):
            check_all_passes(data, off, n=4, k=5, Z=7, base_n=1, mode=mode)
            check_all_passes(data, off, n=3, k=3, Z=3, base_n=3, mode=mode)   # n == base_n


# registration log forced on, with small chunks (steps of 2048 registrations)
# and a 2^19-slot counter array split into 32 ranges
LOG_ON = dict(log_mode=1, log_chunk_log2=14, log_range_log2=12)


@pytest.mark.parametrize("mode", [0, 1])
def test_registration_log_every_pass(mode):
    """Registrations go to per-range log chunks and are counted range by range after each scan."""
    data, off, _ = synth.make_corpus("malware_8gb", m=40, max_len=64 * 1024, seed=9)
    check_all_passes(data, off, n=8, k=512, Z=2048, base_n=3, mode=mode, tuning=LOG_ON)


def test_registration_log_pool_exhausted():
    """A log of one chunk: once the pool is used up, registrations are counted at once."""
    data, off, _ = synth.make_corpus("malware_8gb", m=40, max_len=64 * 1024, seed=10)
    check_all_passes(data, off, n=6, k=256, Z=2048, base_n=2, tuning=dict(LOG_ON, log_pct=1))


@pytest.mark.parametrize("mode", [0, 1])
def test_registration_log_with_chain_passes(mode):
    data, off, _ = synth.make_corpus("largen_6gb", m=24, max_len=12000, seed=4)
    check_passes(data, off, n=16, k=200, Z=800, base_n=3, js={4, 9, 10, 16}, mode=mode, tuning=LOG_ON)


def test_many_short_sequences_use_32bit_counters():
    """m >= 65536 sequences: Eq. 2 counts may exceed 16 bits, so the counters are 32-bit."""
    rng = np.random.default_rng(17)
    m = 70000
    lens = rng.integers(3, 24, size=m)
    off = np.zeros(m + 1, np.uint64)
    off[1:] = np.cumsum(lens)
    # a small alphabet so that counts go far beyond 65535 for the top n-grams
    data = rng.integers(0, 3, size=int(off[-1])).astype(np.uint8)
    check_all_passes(data, off, n=5, k=40, Z=150, base_n=2)


def test_k_equals_candidates_and_single_candidate():
    data, off, _ = synth.make_corpus("markov_2mb", m=8, seed=5)
    check_all_passes(data, off, n=6, k=64, Z=64, base_n=1)
    check_all_passes(data, off, n=6, k=1, Z=1, base_n=1)


def test_host_input_graph_rewind_and_unaligned():
    data, off, _ = synth.make_corpus("markov_2mb", m=20, seed=9)
    ek, ec = O.intergrams(data, off, 6, 200, 900, base_n=2)
    # host buffers: the library copies them itself
    pl = B.Plan(data, off, n=6, k=200, candidates=900, base_n=2, host_input=True)
    pl.run()
    gk, gc, _ = pl.topk()
    assert np.array_equal(gk, ek) and np.array_equal(gc, ec)
    pl.close()
    # CUDA graph: capture on the first run, replay after rewind
    d, o = dev(data, off)
    pl = B.Plan(d, o, n=6, k=200, candidates=900, base_n=2, graph=True)
    for _ in range(3):
        pl.run()
        gk, gc, _ = pl.topk()
        assert np.array_equal(gk, ek) and np.array_equal(gc, ec)
        pl.rewind()
    pl.close()
    # data pointer not 16-byte aligned
    big = torch.zeros(len(data) + 64, dtype=torch.uint8, device="cuda")
    big[3:3 + len(data)] = torch.from_numpy(data).cuda()
    pl = B.Plan(big[3:3 + len(data)], o, n=6, k=200, candidates=900, base_n=2)
    pl.run()
    gk, gc, _ = pl.topk()
    assert np.array_equal(gk, ek) and np.array_equal(gc, ec)
    pl.close()


def test_timing_events_in_both_launch_modes():
    data, off, _ = synth.make_corpus("markov_2mb", m=12, seed=4)
    d, o = dev(data, off)
    for graph in (False, True):
        pl = B.Plan(d, o, n=5, k=100, candidates=400, base_n=2, graph=graph, timing=True)
        for _ in range(2):
            pl.rewind()
            if graph:
                pl.run()
            else:
                while pl.step() is not None:
                    pass
            scan, pas, kern = pl.timings()
            assert len(scan) == 4 and (scan > 0).all() and (pas >= scan).all() and kern > 0
        pl.close()


def test_autotune_picks_valid_knobs_and_keeps_results():
    data, off, _ = synth.make_corpus("malware_8gb", m=50, max_len=64 * 1024, seed=13)
    d, o = dev(data, off)
    best, ms = B.autotune(d, o, n=7, k=500, candidates=2000, base_n=3, sample_bytes=1 << 20)
    assert best["threads"] in (256, 512, 1024) and best["words_per_thread"] % 2 == 1 and ms > 0
    ek, ec = O.intergrams(data, off, 7, 500, 2000, base_n=3)
    with B.Plan(d, o, n=7, k=500, candidates=2000, base_n=3, autotune=True) as pl:
        pl.run()
        gk, gc, _ = pl.topk()
    assert np.array_equal(gk, ek) and np.array_equal(gc, ec)


def test_repeated_runs_identical():
    data, off, _ = synth.make_corpus("malware_8gb", m=40, max_len=64 * 1024, seed=3)
    d, o = dev(data, off)
    outs = []
    for _ in range(3):
        pl = B.Plan(d, o, n=7, k=800, candidates=3000, base_n=3)
        pl.run()
        outs.append(pl.topk())
        pl.close()
    for x in outs[1:]:
        assert np.array_equal(x[0], outs[0][0]) and np.array_equal(x[1], outs[0][1])


def test_invalid_arguments_rejected():
    data, off, _ = synth.make_corpus("markov_2mb", m=4)
    d, o = dev(data, off)
    bad = [dict(n=0, k=1, candidates=1), dict(n=4, k=10, candidates=5), dict(n=4, k=1, candidates=1 << 24),
           dict(n=4, k=1, candidates=4, base_n=4), dict(n=4, k=1, candidates=4, symbol_bits=4),
           dict(n=4, k=1, candidates=4, count_mode=2)]
    for kw in bad:
        with pytest.raises(B.IntergramsError) as ei:
            B.Plan(d, o, **kw)
        assert ei.value.status == -1
    bad_off = off.copy()
    bad_off[2], bad_off[3] = bad_off[3], bad_off[2]
    with pytest.raises(B.IntergramsError):
        B.Plan(d, dev(data, bad_off)[1], n=4, k=1, candidates=4)


@pytest.mark.parametrize("mode", [O.EQ2_ONCE_PER_SEQUENCE, O.EQ1_EVERY_OCCURRENCE])
def test_maximum_candidate_count(mode):
    """Z = 2^24 - 1, the largest the ABI takes: sigma * Z slots use the whole
    32-bit slot range (the highest slot stays below the empty-entry marker).
    Z covers every prefix of this corpus, so the result is the exhaustive
    top-k (Algorithm 3 with nothing filtered out)."""
    data, off, _ = synth.make_corpus("markov_2mb", seed=9, m=6, max_len=8192)
    d, o = dev(data, off)
    Z = (1 << 24) - 1
    with B.Plan(d, o, n=4, k=1000, candidates=Z, base_n=1, count_mode=mode) as pl:
        pl.run()
        gk, gc, _ = pl.topk()
    ek, ec = O.exhaustive(data, off, 4, 1000, count_mode=mode)
    assert np.array_equal(gk, ek) and np.array_equal(gc, ec)
