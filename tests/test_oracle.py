"""Pins for the CPU oracle (no GPU).

The oracle is checked against things other than itself:
  * brute force (plain Python dictionaries) on tiny corpora, Eq. 1 and Eq. 2,
    for the exhaustive count and for Algorithm 3 with small Z (a selection
    tie order reversed, one candidate too many, or prefixes taken from the
    wrong end each fail it on nearly every seed);
  * closed forms: de Bruijn sequences (every n-gram exactly once, so the
    top-k is the k smallest n-grams in byte order - this pins tie-breaking),
    all-zero sequences, periodic sequences;
  * the Lemma 1 window identity (Sec. 8) under Eq. 1;
  * the special cases in which Algorithm 3 must equal the exhaustive count;
  * the example trie of Fig. 4 (tests/golden/fig4_trie_keys.json).
"""
import itertools
import json
import os
from collections import Counter

import numpy as np
import pytest

from oracle import oracle as O

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")


def corpus(seqs):
    """(data, offsets) from a list of byte strings / code lists."""
    lens = [len(s) for s in seqs]
    off = np.zeros(len(seqs) + 1, np.uint64)
    off[1:] = np.cumsum(lens) if seqs else []
    data = np.concatenate([np.asarray(list(s), np.uint8) for s in seqs]) if sum(lens) else np.zeros(0, np.uint8)
    return data, off


def brute_counts(seqs, n, mode):
    c = Counter()
    for s in seqs:
        grams = [tuple(s[p:p + n]) for p in range(len(s) - n + 1)]
        if mode == O.EQ2_ONCE_PER_SEQUENCE:
            grams = set(grams)
        c.update(grams)
    return c


def brute_top(seqs, n, k, mode):
    c = brute_counts(seqs, n, mode)
    items = sorted(c.items(), key=lambda kv: (-kv[1], kv[0]))[:k]
    return [list(g) for g, _ in items], [v for _, v in items]


def random_seqs(rng, m, maxlen, sigma):
    return [list(rng.integers(0, sigma, size=int(rng.integers(0, maxlen + 1)))) for _ in range(m)]


@pytest.mark.parametrize("seed", range(40))
def test_exhaustive_matches_brute_force(seed):
    rng = np.random.default_rng(seed)
    sigma = [2, 3, 4, 256][seed % 4]
    seqs = random_seqs(rng, int(rng.integers(1, 9)), 64, sigma)
    data, off = corpus(seqs)
    for n in range(1, 7):
        for mode in (O.EQ2_ONCE_PER_SEQUENCE, O.EQ1_EVERY_OCCURRENCE):
            k = int(rng.integers(1, 50))
            keys, counts = O.exhaustive(data, off, n, k, mode)
            bk, bc = brute_top(seqs, n, k, mode)
            assert keys.tolist() == bk
            assert counts.tolist() == bc


def brute_intergrams(seqs, n, k, Z, base_n, mode):
    """Algorithm 3 restated with Python dictionaries: exact base_n-gram counts,
    then for j = base_n+1 .. n the j-grams whose (j-1)-prefix is among the
    previous pass's top-Z, counted exactly; the top-k of the last pass. Every
    selection orders by count descending, then symbols ascending."""
    b = min(base_n, n)

    def select(c, t):
        return [g for g, _ in sorted(c.items(), key=lambda kv: (-kv[1], kv[0]))[:t]]

    counts = brute_counts(seqs, b, mode)
    for j in range(b + 1, n + 1):
        kept = set(select(counts, Z))
        counts = {g: v for g, v in brute_counts(seqs, j, mode).items() if g[:-1] in kept}
    items = sorted(counts.items(), key=lambda kv: (-kv[1], kv[0]))[:k]
    return [list(g) for g, _ in items], [v for _, v in items]


@pytest.mark.parametrize("seed", range(40))
def test_intergrams_matches_brute_force(seed):
    """Algorithm 3 on tiny corpora with small Z (so the filter removes
    prefixes and ties decide membership), every base length, both modes."""
    rng = np.random.default_rng(1000 + seed)
    sigma = [2, 3, 4, 256][seed % 4]
    seqs = random_seqs(rng, int(rng.integers(1, 9)), 80, sigma)
    data, off = corpus(seqs)
    for n in (2, 3, 5, 6):
        for base in (1, 2, 3):
            for mode in (O.EQ2_ONCE_PER_SEQUENCE, O.EQ1_EVERY_OCCURRENCE):
                Z = int(rng.integers(1, 12))
                k = int(rng.integers(1, Z + 1))
                keys, counts = O.intergrams(data, off, n, k, Z, base_n=base, count_mode=mode)
                bk, bc = brute_intergrams(seqs, n, k, Z, base, mode)
                assert keys.tolist() == bk and counts.tolist() == bc, (n, base, mode, Z, k)
                if sigma == 4:  # the same corpus packed 2 bits per base
                    pk, pc = O.intergrams(_pack_by_hand([c for q in seqs for c in q]), off, n, k, Z,
                                          base_n=base, count_mode=mode, symbol_bits=2)
                    assert pk.tolist() == bk and pc.tolist() == bc, (n, base, mode, Z, k, "2-bit")


def _pack_by_hand(codes):
    out = bytearray((len(codes) + 3) // 4)
    for g, c in enumerate(codes):
        out[g // 4] |= (int(c) & 3) << (6 - 2 * (g % 4))
    return np.frombuffer(bytes(out), np.uint8) if out else np.zeros(0, np.uint8)


@pytest.mark.parametrize("seed", range(12))
def test_two_bit_input_matches_brute_force(seed):
    """2-bit packed input, sequences at arbitrary base offsets."""
    rng = np.random.default_rng(100 + seed)
    seqs = random_seqs(rng, int(rng.integers(1, 7)), 70, 4)
    flat = [c for s in seqs for c in s]
    data = _pack_by_hand(flat)
    off = np.zeros(len(seqs) + 1, np.uint64)
    off[1:] = np.cumsum([len(s) for s in seqs])
    for n in (1, 2, 5, 9):
        for mode in (0, 1):
            keys, counts = O.exhaustive(data, off, n, 30, mode, symbol_bits=2)
            bk, bc = brute_top(seqs, n, 30, mode)
            assert keys.tolist() == bk and counts.tolist() == bc


def de_bruijn(sigma, n):
    """de Bruijn sequence B(sigma, n) by the Fredricksen-Kessler-Maiorana
    concatenation of Lyndon words (textbook algorithm)."""
    a = [0] * (sigma * n)
    seq = []

    def db(t, p):
        if t > n:
            if n % p == 0:
                seq.extend(a[1:p + 1])
        else:
            a[t] = a[t - p]
            db(t + 1, p)
            for j in range(a[t - p] + 1, sigma):
                a[t] = j
                db(t + 1, t)

    db(1, 1)
    return seq


@pytest.mark.parametrize("sigma,n", [(2, 5), (3, 4), (4, 3), (16, 2)])
def test_de_bruijn_closed_form(sigma, n):
    cyc = de_bruijn(sigma, n)
    assert len(cyc) == sigma ** n
    lin = cyc + cyc[:n - 1]           # every n-gram appears exactly once
    data, off = corpus([lin])
    k = min(37, sigma ** n)
    keys, counts = O.exhaustive(data, off, n, sigma ** n + 5, O.EQ1_EVERY_OCCURRENCE)
    assert len(keys) == sigma ** n
    assert set(counts.tolist()) == {1}
    # all counts tie, so the order is the byte order of the n-grams
    expect = [list(t) for t in itertools.product(range(sigma), repeat=n)]
    assert keys.tolist() == expect
    keys_k, _ = O.exhaustive(data, off, n, k, O.EQ2_ONCE_PER_SEQUENCE)
    assert keys_k.tolist() == expect[:k]


def test_zero_runs_closed_form():
    L, m, n = 1000, 7, 5
    seqs = [[0] * (L + 3 * i) for i in range(m)] + [[0] * 3]   # one sequence shorter than n
    data, off = corpus(seqs)
    keys, counts = O.exhaustive(data, off, n, 10, O.EQ1_EVERY_OCCURRENCE)
    assert keys.tolist() == [[0] * n]
    assert counts.tolist() == [sum(L + 3 * i - n + 1 for i in range(m))]
    keys, counts = O.exhaustive(data, off, n, 10, O.EQ2_ONCE_PER_SEQUENCE)
    assert counts.tolist() == [m]


def test_periodic_closed_form():
    r = 50
    s = list(b"abc") * r
    data, off = corpus([s, s])
    keys, counts = O.exhaustive(data, off, 3, 10, O.EQ1_EVERY_OCCURRENCE)
    # abc occurs r times, bca and cab r-1 times, per copy
    assert [bytes(k) for k in keys] == [b"abc", b"bca", b"cab"]
    assert counts.tolist() == [2 * r, 2 * (r - 1), 2 * (r - 1)]


def test_empty_and_short_inputs():
    for seqs in ([], [[]], [[1, 2]], [[], [3], [4, 5]]):
        data, off = corpus(seqs)
        keys, counts = O.exhaustive(data, off, 3, 5)
        assert len(keys) == 0 and len(counts) == 0
        keys, counts = O.intergrams(data, off, 4, 5, 8, base_n=1)
        assert len(keys) == 0


def _markov(seed, m, lo, hi):
    from paper_2511_14955_gb300 import synth
    w = synth.WORKLOADS["markov_2mb"]
    L = np.random.default_rng(seed).integers(lo, hi, size=m).astype(np.uint64)
    off = synth.offsets_from_lengths(L)
    return synth.fill(w.model, seed, off, 8), off


@pytest.mark.parametrize("mode", [0, 1])
def test_sum_invariants(mode):
    data, off = _markov(3, 9, 50, 400)
    seqs = [data[int(off[i]):int(off[i + 1])] for i in range(len(off) - 1)]
    big = 10 ** 6
    keys, counts = O.exhaustive(data, off, 1, big, mode)
    if mode == O.EQ1_EVERY_OCCURRENCE:
        assert int(counts.sum()) == int(off[-1])                         # I1
        for j in (2, 3, 7):
            _, cj = O.exhaustive(data, off, j, big, mode)
            assert int(cj.sum()) == sum(max(0, len(s) - j + 1) for s in seqs)
    else:
        assert int(counts.sum()) == sum(len(set(s.tolist())) for s in seqs)   # I1'
        assert int(counts.max()) <= len(seqs)


@pytest.mark.parametrize("mode", [0, 1])
def test_prefix_monotonicity(mode):
    """I2: no j-gram outnumbers its (j-1)-gram prefix."""
    data, off = _markov(4, 6, 100, 600)
    big = 10 ** 6
    prev = None
    for j in range(1, 6):
        keys, counts = O.exhaustive(data, off, j, big, mode)
        table = {bytes(k): int(c) for k, c in zip(keys, counts)}
        if prev is not None:
            for g, c in table.items():
                assert c <= prev[g[:-1]]
        prev = table


def _distinct(data, off, j):
    keys, _ = O.exhaustive(data, off, j, 10 ** 7, 1)
    return len(keys)


@pytest.mark.parametrize("mode", [0, 1])
def test_intergrams_equals_exhaustive_when_all_prefixes_kept(mode):
    """Special case: Z >= #distinct (j-1)-grams at every level -> IG == EXH."""
    data, off = _markov(5, 8, 100, 700)
    n = 5
    Z = max(_distinct(data, off, j) for j in range(1, n))
    for base in (1, 2, 3):
        ik, ic = O.intergrams(data, off, n, 60, Z, base_n=base, count_mode=mode)
        ek, ec = O.exhaustive(data, off, n, 60, mode)
        assert ik.tolist() == ek.tolist() and ic.tolist() == ec.tolist()
    # n <= base_n: the dense pass alone is the exact answer
    ik, ic = O.intergrams(data, off, 2, 60, 3, base_n=3, count_mode=mode)
    ek, ec = O.exhaustive(data, off, 2, 60, mode)
    assert ik.tolist() == ek.tolist() and ic.tolist() == ec.tolist()


@pytest.mark.parametrize("mode", [0, 1])
def test_intergrams_counts_are_exact_and_filtered(mode):
    """I3: every IG count equals the exhaustive count of that n-gram.
    I4: the IG answer is the exact top-k among n-grams whose prefix is in
    P^(n-1), where P^(n-1) is the top-Z of the previous pass."""
    data, off = _markov(6, 10, 200, 900)
    n, Z, k = 5, 40, 25
    ik, ic = O.intergrams(data, off, n, k, Z, base_n=2, count_mode=mode)
    allk, allc = O.exhaustive(data, off, n, 10 ** 7, mode)
    exact = {bytes(a): int(b) for a, b in zip(allk, allc)}
    for key, c in zip(ik, ic):
        assert exact[bytes(key)] == int(c)
    pk, _ = O.intergrams(data, off, n, Z, Z, base_n=2, count_mode=mode, stop_j=n - 1)
    P = {bytes(p) for p in pk}
    assert len(P) == Z
    filt = sorted(((g, c) for g, c in exact.items() if g[:-1] in P), key=lambda t: (-t[1], t[0]))[:k]
    assert [bytes(x) for x in ik] == [g for g, _ in filt]
    assert ic.tolist() == [c for _, c in filt]
    # I7: sorted by (count desc, bytes asc), no duplicates
    pairs = [(-int(c), bytes(x)) for x, c in zip(ik, ic)]
    assert pairs == sorted(pairs) and len(set(pairs)) == len(pairs)


def test_lemma1_window_identity():
    """Lemma 1 (Sec. 8) under Eq. 1: extending each window of a kept
    (j-1)-gram by one symbol yields a j-window, except the last (j-1)-window
    of each sequence. So the windows counted in pass j equal the summed
    counts of P^(j-1) minus the sequences whose last (j-1)-gram is in P^(j-1)."""
    data, off = _markov(7, 12, 20, 500)
    seqs = [bytes(data[int(off[i]):int(off[i + 1])]) for i in range(len(off) - 1)]
    Z = 30
    for base, j in [(1, 2), (1, 4), (2, 3), (3, 6)]:
        pk, pc = O.intergrams(data, off, j, Z, Z, base_n=base, count_mode=1, stop_j=j - 1)
        P = {bytes(x) for x in pk}
        _, _, surv = O.intergrams(data, off, j, 5, Z, base_n=base, count_mode=1, stop_j=j,
                                  want_survivors=True)
        ends = sum(1 for s in seqs if len(s) >= j - 1 and s[len(s) - (j - 1):] in P)
        assert surv == int(pc.sum()) - ends


def test_fig4_trie_example():
    """The example trie of Fig. 4: only 4-grams whose 3-byte prefix is one of
    its six keys survive the candidate pass."""
    g = json.load(open(os.path.join(GOLDEN, "fig4_trie_keys.json")))
    keys = [bytes.fromhex(h) for h in g["keys_hex"]]
    seqs = [list(kk) for kk in keys for _ in range(5)]
    probes = [bytes.fromhex(h) for h in g["lookups"]] + [bytes.fromhex("010000")]
    for p in probes:
        seqs.append(list(p + b"\x01"))
    data, off = corpus(seqs)
    pk, pc = O.intergrams(data, off, 4, 6, 6, base_n=3, count_mode=0, stop_j=3)
    assert {bytes(x) for x in pk} == set(keys)
    for h, inside in g["lookups"].items():
        assert (bytes.fromhex(h) in {bytes(x) for x in pk}) == inside
    ik, ic = O.intergrams(data, off, 4, 50, 6, base_n=3, count_mode=0)
    expect = sorted(p + b"\x01" for p in probes if p in set(keys))
    assert [bytes(x) for x in ik] == expect and set(ic.tolist()) == {1}


def test_repeatable():
    data, off = _markov(8, 5, 300, 800)
    a = O.intergrams(data, off, 6, 50, 64, base_n=2)
    b = O.intergrams(data, off, 6, 50, 64, base_n=2)
    assert a[0].tolist() == b[0].tolist() and a[1].tolist() == b[1].tolist()


@pytest.mark.parametrize("mode", [0, 1])
@pytest.mark.parametrize("bits", [8, 2])
def test_count_keys_matches_exhaustive(mode, bits):
    """Exact counts of chosen n-grams agree with the exhaustive count (and
    absent keys count zero)."""
    rng = np.random.default_rng(40 + mode + bits)
    sigma = 4 if bits == 2 else 6
    seqs = random_seqs(rng, 7, 300, sigma)
    flat = [c for s in seqs for c in s]
    data = _pack_by_hand(flat) if bits == 2 else np.asarray(flat, np.uint8)
    off = np.zeros(len(seqs) + 1, np.uint64)
    off[1:] = np.cumsum([len(s) for s in seqs])
    for n in (1, 3, 9):
        ek, ec = O.exhaustive(data, off, n, 10 ** 6, mode, symbol_bits=bits)
        pick = rng.choice(len(ek), size=min(25, len(ek)), replace=False)
        keys = np.concatenate([ek[pick], np.full((1, n), sigma - 1 if n > 3 else 0, np.uint8)])
        got = O.count_keys(data, off, keys, mode, symbol_bits=bits)
        table = {bytes(k): int(c) for k, c in zip(ek, ec)}
        assert got.tolist() == [table.get(bytes(k), 0) for k in keys]


@pytest.mark.parametrize("seed", range(10))
def test_features_match_brute_force(seed):
    """Fig. 1's Boolean matrix: row i lists, ascending, the features whose
    n-gram occurs in sequence i (sets of n-grams by brute force)."""
    rng = np.random.default_rng(300 + seed)
    sigma = [2, 3, 5, 256][seed % 4]
    seqs = random_seqs(rng, int(rng.integers(1, 12)), 80, sigma)
    data, off = corpus(seqs)
    for n in (1, 2, 4):
        allg = sorted(brute_counts(seqs, n, O.EQ2_ONCE_PER_SEQUENCE))
        if not allg:
            continue
        pick = rng.choice(len(allg), size=min(len(allg), 1 + int(rng.integers(0, 30))), replace=False)
        keys = np.array([allg[i] for i in pick], np.uint8).reshape(-1, n)
        row_ptr, cols = O.features(data, off, keys)
        assert row_ptr[0] == 0 and row_ptr[-1] == len(cols)
        for i, s in enumerate(seqs):
            present = {tuple(s[p:p + n]) for p in range(len(s) - n + 1)}
            want = [f for f in range(len(keys)) if tuple(keys[f]) in present]
            assert cols[row_ptr[i]:row_ptr[i + 1]].tolist() == want


@pytest.mark.parametrize("bits", [8, 2])
def test_feature_column_sums_are_eq2_counts(bits):
    """Summing the matrix over sequences gives each feature's Eq. 2 count
    (its number of sequences), here for the exhaustive top-k."""
    rng = np.random.default_rng(77 + bits)
    sigma = 4 if bits == 2 else 7
    seqs = random_seqs(rng, 9, 400, sigma)
    flat = [c for s in seqs for c in s]
    data = _pack_by_hand(flat) if bits == 2 else np.asarray(flat, np.uint8)
    off = np.zeros(len(seqs) + 1, np.uint64)
    off[1:] = np.cumsum([len(s) for s in seqs])
    for n in (2, 5):
        keys, counts = O.exhaustive(data, off, n, 60, O.EQ2_ONCE_PER_SEQUENCE, symbol_bits=bits)
        row_ptr, cols = O.features(data, off, keys, symbol_bits=bits)
        assert np.bincount(cols, minlength=len(keys)).tolist() == counts.tolist()
        assert all(np.all(np.diff(cols[row_ptr[i]:row_ptr[i + 1]].astype(np.int64)) > 0) for i in range(len(seqs)))


# --------------------------------------------------------------- one pass alone

@pytest.mark.parametrize("seed", range(12))
def test_count_pass_matches_brute_force(seed):
    """One counting step of Algorithm 3 with a given prefix set equals a
    dictionary count of the j-grams whose (j-1)-prefix is in the set."""
    rng = np.random.default_rng(1000 + seed)
    sigma = [2, 4, 256][seed % 3]
    seqs = random_seqs(rng, int(rng.integers(1, 7)), 40, sigma)
    data, off = corpus(seqs)
    mode = seed % 2
    j = int(rng.integers(2, 5))
    prev = sorted(brute_counts(seqs, j - 1, mode))
    keep = [g for g in prev if rng.random() < 0.5]
    pre = np.array(keep, np.uint8).reshape(len(keep), j - 1)
    keys, counts = O.count_pass(data, off, j, pre, count_mode=mode)
    want = {g: c for g, c in brute_counts(seqs, j, mode).items() if g[:-1] in set(keep)}
    assert [tuple(r) for r in keys] == sorted(want)            # ascending symbol order
    assert [int(c) for c in counts] == [want[g] for g in sorted(want)]
    # no prefix set: the dense pass over every j-gram
    keys, counts = O.count_pass(data, off, j, None, count_mode=mode)
    want = brute_counts(seqs, j, mode)
    assert [tuple(r) for r in keys] == sorted(want)
    assert [int(c) for c in counts] == [want[g] for g in sorted(want)]


# ------------------------------------------- the oracle over groups of sequences

def _sharded():
    from oracle import sharded
    return sharded


@pytest.mark.parametrize("mode", [0, 1])
@pytest.mark.parametrize("workers", [1, 2, 5])
def test_sharded_equals_single_threaded_oracle(mode, workers):
    """The harness that runs the counting step over groups of whole sequences
    on several cores, sums the counts and selects between passes gives the
    single-threaded oracle's rows after every pass (ties included: Z and k cut
    through runs of equal counts)."""
    S = _sharded()
    rng = np.random.default_rng(7 + workers + 10 * mode)
    seqs = [list(rng.integers(0, 6, size=int(rng.integers(0, 400)))) for _ in range(9)] + [[], [1, 2]]
    data, off = corpus(seqs)
    out = S.intergrams(data, off, 6, 40, 60, base_n=2, count_mode=mode, workers=workers, per_pass=True)
    assert [j for j, _, _ in out] == [2, 3, 4, 5, 6]
    for j, keys, counts in out:
        ek, ec = O.intergrams(data, off, 6, 40, 60, base_n=2, count_mode=mode, stop_j=j)
        assert np.array_equal(keys, ek) and np.array_equal(counts, ec), j


def test_sharded_two_bit_and_long_keys():
    """2-bit input split at sequence starts that fall inside a byte, and keys
    longer than 8 symbols (compared as byte rows)."""
    S = _sharded()
    rng = np.random.default_rng(3)
    codes = [list(rng.integers(0, 4, size=int(rng.integers(5, 300)))) for _ in range(7)]
    flat = [c for s in codes for c in s]
    pad = (-len(flat)) % 4
    f = np.array(flat + [0] * pad, np.uint8).reshape(-1, 4)
    data = ((f[:, 0] << 6) | (f[:, 1] << 4) | (f[:, 2] << 2) | f[:, 3]).astype(np.uint8)
    _, off = corpus(codes)
    for n, base in ((11, 4), (6, 6)):
        ek, ec = O.intergrams(data, off, n, 30, 50, base_n=base, symbol_bits=2)
        gk, gc = S.intergrams(data, off, n, 30, 50, base_n=base, symbol_bits=2, workers=3)
        assert np.array_equal(gk, ek) and np.array_equal(gc, ec)


def test_shard_groups_cover_every_sequence_once():
    S = _sharded()
    off = np.cumsum([0, 5, 0, 100, 1, 1, 7, 0, 300]).astype(np.uint64)
    L = np.diff(off.astype(np.int64))
    for g in (1, 2, 3, 8, 20):
        groups = S.shard_groups(off, g)
        allidx = np.concatenate(groups)
        assert sorted(allidx.tolist()) == list(range(len(L)))
        assert len(groups) <= g
        loads = sorted(int(L[x].sum()) for x in groups)
        assert loads[-1] <= max(int(L.max()), loads[0] + int(L.max()))  # greedy by bytes
