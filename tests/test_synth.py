"""Seeded generators: Philox known answers, determinism, workload shapes."""
import numpy as np
import pytest

from paper_2511_14955_gb300 import synth


def test_philox_known_answers():
    # Known-answer vectors for Philox4x32-10 (Salmon et al., SC 2011; Random123 kat_vectors)
    assert [hex(x) for x in synth.philox4x32_10([0, 0, 0, 0], [0, 0])] == \
        ["0x6627e8d5", "0xe169c58d", "0xbc57ac4c", "0x9b00dbd8"]
    assert [hex(x) for x in synth.philox4x32_10([0xffffffff] * 4, [0xffffffff] * 2)] == \
        ["0x408f276d", "0x41c83b0e", "0xa20bc7c6", "0x6d5451fd"]
    assert [hex(x) for x in synth.philox4x32_10([0x243f6a88, 0x85a308d3, 0x13198a2e, 0x03707344],
                                                [0xa4093822, 0x299f31d0])] == \
        ["0xd16cfe09", "0x94fdcceb", "0x5001e420", "0x24126ea1"]


def test_deterministic_and_thread_independent():
    a = synth.make_corpus("markov_2mb", seed=3, threads=1)
    b = synth.make_corpus("markov_2mb", seed=3, threads=7)
    assert np.array_equal(a[0], b[0]) and np.array_equal(a[1], b[1])
    c = synth.make_corpus("markov_2mb", seed=4)
    assert not np.array_equal(a[0][:1000], c[0][:1000])


def test_markov_2mb_shape():
    data, off, bits = synth.make_corpus("markov_2mb")
    L = np.diff(off)
    assert bits == 8 and len(L) == 64 and L.min() >= 4096 and L.max() <= 65536
    assert 1.0e6 < off[-1] < 3.5e6
    # about 5% of 4 KiB blocks are zero runs
    blocks = [data[int(off[i]) + b: int(off[i]) + b + 4096] for i in range(64)
              for b in range(0, int(L[i]) - 4095, 4096)]
    zero = np.mean([not blk.any() for blk in blocks])
    assert 0.02 < zero < 0.09


def test_lognormal_lengths():
    w = synth.WORKLOADS["malware_8gb"]
    L = synth.lengths_for(w, seed=1)
    assert len(L) == 20000 and L.max() <= 8 << 20
    med = float(np.median(L))
    assert 0.9 * 256 * 1024 < med < 1.1 * 256 * 1024
    assert 7.0e9 < L.sum() < 9.5e9


def test_dna_packing_roundtrip():
    data, off, bits = synth.make_corpus("genomic_5gbp", m=3, max_len=10001)
    assert bits == 2
    codes = synth.unpack_2bit(data, int(off[-1]))
    assert codes.max() <= 3
    assert np.array_equal(synth.pack_2bit(codes), data)


def test_planted_motifs_repeat_across_sequences():
    data, off, _ = synth.make_corpus("largen_6gb", m=40, max_len=65536)
    # a uniform background has almost no repeated 32-byte windows; planted
    # motifs make many
    s = bytes(data[: int(off[-1])])
    grams = [s[p:p + 32] for p in range(0, len(s) - 32, 16)]
    assert len(grams) - len(set(grams)) > 100
