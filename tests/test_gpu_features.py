"""Boolean sequence x feature matrix (paper Sec. 1, Fig. 1) on the GPU against
the CPU oracle's, through the C ABI: bit-exact CSR (row starts and feature
ids), and column sums equal to the Eq. 2 counts of the top-k rows."""
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


def codes(rows, n, bits):
    """Library rows -> symbol codes per row (what the oracle takes)."""
    if bits == 8:
        return rows
    return np.stack([synth.unpack_2bit(r, n) for r in rows]) if len(rows) else np.zeros((0, n), np.uint8)


def check(data, off, *, n, k, Z, base_n, bits=8, mode=0, tuning=None):
    d, o = dev(data, off)
    with B.Plan(d, o, n=n, k=k, candidates=Z, base_n=base_n, symbol_bits=bits, count_mode=mode,
                tuning=tuning) as pl:
        pl.run()
        keys, counts, _ = pl.topk()
        row_ptr, cols = pl.features()
        row_ptr2, cols2 = pl.features()   # the count is kept: same answer
    er, ec = O.features(data, off, codes(keys, n, bits), symbol_bits=bits)
    assert np.array_equal(row_ptr, er)
    assert np.array_equal(cols, ec)
    assert np.array_equal(row_ptr2, row_ptr) and np.array_equal(cols2, cols)
    if mode == O.EQ2_ONCE_PER_SEQUENCE:
        assert np.bincount(cols, minlength=len(keys)).tolist() == counts.tolist()
    return row_ptr, cols


def test_markov_2mb():
    data, off, _ = synth.make_corpus("markov_2mb")
    check(data, off, n=4, k=1024, Z=4096, base_n=1)


@pytest.mark.parametrize("mode", [0, 1])
def test_malware_like_reduced(mode):
    data, off, _ = synth.make_corpus("malware_8gb", m=50, max_len=40 * 1024, seed=3)
    check(data, off, n=8, k=700, Z=2800, base_n=3, mode=mode)


def test_dna_reduced():
    data, off, bits = synth.make_corpus("genomic_5gbp", m=4, max_len=30011, seed=2)
    check(data, off, n=21, k=300, Z=1200, base_n=10, bits=bits)


def test_small_tiles_and_edge_sequences():
    seqs = [b"", b"ab", b"abcabcabc" * 50, b"\x00" * 3000, bytes(range(256)) * 3, b"xyz"]
    off = np.zeros(len(seqs) + 1, np.uint64)
    off[1:] = np.cumsum([len(s) for s in seqs])
    data = np.frombuffer(b"".join(seqs), np.uint8)
    check(data, off, n=3, k=40, Z=160, base_n=1, tuning=dict(threads=256, words_per_thread=1, smem_set_log2=8))


def test_errors():
    data, off, _ = synth.make_corpus("markov_2mb", m=4)
    d, o = dev(data, off)
    with B.Plan(d, o, n=4, k=16, candidates=64, base_n=1) as pl:
        with pytest.raises(B.IntergramsError) as ei:
            pl.features()                      # no pass has run
        assert ei.value.status == -7
        pl.step()
        with pytest.raises(B.IntergramsError):
            pl.features()                      # passes remain
    with B.Plan(d, o, n=9, k=16, candidates=64, base_n=1) as pl:
        pl.run()
        with pytest.raises(B.IntergramsError) as ei:
            pl.features()                      # 9-byte keys exceed 64 bits
        assert ei.value.status == -1
