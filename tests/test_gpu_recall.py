"""The recall measurement's exact top-k (GPU): a job whose every pass keeps
all of its nonzero n-grams (Z = k = 2^22) counts every n-gram, so it must
equal the oracle's exhaustive count (Eq. 1 / Eq. 2, Sec. 2) row for row, on
the 2 MiB Markov workload at full size; and the Sec. 8 calculator gets
finite inputs from it."""
import math

import numpy as np
import pytest

torch = pytest.importorskip("torch")

from oracle import oracle as O  # noqa: E402
from paper_2511_14955_gb300 import synth  # noqa: E402

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def markov():
    data, off, _ = synth.make_corpus("markov_2mb", seed=1)
    d = torch.from_numpy(data).cuda()
    o = torch.from_numpy(off.view(np.int64)).cuda()
    return data, off, d, o


@pytest.mark.parametrize("mode", [O.EQ2_ONCE_PER_SEQUENCE, O.EQ1_EVERY_OCCURRENCE])
@pytest.mark.parametrize("n", [3, 4])
def test_every_n_gram_job_equals_exhaustive(markov, mode, n):
    import bench
    data, off, d, o = markov
    every = 1 << 22
    gk, gc, kept_all = bench._job_topk(d, o, n=n, k=every, Z=every, base_n=1, count_mode=mode)
    ek, ec = O.exhaustive(data, off, n, every, count_mode=mode)
    assert kept_all and len(ec) < every
    assert np.array_equal(gk, ek) and np.array_equal(gc, ec)


def test_recall_leg_reports_bound(markov):
    import bench
    r = bench.recall_leg(1)
    for name in ("eq2", "eq1"):
        assert r[name]["exact_counted_every_n_gram"] and r[name]["counts_exact_on_common_rows"]
        assert 0.9 <= r[name]["recall_at_k"] <= 1.0
    t = r["eq1"]["theory"]
    assert 0 < t["beta"] <= 1 and t["beta_prime"] < t["beta"]
    assert math.isfinite(t["theorem1"]["recall_mass_bound"]) and 0 <= t["theorem1"]["clamped"] <= 1
