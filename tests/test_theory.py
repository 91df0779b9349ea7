"""Pins for the Sec. 8 recall calculator (no GPU).

Each statement is checked against direct computation, not against itself:
  * Lemma 3's integral bounds against the partial sums M_x;
  * Theorem 1 (1) and (3) against the exact worst case of a Zipf
    distribution (the found (n+1)-grams are the least frequent ones whose
    mass reaches beta'), by direct summation over every rank;
  * Lemma 1 against the exhaustive Eq. 1 counts of a corpus (oracle);
  * Lemma 2 against multinomial draws of a Zipf law;
  * the Zipf fit against exact power laws.
"""
import math

import numpy as np
import pytest

from oracle import oracle as O
from paper_2511_14955_gb300 import synth, theory as T


def zipf_p(D, a):
    p = np.arange(1, D + 1, dtype=np.float64) ** -a
    return p / p.sum()


def worst_case(D, a, bp, k):
    """Exact (u, share of the top-k mass found) when the found items are the
    tail of Zipf(a) over D items whose mass first reaches bp."""
    p = zipf_p(D, a)
    tail = np.cumsum(p[::-1])[::-1]
    u = int(np.nonzero(tail >= bp - 1e-12)[0].max()) + 1
    if u > k:
        return u, 0.0
    return u, float((p[:k].sum() - p[:u - 1].sum()) / p[:k].sum())


@pytest.mark.parametrize("a", [0.3, 0.7, 1.0, 1.3, 2.5])
def test_integral_bounds_hold(a):
    for x in (1, 2, 3, 10, 1000, 100000):
        M = float(np.sum(np.arange(1, x + 1, dtype=np.float64) ** -a))
        lo, hi = T.zipf_mass_bounds(x, a)
        assert lo <= M * (1 + 1e-12) and M <= hi * (1 + 1e-12), (x, a, lo, M, hi)


GRID = [(D, a, bp, k) for D in (1000, 20000, 200000) for a in (0.3, 0.7, 0.9, 1.1, 1.5, 2.0, 3.0)
        for bp in (0.05, 0.3, 0.6, 0.9, 0.99, 0.999, 1.0) for k in (1, 10, 100, 999)]


def test_theorem1_bounds_hold_in_the_worst_case():
    for D, a, bp, k in GRID:
        u, frac = worst_case(D, a, bp, k)
        assert u <= T.u_bound(D, a, bp) * (1 + 1e-9), (D, a, bp, k, u)
        assert frac >= T.recall_mass_bound(D, a, bp, k) - 1e-12, (D, a, bp, k, frac)


def test_theorem1_printed_forms_are_off_by_one():
    """The reading taken for Theorem 1: its printed u bound (one less) and
    recall numerator (one less) are exceeded by the exact worst case, e.g.
    all of the mass found (beta' = 1) gives a 'bound' above 1."""
    a, k, D = 0.5, 100, 20000
    printed = 1 - ((D ** (1 - a) - a) * 0 - a) / ((k + 1) ** (1 - a) - 1)
    assert printed > 1.0 >= T.recall_mass_bound(D, a, 1.0, k)
    misses_u = 0
    for D, a, bp, k in GRID:
        u, _ = worst_case(D, a, bp, k)
        b = (D ** (1 - a) - a) * (1 - bp) + 1
        if b > 0 and u > b ** (1 / (1 - a)) - 1 + 1e-9:
            misses_u += 1
    assert misses_u > 0


def test_theorem1_limits():
    # nearly all mass kept, a < 1 and a large k: the bound approaches 1
    assert T.recall_mass_bound(10 ** 6, 0.8, 0.9999, 10 ** 5) > 0.97
    # for a > 1 the Lemma 3 lower bound of M_k caps it below 2 - a
    assert T.recall_mass_bound(10 ** 6, 1.5, 1.0, 10 ** 5) < 0.5
    # nothing kept: nothing is promised
    assert T.recall_mass_bound(10 ** 6, 0.8, 0.0, 1000) < 0
    # a > 1 and a small kept share: every rank satisfies (1)
    assert T.u_bound(1000, 3.0, 0.1) == 1000.0
    with pytest.raises(ValueError):
        T.u_bound(100, 1.0, 0.5)


def test_lemma1_on_exhaustive_counts():
    """Share of the (n+1)-gram windows prefixed by the top-k' n-grams lies in
    [(c - m) / (N - m), c / (N - m)] (the lemma's proof), so it is >= beta'."""
    data, off, _ = synth.make_corpus("markov_2mb", seed=3, m=12, max_len=6000)
    m = len(off) - 1
    L = np.diff(off.astype(np.int64))
    for n, kp in ((2, 64), (3, 512)):
        kn, cn = O.exhaustive(data, off, n, 1 << 22, count_mode=O.EQ1_EVERY_OCCURRENCE)
        k1, c1 = O.exhaustive(data, off, n + 1, 1 << 22, count_mode=O.EQ1_EVERY_OCCURRENCE)
        N = int(np.maximum(L - n + 1, 0).sum())
        assert int(cn.sum()) == N
        kept = {bytes(r) for r in kn[:kp]}
        c = int(cn[:kp].sum())
        pref = sum(int(cc) for r, cc in zip(k1, c1) if bytes(r[:n]) in kept)
        share = pref / (N - m)
        assert (c - m) / (N - m) <= share <= c / (N - m)
        assert share >= T.beta_prime(c / N, m, N) - 1e-15


def test_lemma2_covers_multinomial_draws():
    """Empirical top-k mass within Delta(delta) of the true top-k mass in at
    least 1 - delta of the draws."""
    rng = np.random.default_rng(7)
    D, a, k, N, delta = 2000, 1.1, 20, 20000, 0.1
    p = zipf_p(D, a)
    true_top = p[:k].sum()
    d = T.concentration_delta(k, D, N, delta)
    trials, miss = 200, 0
    for _ in range(trials):
        c = rng.multinomial(N, p)
        emp = np.sort(c)[::-1][:k].sum() / N
        miss += abs(emp - true_top) > d
    assert miss <= delta * trials
    with pytest.raises(ValueError):
        T.concentration_delta(k, D, N, 0.0)


@pytest.mark.parametrize("a", [0.4, 1.0, 1.7])
def test_fit_recovers_exact_power_law(a):
    counts = 1e9 * np.arange(1, 5001, dtype=np.float64) ** -a
    assert abs(T.fit_zipf_exponent(counts) - a) < 1e-9
    assert abs(T.fit_zipf_exponent(np.concatenate([counts, np.zeros(10)]), ranks=100) - a) < 1e-9


def test_predict_wiring():
    r = T.predict(beta=0.9995, m=10, N=10 ** 7, distinct_n=5000, distinct_next=10 ** 5, a=1.8, k=100,
                  k_prime=400)
    assert math.isclose(r["beta_prime"], 0.9995 - 10 / (10 ** 7 - 10))
    assert r["theorem1"]["recall_mass_bound"] == T.recall_mass_bound(10 ** 5, 1.8, r["beta_prime"], 100)
    assert r["theorem2"]["beta_double_prime"] < r["beta_prime"]
    assert 0 <= r["theorem1"]["clamped"] <= 1
    _, frac = worst_case(10 ** 5, 1.8, r["beta_prime"], 100)
    assert frac >= r["theorem1"]["recall_mass_bound"]
    assert "note" in T.predict(beta=0.5, m=1, N=100, distinct_n=10, distinct_next=10, a=1.0, k=1, k_prime=1)
