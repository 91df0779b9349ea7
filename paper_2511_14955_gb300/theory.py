"""Recall bounds of the intermediate filter under a Zipf model (Sec. 8).

Host-side arithmetic only (no corpus work): given the statistics of a job,
it evaluates what Sec. 8 predicts for the share of the true top-k
(n+1)-grams that a pass keeping the top k' n-grams can still find.

- Lemma 1: the (n+1)-grams prefixed by the kept n-grams hold at least
  beta' = beta - m / (N - m) of all (n+1)-grams, where beta is the kept
  n-grams' share of the N n-grams of the m sequences.
- Lemma 2: with probability at least 1 - delta, the empirical top-k mass is
  within Delta(delta) = 4 sqrt(k^2 ln(2 |D_n| / delta) / (2 N)) of the true one.
- Lemma 3 (appendix): for a != 1, ((x+1)^(1-a) - 1) / (1-a) <= M_x <=
  (x^(1-a) - a) / (1-a), with M_x = sum_{i <= x} i^-a; for a = 1,
  ln(x+1) <= M_x <= ln(x) + 1.
- Theorem 1: if the (n+1)-grams follow Zipf(a) exactly over |D_{n+1}|
  items and the kept prefixes' (n+1)-grams hold beta' of the mass, (1) the
  most frequent one found has true rank at most u, (3) the found part of the
  true top-k holds at least a fraction of the top-k mass.
- Theorem 2: the same with beta'' = beta' - Delta(delta), with probability
  at least 1 - delta.

Readings (the printed forms of Theorem 1 are off by one; the brute-force
Zipf tests show that the printed forms are not bounds in many cases, while
the forms below hold in every case tried):
- (1) the mass above the most frequent found item x_u is M_{u-1} (the
  proof writes M_u), so the bound is u <= (X + 1)^(1/(1-a)) with
  X = (|D_{n+1}|^(1-a) - a)(1 - beta'), not that minus one. When
  X + 1 <= 0 (possible for a > 1) the inequality holds for every u and the
  bound is |D_{n+1}|.
- (3) substituting (1) into 1 - (u^(1-a) - a) / ((k+1)^(1-a) - 1) gives
  the numerator X + 1 - a (the printed numerator drops the 1).
- Both are bounds in the theorem's worst case, where the found
  (n+1)-grams are the least frequent ones whose mass reaches beta'.
A value at or below 0 means the bound says nothing for those statistics;
`recall_mass_bound` reports it unclamped and `clamped` in [0, 1].
"""
from __future__ import annotations

import math

import numpy as np


def zipf_mass_bounds(x: float, a: float) -> tuple[float, float]:
    """(lower, upper) bounds of M_x = sum_{i=1..x} i^-a (Lemma 3)."""
    if x < 1:
        return 0.0, 0.0
    if a == 1:
        return math.log(x + 1), math.log(x) + 1
    return ((x + 1) ** (1 - a) - 1) / (1 - a), (x ** (1 - a) - a) / (1 - a)


def beta_prime(beta: float, m: int, N: int) -> float:
    """Lemma 1: the share of (n+1)-grams prefixed by the kept n-grams is at
    least beta - m / (N - m) (N n-grams over m sequences, N > m)."""
    if N <= m:
        raise ValueError("Lemma 1 needs more n-grams than sequences")
    return beta - m / (N - m)


def concentration_delta(k: int, distinct_n: int, N: int, delta: float) -> float:
    """Lemma 2: Delta(delta) for the empirical top-k mass of N draws over
    |D_n| = distinct_n outcomes."""
    if not (0 < delta < 1) or N <= 0 or distinct_n <= 0:
        raise ValueError("Lemma 2 needs 0 < delta < 1, N > 0 and |D_n| > 0")
    return 4.0 * math.sqrt(k * k * math.log(2.0 * distinct_n / delta) / (2.0 * N))


def _x(distinct_next: float, a: float, bp: float) -> float:
    return (distinct_next ** (1 - a) - a) * (1 - bp)


def u_bound(distinct_next: float, a: float, bp: float) -> float:
    """Theorem 1 (1), with the reading above: the true rank of the most
    frequent (n+1)-gram found is at most this."""
    if a == 1:
        raise ValueError("Theorem 1 is stated for a != 1")
    b = _x(distinct_next, a, bp) + 1
    if b <= 0:
        return float(distinct_next)
    return min(float(distinct_next), b ** (1 / (1 - a)))


def recall_mass_bound(distinct_next: float, a: float, bp: float, k: int) -> float:
    """Theorem 1 (3), with the reading above: lower bound of the share of the
    true top-k (n+1)-grams' mass that the found (n+1)-grams hold (unclamped)."""
    if a == 1:
        raise ValueError("Theorem 1 is stated for a != 1")
    return 1 - (_x(distinct_next, a, bp) + 1 - a) / ((k + 1) ** (1 - a) - 1)


def fit_zipf_exponent(counts, ranks: int | None = None) -> float:
    """Least-squares slope of log(count) against log(rank) over the first
    `ranks` counts (sorted descending; zeros ignored), negated: the Zipf
    exponent a of p_i ~ i^-a that fits them."""
    c = np.asarray(counts, dtype=np.float64)
    c = c[c > 0][: (ranks or len(c))]
    if len(c) < 2:
        raise ValueError("need at least two nonzero counts to fit a Zipf exponent")
    r = np.arange(1, len(c) + 1, dtype=np.float64)
    slope = np.polyfit(np.log(r), np.log(c), 1)[0]
    return float(-slope)


def predict(*, beta: float, m: int, N: int, distinct_n: int, distinct_next: int, a: float, k: int,
            k_prime: int, delta: float = 0.05) -> dict:
    """Theorem 1 (no sampling noise) and Theorem 2 (probability 1 - delta)
    for one pass: the kept k' n-grams hold `beta` of the N n-grams of m
    sequences; the (n+1)-grams are fitted by Zipf(a) over `distinct_next`
    items; k results are wanted."""
    bp = beta_prime(beta, m, N)
    d = concentration_delta(k_prime, distinct_n, N, delta)
    bpp = bp - d
    out = {"beta": beta, "beta_prime": bp, "zipf_a": a, "distinct_n": distinct_n,
           "distinct_next": distinct_next, "k": k, "k_prime": k_prime}
    if a == 1:
        out["note"] = "a = 1: Theorem 1 is stated for a != 1"
        return out
    rb = recall_mass_bound(distinct_next, a, bp, k)
    out["theorem1"] = {"u_bound": u_bound(distinct_next, a, bp), "recall_mass_bound": rb,
                       "clamped": min(1.0, max(0.0, rb))}
    rb2 = recall_mass_bound(distinct_next, a, bpp, k)
    out["theorem2"] = {"delta": delta, "Delta": d, "beta_double_prime": bpp,
                       "u_bound": u_bound(distinct_next, a, bpp), "recall_mass_bound": rb2,
                       "clamped": min(1.0, max(0.0, rb2))}
    return out
