"""Algorithmic operation count of p-FHT-FSCL-L-P per frame (the roofline numerator).

Counting rules (additions, subtractions, min/abs and comparisons; gathers are memory traffic,
not operations), following the paper's complexity accounting (Section III-B, Table 1) with
the selection costs written out:
  f and g: 1 per output value;
  permutation candidate (Algorithm 2): N_v/2 f plus N_v/2 additions for LM, per candidate;
  LM selection: merge-sort comparisons of the 2L candidates;
  FHT node of size 2^s per path: s 2^s butterflies + 2^s for sum|alpha| + T metrics +
      min(T, s) 2^s comparisons for the top-T (T = min(L, 2^s));
  FHT list sort: merge-sort comparisons of the L T candidates;
  SPC node of size 2^s per path: min(tau + 1, s) 2^s sorting comparisons + 1 initial metric,
      and per split 2L metrics plus a merge sort of 2L;
  final selection: L per decoder.
A merge sort of n items costs n ceil(log2 n) comparisons.
"""
from __future__ import annotations

import math


def sort_cost(n: int) -> int:
    return n * math.ceil(math.log2(n)) if n > 1 else 0


def _node(r: int, s: int, L: int, spine: bool) -> int:
    N = 1 << s
    if r == 1:
        T = min(L, N)
        return L * (s * N + N + T + min(T, s) * N) + sort_cost(L * T)
    if r == s - 1:
        tau = min(L, N - 1)
        return L * (min(tau + 1, s) * N + 1) + tau * (2 * L + sort_cost(2 * L))
    ops = 0
    if spine:
        ops += 2 * L * N + sort_cost(2 * L)
    ops += 2 * L * (N // 2)  # f and g
    return ops + _node(r - 1, s - 1, L, spine) + _node(r, s - 1, L, False)


def ops_per_frame(m: int, r: int, P: int, L: int) -> int:
    """Operations to decode one frame with P decoders of list size L (root permuted)."""
    return P * (_node(r, m, L, True) + L)
