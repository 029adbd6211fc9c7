"""Template-bank structuring (oracle; test infrastructure only).

Sec. III.A.  The bank is organised into sets of one reference and its dependent templates:

* Durations: tau = -t(f_low), the time from f_low to coalescence of the stationary-phase
  template (Eq. A2, t(f) = Psi'(f) / (2 pi) with t_c = 0).
* Chirp-mass bisection: the bank in chirp-mass order, mc = (m1 m2)^(3/5) / (m1 + m2)^(1/5)
  (equal chirp masses in bank order), is split into halves (the first half holds the floor
  of half the templates) until every set's duration spread, max tau - min tau, is at most
  the limit (10 s in the paper).
* Symmetric-mass-ratio bisection: each set, in eta = m1 m2 / (m1 + m2)^2 order (equal eta in
  bank order), is split into halves the same way until it holds at most the size limit (500
  in the paper); the halves of a set keep its duration spread.
* Reference: the template minimising sum_j |tau_i - tau_j| over its set.  Reading: in one
  dimension every template between the two middle durations of an even-sized set reaches the
  minimum, so sums within 1e-9 of each other (relative) count as equal and the lowest bank
  index among them is taken.
Sets are listed depth first, first half first.
"""
from __future__ import annotations

import math
from typing import List, Sequence, Tuple

import numpy as np

from . import taylorf2


def chirp_mass(m1: float, m2: float) -> float:
    return (m1 * m2) ** 0.6 / (m1 + m2) ** 0.2


def sym_mass_ratio(m1: float, m2: float) -> float:
    return m1 * m2 / ((m1 + m2) * (m1 + m2))


def duration(m1: float, m2: float, f_low: float, pn_order: int) -> float:
    """tau = -t(f_low) with t_c = 0 (Eq. A2)."""
    return -float(taylorf2.time_of_frequency(np.array([f_low]), m1, m2, pn_order, 0.0)[0])


def _halves(idx: List[int], keep) -> List[List[int]]:
    """Split into halves until keep(set) holds, depth first."""
    if len(idx) <= 1 or keep(idx):
        return [idx]
    h = len(idx) // 2
    return _halves(idx[:h], keep) + _halves(idx[h:], keep)


def reference_of(idx: Sequence[int], tau: np.ndarray) -> int:
    best, best_sum = -1, math.inf
    for i in idx:
        s = 0.0
        for j in idx:
            s += abs(tau[i] - tau[j])
        if best < 0 or s < best_sum - 1e-9 * best_sum:
            best, best_sum = i, s
        elif abs(s - best_sum) <= 1e-9 * best_sum and i < best:
            best, best_sum = i, min(s, best_sum)
    return best


def structure(bank: Sequence, f_low: float, pn_order: int, max_spread: float = 10.0,
              max_size: int = 500) -> Tuple[List[List[int]], List[int], np.ndarray]:
    """Sets of bank indices, their references, and the durations."""
    n = len(bank)
    mc = [chirp_mass(t.m1, t.m2) for t in bank]
    eta = [sym_mass_ratio(t.m1, t.m2) for t in bank]
    tau = np.array([duration(t.m1, t.m2, f_low, pn_order) for t in bank])
    order = sorted(range(n), key=lambda i: (mc[i], i))
    by_mc = _halves(order, lambda s: float(tau[s].max() - tau[s].min()) <= max_spread)
    sets: List[List[int]] = []
    for s in by_mc:
        sets += _halves(sorted(s, key=lambda i: (eta[i], i)), lambda x: len(x) <= max_size)
    refs = [reference_of(s, tau) for s in sets]
    return sets, refs, tau
