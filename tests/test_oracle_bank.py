"""Pins of the bank structuring (Sec. III.A): duration against the Newtonian chirp time,
partition and limits, chirp-mass contiguity, medoid references by brute force."""
import math

import numpy as np
import pytest

import workload
from oracle import bank


def test_duration_is_the_newtonian_chirp_time_at_0pn():
    """tau = -t(f_low) (Eq. A2) reduces to (5/256) (pi f)^(-8/3) Mc^(-5/3) at Newtonian order."""
    for m1, m2 in [(1.4, 1.4), (2.9, 1.05), (2.2, 1.7)]:
        t = workload.Template(m1, m2)
        assert bank.duration(m1, m2, 20.0, 0) == pytest.approx(workload.newtonian_duration(t, 20.0), rel=1e-12)
    # the PN corrections change a 1.4 + 1.4 inspiral from 20 Hz (about 158 s) by a few per cent
    # (the positive 1PN term lengthens it)
    t0, t7 = bank.duration(1.4, 1.4, 20.0, 0), bank.duration(1.4, 1.4, 20.0, 7)
    assert t0 < t7 < 1.05 * t0


@pytest.mark.parametrize("count,spread,size", [(3000, 10.0, 500), (3000, 2.0, 64), (40, 1e9, 7)])
def test_sets_partition_the_bank_within_the_limits(count, spread, size):
    b = workload.synthetic_bank(count, seed=3)
    sets, refs, tau = bank.structure(b, 20.0, 7, spread, size)
    allidx = np.sort(np.concatenate([np.array(s) for s in sets]))
    assert np.array_equal(allidx, np.arange(count))
    for s, r in zip(sets, refs):
        assert len(s) <= size
        assert len(s) == 1 or tau[s].max() - tau[s].min() <= spread
        assert r in s
        # medoid by brute force: no template of the set has a smaller sum of |d tau|
        sums = np.abs(tau[s][:, None] - tau[s][None, :]).sum(axis=1)
        assert sums[s.index(r)] <= sums.min() * (1 + 1e-9) + 1e-300
        # ties go to the lowest bank index
        tied = [i for i, v in zip(s, sums) if v <= sums.min() * (1 + 1e-9)]
        assert r == min(tied)


def test_chirp_mass_sets_are_contiguous_and_split_only_when_needed():
    """Stage one cuts the chirp-mass order into runs; merging two neighbouring runs of one
    split would exceed the duration limit for at least one of the splits made."""
    b = workload.synthetic_bank(4000, seed=5)
    spread = 10.0
    sets, _, tau = bank.structure(b, 20.0, 7, spread, 10 ** 9)      # stage one only
    mc = np.array([bank.chirp_mass(t.m1, t.m2) for t in b])
    order = sorted(range(len(b)), key=lambda i: (mc[i], i))
    flat = [i for s in sets for i in sorted(s, key=lambda i: (mc[i], i))]
    assert flat == order                                               # contiguous runs, in order
    # the coarsest split is needed: the whole bank's spread exceeds the limit
    assert tau.max() - tau.min() > spread and len(sets) > 1
    # sizes follow halving: every run is floor or ceil of n / 2^depth for some depth
    n = len(b)
    ok = {n}
    frontier = [n]
    for _ in range(20):
        frontier = sorted({x for f in frontier for x in (f // 2, f - f // 2)})
        ok.update(frontier)
    assert all(len(s) in ok for s in sets)


def test_references_are_the_duration_medians():
    """In one dimension the minimiser of sum |tau_i - tau_j| is a median of the set."""
    b = workload.synthetic_bank(1500, seed=7)
    sets, refs, tau = bank.structure(b, 20.0, 7, 10.0, 500)
    for s, r in zip(sets, refs):
        d = np.sort(tau[s])
        lo, hi = d[(len(s) - 1) // 2], d[len(s) // 2]
        assert lo - 1e-9 <= tau[r] <= hi + 1e-9


def test_hand_worked_bisection_of_three_templates():
    """Sec. III.A by hand: three equal-mass templates whose Newtonian durations at 20 Hz are
    111, 100 and 104 s (bank order).  In chirp-mass order (111, 104, 100 s) the spread of 11 s
    exceeds 10 s, so the set is halved with the floor of half first: {111 s} and {104, 100 s}
    (spread 4 s).  The second set's two durations tie on the summed difference, and the lower
    bank index is its reference."""
    f = 20.0
    taus = [111.0, 100.0, 104.0]

    def equal_mass(tau):
        mc = (tau * 256.0 / 5.0 * (math.pi * f) ** (8.0 / 3.0)) ** (-3.0 / 5.0) / workload.MSUN_S
        m = mc * 2.0 ** 0.2
        return workload.Template(m, m)

    bnk = [equal_mass(t) for t in taus]
    sets, refs, tau = bank.structure(bnk, f, 0, max_spread=10.0, max_size=500)
    np.testing.assert_allclose(tau, taus, rtol=1e-12)
    assert sets == [[0], [1, 2]]
    assert refs == [0, 1]


def test_chirp_mass_and_symmetric_mass_ratio_closed_forms():
    """The bisection keys: equal masses m give Mc = m 2^(-1/5) (1.4 + 1.4 Msun: 1.2188 Msun)
    and eta = 1/4; masses 3 and 1 give Mc = 3^(3/5) / 4^(1/5) and eta = 3/16."""
    assert bank.chirp_mass(1.4, 1.4) == pytest.approx(1.4 * 2.0 ** -0.2, rel=1e-14)
    assert round(bank.chirp_mass(1.4, 1.4), 4) == 1.2188
    assert bank.sym_mass_ratio(1.7, 1.7) == pytest.approx(0.25, rel=1e-15)
    assert bank.chirp_mass(3.0, 1.0) == pytest.approx(3.0 ** 0.6 / 4.0 ** 0.2, rel=1e-14)
    assert bank.sym_mass_ratio(3.0, 1.0) == pytest.approx(3.0 / 16.0, rel=1e-15)


def test_spread_limit_is_inclusive():
    """Sec. III.A halves until the duration spread is equal to or less than the limit: a set
    whose spread equals the limit (the same double) stays whole, one ulp less splits it."""
    bnk = [workload.Template(1.4, 1.4), workload.Template(1.5, 1.45), workload.Template(1.6, 1.5)]
    _, _, tau = bank.structure(bnk, 20.0, 7, 1e9, 500)
    spread = float(tau.max() - tau.min())
    assert spread > 1.0
    assert sorted(map(sorted, bank.structure(bnk, 20.0, 7, spread, 500)[0])) == [[0, 1, 2]]
    assert len(bank.structure(bnk, 20.0, 7, float(np.nextafter(spread, 0.0)), 500)[0]) > 1


def test_size_limit_is_inclusive():
    """Sets hold no more than the size limit: eight equal templates stay one set at a limit of
    eight and split into halves at seven."""
    t = workload.Template(1.4, 1.3)
    assert bank.structure([t] * 8, 20.0, 7, 10.0, 8)[0] == [list(range(8))]
    assert bank.structure([t] * 8, 20.0, 7, 10.0, 7)[0] == [[0, 1, 2, 3], [4, 5, 6, 7]]


def test_equal_chirp_masses_keep_bank_order():
    """By hand: two copies of a 1.4 + 1.4 template (indices 0, 1) and a 2 + 2 one, whose
    durations at 20 Hz differ by far more than 10 s.  In chirp-mass order, equal keys in bank
    order, the halving gives {0} and {1, 2}, then {1} and {2}."""
    x, y = workload.Template(1.4, 1.4), workload.Template(2.0, 2.0)
    sets, refs, tau = bank.structure([x, x, y], 20.0, 7, 10.0, 500)
    assert tau[0] - tau[2] > 10.0
    assert sets == [[0], [1], [2]] and refs == [0, 1, 2]
