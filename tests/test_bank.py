"""Bank structuring through the C ABI (host code; no GPU) against the oracle's same
definition (Sec. III.A): identical sets, references and durations."""
import numpy as np
import pytest

import workload
from oracle import bank as obank


@pytest.fixture(scope="module")
def rfmod():
    from paper_2511_12894_gb300 import build
    build.build()
    import paper_2511_12894_gb300 as P
    return P


@pytest.mark.parametrize("count,spread,size,pn", [(3000, 10.0, 500, 7), (2000, 1.0, 37, 4), (257, 1e6, 8, 0),
                                                  (1, 10.0, 500, 7)])
def test_bank_structure_matches_the_oracle(rfmod, count, spread, size, pn):
    b = workload.synthetic_bank(count, seed=11)
    sets, refs, tau = rfmod.bank_structure(b, 20.0, pn, spread, size)
    osets, orefs, otau = obank.structure(b, 20.0, pn, spread, size)
    np.testing.assert_allclose(tau, otau, rtol=1e-12)
    assert [sorted(s) for s in sets] == [sorted(s) for s in osets]
    assert refs == orefs


def test_bank_structure_edge_cases(rfmod):
    from paper_2511_12894_gb300 import RFError
    sets, refs, tau = rfmod.bank_structure([], 20.0)
    assert sets == [] and refs == []
    # equal templates: one set, the lowest index is the reference
    t = workload.Template(1.4, 1.3)
    sets, refs, _ = rfmod.bank_structure([t, t, t, t], 20.0)
    assert sets == [[0, 1, 2, 3]] and refs == [0]
    for kw in [dict(f_low=0.0), dict(f_low=20.0, pn_order=8), dict(f_low=20.0, max_spread=0.0),
               dict(f_low=20.0, max_size=0)]:
        with pytest.raises(RFError):
            rfmod.bank_structure([t], **kw)



def test_spread_limit_is_inclusive(rfmod):
    """Sec. III.A halves a set until its duration spread is equal to or less than the limit: a
    set whose spread equals the limit exactly (the library's own durations) is kept whole."""
    bnk = [workload.Template(1.4, 1.4), workload.Template(1.5, 1.45), workload.Template(1.6, 1.5)]
    _, _, tau = rfmod.bank_structure(bnk, 20.0, 7, 1e9, 500)
    spread = float(tau.max() - tau.min())
    assert spread > 1.0
    assert sorted(map(sorted, rfmod.bank_structure(bnk, 20.0, 7, spread, 500)[0])) == [[0, 1, 2]]
    assert len(rfmod.bank_structure(bnk, 20.0, 7, float(np.nextafter(spread, 0.0)), 500)[0]) > 1


def test_durations_do_not_depend_on_the_coalescence_time(rfmod):
    """tau = -t(f_low) is the time from f_low to coalescence: the templates' t_c and phase do not
    enter it, nor the sets built from it."""
    base = workload.synthetic_bank(300, seed=5)
    moved = [workload.Template(t.m1, t.m2, tc=3.0 + 0.1 * i, phic=0.5) for i, t in enumerate(base)]
    a, b = rfmod.bank_structure(base, 20.0, 7, 10.0, 40), rfmod.bank_structure(moved, 20.0, 7, 10.0, 40)
    np.testing.assert_array_equal(a[2], b[2])
    assert a[0] == b[0] and a[1] == b[1]


def test_equal_chirp_masses_keep_bank_order(rfmod):
    """Templates with equal chirp mass take bank order in the chirp-mass ordering (the same
    hand-worked bank as the oracle's pin)."""
    x, y = workload.Template(1.4, 1.4), workload.Template(2.0, 2.0)
    sets, refs, _ = rfmod.bank_structure([x, x, y], 20.0, 7, 10.0, 500)
    assert sets == [[0], [1], [2]] and refs == [0, 1, 2]
