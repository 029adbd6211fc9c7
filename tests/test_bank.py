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
