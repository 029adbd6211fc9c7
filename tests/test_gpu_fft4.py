"""The four-step FP32 transforms behind the matched filter (n = 2^18 .. 2^24): column DFTs
in tiles of adjacent columns with the inter-pass twiddle, then row DFTs with the transposed
store.  Checked through the matched filter (Eqs. 2-4: the data's forward transform, then one
inverse transform per reference) against the FP64 oracle, at every supported split of n
(N1 x N2 = 512 x 512 .. 4096 x 4096), for the stored-filter product form (several
references per launch, a ragged last launch) and the on-the-fly form (complex input).
"""
import numpy as np
import pytest

import workload
from oracle import data, mf

pytestmark = pytest.mark.gpu

TOL32 = 2e-6   # of max|z|, the FP32-equivalent bar


@pytest.fixture(scope="module")
def torch():
    import torch as t
    if not t.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2511_12894_gb300 import build
    build.build()
    return t


def _relerr(a, b):
    return np.abs(a - b).max() / np.abs(b).max()


@pytest.mark.parametrize("n,k", [(1 << 18, 3), (1 << 19, 3), (1 << 21, 2), (1 << 24, 2)])
def test_stored_filter_matches_oracle(torch, n, k):
    from paper_2511_12894_gb300 import RatioFilter
    cfg = workload.config(2, n_override=n, k_override=k)
    ref, nb = cfg.groups[0]
    refs = [ref] + list(nb[:k - 1])
    ip = workload.inv_psd(cfg)
    x = data.strain(cfg)
    rf = RatioFilter.from_config(cfg)
    filt, _ = rf.reference_filters(torch.tensor(ip, device="cuda"), refs)
    z = rf.mf_filtered(torch.tensor(x, dtype=torch.float32, device="cuda"), filt)
    for r, t in enumerate(refs):
        zo, _ = mf.matched_filter(x, ip, cfg.n, cfg.fs, cfg.f_low, cfg.f_high, t.m1, t.m2, cfg.pn_order)
        assert _relerr(z[r].cpu().numpy(), zo) < TOL32, (n, r)


def test_ragged_launches_equal_single_rows(torch):
    """At n = 2^20 eight references share a launch pair: eleven references run as 8 + 3, and
    every row equals the row computed alone and the oracle's."""
    from paper_2511_12894_gb300 import RatioFilter
    n = 1 << 20
    cfg = workload.config(2, n_override=n, k_override=11)
    ref, nb = cfg.groups[0]
    refs = [ref] + list(nb[:10])
    ip = workload.inv_psd(cfg)
    x = data.strain(cfg)
    rf = RatioFilter.from_config(cfg)
    filt, _ = rf.reference_filters(torch.tensor(ip, device="cuda"), refs)
    xt = torch.tensor(x, dtype=torch.float32, device="cuda")
    z = rf.mf_filtered(xt, filt)
    for r in (0, 7, 8, 10):
        assert torch.equal(rf.mf_filtered(xt, filt[r:r + 1])[0], z[r]), r
        t = refs[r]
        zo, _ = mf.matched_filter(x, ip, cfg.n, cfg.fs, cfg.f_low, cfg.f_high, t.m1, t.m2, cfg.pn_order)
        assert _relerr(z[r].cpu().numpy(), zo) < TOL32, r


@pytest.mark.parametrize("n", [1 << 18, 1 << 20, 1 << 23])
def test_on_the_fly_matches_oracle(torch, n):
    from paper_2511_12894_gb300 import RatioFilter
    cfg = workload.config(2, n_override=n, k_override=2)
    ref, nb = cfg.groups[0]
    refs = [ref, nb[0]]
    ip = workload.inv_psd(cfg)
    x = data.strain(cfg)
    rf = RatioFilter.from_config(cfg)
    z, _ = rf.mf_reference(torch.tensor(x, dtype=torch.float32, device="cuda"), torch.tensor(ip, device="cuda"),
                           refs)
    for r, t in enumerate(refs):
        zo, _ = mf.matched_filter(x, ip, cfg.n, cfg.fs, cfg.f_low, cfg.f_high, t.m1, t.m2, cfg.pn_order)
        assert _relerr(z[r].cpu().numpy(), zo) < TOL32, (n, r)
