"""The real-kernel form (the paper's r = 2 Re of the App. A integrand, Eq. 8) through every
reconstruction path, against the FP64 oracle.

A real-form kernel set stores its taps as real values; the direct form multiplies complex
z_ref by real taps, overlap-save keeps the Hermitian half of each partition spectrum, the
tensor-core form builds complex operands from the real taps.  Each is compared with the
oracle's direct sum (Eq. 8) over the oracle's own real-form kernels (spans exact), on full
series and window peaks, at the tolerances of the complex paths.
"""
import numpy as np
import pytest

import workload
from oracle import data, mf, ratio, reconstruct

pytestmark = pytest.mark.gpu

TOL = {"f64": 1e-12, "f32": 2e-6}


@pytest.fixture(scope="module")
def torch():
    import torch as t
    if not t.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2511_12894_gb300 import build
    build.build()
    return t


def _case(dtype, n, k, thr):
    if dtype == "f64":
        cfg = workload.config(1, n_override=n, k_override=k)
    else:
        cfg = workload.config(2, n_override=n, k_override=k)
    ref, nb = cfg.groups[0]
    ip = workload.inv_psd(cfg)
    x = data.strain(cfg)
    zo, _ = mf.matched_filter(x, ip, cfg.n, cfg.fs, cfg.f_low, cfg.f_high, ref.m1, ref.m2, cfg.pn_order)
    pk = ratio.build_ratio_kernels(ref, nb, cfg.n, cfg.fs, cfg.f_low, cfg.f_high, cfg.pn_order, ip, thr, real=True)
    return cfg, ref, nb, ip, zo, pk


def _oracle_series(zo, pk):
    return [reconstruct.reconstruct_direct(zo, *pk.kernel(j)) for j in range(len(pk.length))]


def _check(out_series, P, A, zs, W, tol):
    # the window peaks are float32 outputs on every grid: at least their rounding
    ptol = max(tol, 2.0 ** -23)
    for j, zh in enumerate(zs):
        zmax = np.abs(zh).max()
        if out_series is not None:
            assert np.abs(out_series[j] - zh).max() <= tol * zmax, (j, np.abs(out_series[j] - zh).max() / zmax)
        Po, Ao = reconstruct.window_peaks(zh, W)
        assert np.abs(np.sqrt(P[j]) - np.sqrt(Po)).max() <= ptol * zmax
        m2 = zh.real ** 2 + zh.imag ** 2
        for w in range(Po.shape[0]):
            seg = np.sort(m2[w * W:(w + 1) * W])
            bound = 4.0 * ptol * zmax * np.sqrt(seg[-1])
            if seg.size < 2 or seg[-1] - seg[-2] > bound:
                assert A[j, w] == Ao[w], (j, w)
            else:
                assert m2[A[j, w]] >= seg[-1] - bound


@pytest.mark.parametrize("dtype,n", [("f64", 1 << 13), ("f32", 1 << 15)])
def test_real_form_direct(torch, dtype, n):
    cfg, ref, nb, ip, zo, pk = _case(dtype, n, 6, 1e-3)
    from paper_2511_12894_gb300 import RatioFilter
    rf = RatioFilter.from_config(cfg)
    kern = rf.build_ratio_kernels(ref, nb, torch.tensor(ip, device="cuda"), 1e-3, real=True)
    assert kern.real and np.array_equal(kern.lag0, pk.lag0) and np.array_equal(kern.length, pk.length)
    cdt = torch.complex128 if dtype == "f64" else torch.complex64
    zt = torch.tensor(zo, dtype=cdt, device="cuda")
    zin = zt.cpu().numpy().astype(np.complex128)   # the oracle's z_ref as the GPU sees it
    zs = _oracle_series(zin, pk)
    out = rf.reconstruct(zt, kern, "direct").cpu().numpy()
    P, A = rf.reconstruct_winmax(zt, kern, cfg.window, "direct")
    _check(out, P.cpu().numpy(), A.cpu().numpy(), zs, cfg.window, TOL[dtype])


@pytest.mark.parametrize("cuts,blocks,parts", [([0], [4096], [1024]), ([0], [8192], [4096]), ([0], [512], [64]),
                                               ([0, 2000], [2048, 16384], [512, 4096])])
def test_real_form_overlap_save(torch, cuts, blocks, parts):
    """Hermitian half spectra at several block sizes and partition ratios, and two buckets."""
    cfg, ref, nb, ip, zo, pk = _case("f32", 1 << 15, 6, 1e-3)
    from paper_2511_12894_gb300 import RatioFilter
    rf = RatioFilter.from_config(cfg)
    kern = rf.build_ratio_kernels(ref, nb, torch.tensor(ip, device="cuda"), 1e-3, real=True)
    kern.prepare_buckets(cuts, blocks, parts)
    zt = torch.tensor(zo, dtype=torch.complex64, device="cuda")
    zs = _oracle_series(zt.cpu().numpy().astype(np.complex128), pk)
    out = rf.reconstruct(zt, kern, "os").cpu().numpy()
    P, A = rf.reconstruct_winmax(zt, kern, cfg.window, "os")
    _check(out, P.cpu().numpy(), A.cpu().numpy(), zs, cfg.window, TOL["f32"])


def test_real_form_pair_layout_is_refused(torch):
    from paper_2511_12894_gb300 import RatioFilter, RFError
    cfg, ref, nb, ip, zo, pk = _case("f32", 1 << 16, 2, 1e-3)
    rf = RatioFilter.from_config(cfg)
    kern = rf.build_ratio_kernels(ref, nb, torch.tensor(ip, device="cuda"), 1e-3, real=True)
    with pytest.raises(RFError):
        kern.prepare(32768, 8192)


def test_real_form_batched_and_tensor_core(torch):
    """Two references' real-form sets in one persistent overlap-save launch, and the
    tensor-core form (bf16x6) on one of them."""
    base = workload.config(4, n_override=1 << 15, k_override=24)
    rng = np.random.default_rng(77)
    groups = []
    for g, k in enumerate((3, 4)):
        ref = base.groups[g][0]
        nbs = workload.duration_lattice(ref, base.f_low, k, 0.05, 0.6, rng, eta_range=(0.235, 0.25), n_eta=1)
        groups.append((ref, nbs))
    from dataclasses import replace
    cfg = replace(base, groups=tuple(groups), injections=())
    ip = workload.inv_psd(cfg)
    x = data.strain(cfg)
    from paper_2511_12894_gb300 import RatioFilter
    rf = RatioFilter.from_config(cfg)
    ipt = torch.tensor(ip, device="cuda")
    kerns, zts, zss = [], [], []
    for ref, nbs in cfg.groups:
        zo, _ = mf.matched_filter(x, ip, cfg.n, cfg.fs, cfg.f_low, cfg.f_high, ref.m1, ref.m2, cfg.pn_order)
        pk = ratio.build_ratio_kernels(ref, nbs, cfg.n, cfg.fs, cfg.f_low, cfg.f_high, cfg.pn_order, ip, 1e-3,
                                       real=True)
        k = rf.build_ratio_kernels(ref, nbs, ipt, 1e-3, real=True)
        assert np.array_equal(k.lag0, pk.lag0) and np.array_equal(k.length, pk.length)
        zt = torch.tensor(zo, dtype=torch.complex64, device="cuda")
        kerns.append(k)
        zts.append(zt)
        zss.append(_oracle_series(zt.cpu().numpy().astype(np.complex128), pk))
    for k in kerns:
        k.prepare_buckets([0, 1500], [2048, 8192], [512, 2048])
    P, A = rf.reconstruct_batched(zts, kerns, cfg.window, "os")
    P, A = P.cpu().numpy(), A.cpu().numpy()
    row = 0
    for k, zs in zip(kerns, zss):
        _check(None, P[row:row + k.k], A[row:row + k.k], zs, cfg.window, TOL["f32"])
        row += k.k
    if max(int(k.length.max()) for k in kerns) <= 4096:
        out = rf.reconstruct(zts[0], kerns[0], "gemm", prec="bf16x6").cpu().numpy()
        Pg, Ag = rf.reconstruct_winmax(zts[0], kerns[0], cfg.window, "gemm", prec="bf16x6")
        _check(out, Pg.cpu().numpy(), Ag.cpu().numpy(), zss[0], cfg.window, TOL["f32"])


def test_real_form_import_roundtrip(torch):
    from paper_2511_12894_gb300 import RatioFilter
    cfg = workload.config(2, n_override=1 << 13, k_override=1)
    rf = RatioFilter.from_config(cfg)
    rng = np.random.default_rng(3)
    lengths = [5, 0, 300, 17]
    lags = [3, 0, -100, 4000]
    taps = rng.standard_normal(sum(lengths)).astype(np.float32)
    kern = rf.kernels_import(lags, lengths, taps, real=True)
    assert kern.real
    back = kern.taps().cpu().numpy()
    assert back.dtype == np.float32 and np.array_equal(back, taps)
    z = (rng.standard_normal(cfg.n) + 1j * rng.standard_normal(cfg.n)).astype(np.complex64)
    zt = torch.tensor(z, device="cuda")
    out = rf.reconstruct(zt, kern, "direct").cpu().numpy()
    off = np.concatenate([[0], np.cumsum(lengths)])
    for j in range(len(lengths)):
        zo = reconstruct.reconstruct_direct(z.astype(np.complex128), lags[j],
                                            taps[off[j]:off[j + 1]].astype(np.complex128))
        assert np.abs(out[j] - zo).max() <= TOL["f32"] * max(np.abs(zo).max(), 1e-30)
