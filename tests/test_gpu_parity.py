"""Parity of the CUDA path (through the C ABI) with the FP64 oracle.

Tolerances: RF_F64 paths agree to 1e-12 of max|z| (FP64 rounding over a few
thousand operations); RF_F32 paths to 2e-6 of max|z| (the FP32-equivalent bar);
integer outputs (lags, lengths, argmax) exactly, argmax only where the oracle's
top two samples of a window differ by more than the error bound (several
indices are then correct).
"""
from dataclasses import replace

import numpy as np
import pytest

import workload
from oracle import data, mf, ratio, reconstruct, taylorf2

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


def _rf(cfg):
    from paper_2511_12894_gb300 import RatioFilter
    return RatioFilter.from_config(cfg)


def _small_f32_cfg(n=1 << 15, k=6):
    # the FP32 paper-shaped workload (fs 2048 Hz, f_low 20 Hz, 3.5PN) on a shorter segment
    return workload.config(2, n_override=n, k_override=k)


def _relerr(a, b):
    return np.abs(a - b).max() / np.abs(b).max()


def _argmax_ok(P_oracle_series, A_gpu, A_oracle, W, bound):
    """Argmax must match where the window's top two |z|^2 differ by more than `bound`."""
    mag2 = P_oracle_series
    n = mag2.shape[0]
    checked = 0
    for w in range(A_oracle.shape[0]):
        seg = np.sort(mag2[w * W: min(n, (w + 1) * W)])
        if seg.size < 2 or seg[-1] - seg[-2] > bound:
            assert A_gpu[w] == A_oracle[w], (w, A_gpu[w], A_oracle[w])
            checked += 1
        else:
            assert mag2[A_gpu[w]] >= seg[-1] - bound and w * W <= A_gpu[w] < (w + 1) * W
    return checked


# ---------------------------------------------------------------- template and matched filter

@pytest.mark.parametrize("pn,dtype", [(2, "f64"), (7, "f64"), (7, "f32")])
def test_template_fd(torch, pn, dtype):
    n, fs = 1 << 14, 1024.0
    from paper_2511_12894_gb300 import RatioFilter
    rf = RatioFilter(n, fs, 30.0, fs / 2 - 53, pn, dtype)
    t = workload.Template(1.7, 1.3, tc=0.25, phic=0.4)
    h = rf.template_fd(t).cpu().numpy()
    ho = mf.template(n, fs, t.m1, t.m2, pn, t.tc, t.phic)
    # an FP64 phase Psi carries an absolute rounding error of a few ulp(|Psi|), and
    # |Psi| reaches 1e9 rad at the lowest bins: the bound is per bin
    f = mf.freqs(n, fs)[1:]
    psi = np.abs(taylorf2.phase(f, t.m1, t.m2, pn, t.tc, t.phic))
    err = np.abs(h[1:] - ho[1:]) / np.abs(ho[1:])
    eps = 2.0 ** -52 if dtype == "f64" else 2.0 ** -23
    assert np.all(err <= 32 * 2.0 ** -52 * psi + 8 * eps)
    assert h[0] == 0


@pytest.mark.parametrize("n", [1 << 8, 1 << 11, 1 << 12, 1 << 13, 1 << 16])
def test_mf_reference_f64(torch, n):
    cfg = workload.config(1, n_override=n, k_override=2)
    ref = cfg.groups[0][0]
    ip = workload.inv_psd(cfg)
    x = data.strain(cfg)
    rf = _rf(cfg)
    z, sg = rf.mf_reference(torch.tensor(x, device="cuda"), torch.tensor(ip, device="cuda"), [ref, cfg.groups[0][1][0]])
    zo, No = mf.matched_filter(x, ip, cfg.n, cfg.fs, cfg.f_low, cfg.f_high, ref.m1, ref.m2, cfg.pn_order)
    assert _relerr(z[0].cpu().numpy(), zo) < TOL["f64"]
    assert abs(sg[0].item() / No - 1) < 1e-13
    t = cfg.groups[0][1][0]
    zo1, _ = mf.matched_filter(x, ip, cfg.n, cfg.fs, cfg.f_low, cfg.f_high, t.m1, t.m2, cfg.pn_order)
    assert _relerr(z[1].cpu().numpy(), zo1) < TOL["f64"]


@pytest.mark.parametrize("n", [1 << 12, 1 << 15, 1 << 17])
def test_mf_reference_f32(torch, n):
    cfg = _small_f32_cfg(n, 2)
    ref = cfg.groups[0][0]
    ip = workload.inv_psd(cfg)
    x = data.strain(cfg)
    rf = _rf(cfg)
    z, _ = rf.mf_reference(torch.tensor(x, dtype=torch.float32, device="cuda"), torch.tensor(ip, device="cuda"), [ref])
    zo, _ = mf.matched_filter(x, ip, cfg.n, cfg.fs, cfg.f_low, cfg.f_high, ref.m1, ref.m2, cfg.pn_order)
    assert _relerr(z[0].cpu().numpy(), zo) < TOL["f32"]


@pytest.mark.parametrize("dtype,n", [("f64", 1 << 12), ("f64", 1 << 15), ("f32", 1 << 13), ("f32", 1 << 17)])
def test_mf_filtered_matches_oracle(torch, dtype, n):
    """Stored reference filters (Eqs. 2-4 split into a data-independent filter) give the
    oracle's matched filter for several references in one batched call."""
    cfg = workload.config(1, n_override=n, k_override=3) if dtype == "f64" else _small_f32_cfg(n, 3)
    ref, nb = cfg.groups[0]
    refs = [ref] + list(nb[:2])
    ip = workload.inv_psd(cfg)
    x = data.strain(cfg)
    rf = _rf(cfg)
    ipt = torch.tensor(ip, device="cuda")
    filt, sg = rf.reference_filters(ipt, refs)
    assert filt.shape == (3, n // 2 + 1)
    xt = torch.tensor(x, dtype=torch.float64 if dtype == "f64" else torch.float32, device="cuda")
    z = rf.mf_filtered(xt, filt)
    for r, t in enumerate(refs):
        zo, No = mf.matched_filter(x, ip, cfg.n, cfg.fs, cfg.f_low, cfg.f_high, t.m1, t.m2, cfg.pn_order)
        assert _relerr(z[r].cpu().numpy(), zo) < TOL[dtype], (r, dtype, n)
        assert abs(sg[r].item() / No - 1) < 1e-13
    # a single reference (its own filter row) gives the same row
    z1 = rf.mf_filtered(xt, filt[1:2])
    assert torch.equal(z1[0], z[1])


def test_zero_noise_injection_optimal_snr(torch):
    cfg = workload.config(1, n_override=1 << 14, k_override=3)
    inj = workload.Injection(-1, 0, 5000, 10.0)
    cfg = replace(cfg, injections=(inj,))
    x = data.strain(cfg, noise=False)
    ip = workload.inv_psd(cfg)
    rf = _rf(cfg)
    ref = cfg.groups[0][0]
    z, _ = rf.mf_reference(torch.tensor(x, device="cuda"), torch.tensor(ip, device="cuda"), [ref])
    a = np.abs(z[0].cpu().numpy())
    assert int(np.argmax(a)) == 5000 and abs(a[5000] - 10.0) < 1e-10


# ---------------------------------------------------------------- builder

@pytest.mark.parametrize("n,k,thr,rel", [(1 << 13, 5, 1e-3, True), (1 << 16, 16, 1e-3, True),
                                         (1 << 14, 4, 1e-5, True), (1 << 13, 3, 1e-4, False)])
def test_build_ratio_kernels_f64(torch, n, k, thr, rel):
    cfg = workload.config(1, n_override=n, k_override=k)
    ref, nb = cfg.groups[0]
    ip = workload.inv_psd(cfg)
    rf = _rf(cfg)
    kern = rf.build_ratio_kernels(ref, nb, torch.tensor(ip, device="cuda"), thr, rel)
    pk = ratio.build_ratio_kernels(ref, nb, cfg.n, cfg.fs, cfg.f_low, cfg.f_high, cfg.pn_order, ip, thr, rel)
    assert np.array_equal(kern.lag0, pk.lag0)
    assert np.array_equal(kern.length, pk.length)
    assert np.array_equal(kern.offset, pk.offset)
    assert np.allclose(kern.df_low, pk.df_low, rtol=1e-12, atol=0)
    taps = kern.taps().cpu().numpy()
    assert _relerr(taps, pk.taps) < TOL["f64"]


@pytest.mark.parametrize("n_build", [-1, 1 << 13])
def test_build_ratio_kernels_coarse_grid(torch, n_build):
    """Kernels built on a coarser grid (fixed, or per neighbour by the extent rule; Sec. II.D)
    against the oracle's same definition: grids, spans and signed lags exact, taps to FP64
    rounding; neighbours spanning several grids come back in their own order."""
    n = 1 << 16
    cfg = workload.config(1, n_override=n, k_override=4)
    ref = cfg.groups[0][0]
    nb = list(cfg.groups[0][1]) + list(workload.duration_lattice(ref, cfg.f_low, 4, 0.2, 3.0,
                                                                  np.random.default_rng(9), n_eta=1,
                                                                  mrange=(1.0, 4.5)))
    nb = [nb[i] for i in (4, 0, 7, 1, 5, 2, 6, 3)]     # grids out of order
    ip = workload.inv_psd(cfg)
    rf = _rf(cfg)
    kern = rf.build_ratio_kernels(ref, nb, torch.tensor(ip, device="cuda"), 1e-4, n_build=n_build)
    pk = ratio.build_ratio_kernels(ref, nb, n, cfg.fs, cfg.f_low, cfg.f_high, cfg.pn_order, ip, 1e-4,
                                   n_build=n_build)
    assert np.array_equal(kern.grid, pk.grid)
    if n_build < 0:
        assert len(np.unique(kern.grid)) > 1
    assert np.array_equal(kern.lag0, pk.lag0) and np.array_equal(kern.length, pk.length)
    assert _relerr(kern.taps().cpu().numpy(), pk.taps) < TOL["f64"]


@pytest.mark.parametrize("n_build,rel,thr", [(0, True, 3e-5), (0, False, 1e-3), (-1, False, 1e-2), (-1, True, 1e-4),
                                             (-1, False, 1e-30)])
def test_build_ratio_kernels_analytic(torch, n_build, rel, thr):
    """Analytic truncation (Sec. II.D with the App. A expressions) against the oracle's same
    definition: spans and signed lags exact, taps to FP64 rounding; on the data grid and on
    per-neighbour build grids, with relative and absolute (1/s) thresholds; a vanishing
    amplitude keeps each whole grid."""
    n = 1 << 16
    cfg = workload.config(1, n_override=n, k_override=4)
    ref = cfg.groups[0][0]
    nb = list(cfg.groups[0][1]) + list(workload.duration_lattice(ref, cfg.f_low, 4, 0.2, 3.0,
                                                                  np.random.default_rng(9), n_eta=1,
                                                                  mrange=(1.0, 4.5)))
    ip = workload.inv_psd(cfg)
    rf = _rf(cfg)
    kern = rf.build_ratio_kernels(ref, nb, torch.tensor(ip, device="cuda"), thr, relative=rel, n_build=n_build,
                                  analytic=True)
    pk = ratio.build_ratio_kernels(ref, nb, n, cfg.fs, cfg.f_low, cfg.f_high, cfg.pn_order, ip, thr, rel,
                                   n_build=n_build, analytic=True)
    assert np.array_equal(kern.grid, pk.grid)
    assert np.array_equal(kern.lag0, pk.lag0) and np.array_equal(kern.length, pk.length)
    assert _relerr(kern.taps().cpu().numpy(), pk.taps) < TOL["f64"]
    if thr < 1e-20:
        assert np.array_equal(kern.length, kern.grid) and not kern.lag0.any()
        return
    # the same threshold without the analytic flag truncates numerically (different spans)
    num = rf.build_ratio_kernels(ref, nb, torch.tensor(ip, device="cuda"), thr if rel else thr / (2 * cfg.fs),
                                 relative=rel, n_build=n_build)
    assert not np.array_equal(num.length, kern.length)


@pytest.mark.parametrize("analytic,rel,thr", [(False, True, 1e-3), (True, False, 1e-2)])
def test_build_ratio_kernels_real_form(torch, analytic, rel, thr):
    """The paper's real-kernel form (taps 2 Re rho) against the oracle's same definition,
    numeric and analytic truncation: spans exact, taps (stored as real values) to FP64
    rounding, the oracle's imaginary parts 0."""
    n = 1 << 16
    cfg = workload.config(1, n_override=n, k_override=6)
    ref, nb = cfg.groups[0]
    ip = workload.inv_psd(cfg)
    rf = _rf(cfg)
    kern = rf.build_ratio_kernels(ref, nb, torch.tensor(ip, device="cuda"), thr, relative=rel, analytic=analytic,
                                  real=True)
    pk = ratio.build_ratio_kernels(ref, nb, n, cfg.fs, cfg.f_low, cfg.f_high, cfg.pn_order, ip, thr, rel,
                                   analytic=analytic, real=True)
    assert np.array_equal(kern.lag0, pk.lag0) and np.array_equal(kern.length, pk.length)
    # stored as real values: half the bytes of complex taps
    assert kern.real and np.all(pk.taps.imag == 0)
    taps = kern.taps().cpu().numpy()
    assert taps.dtype == np.float64 and taps.shape == pk.taps.shape
    assert _relerr(taps, pk.taps.real) < TOL["f64"]


def test_build_rejects_unknown_truncation_flags(torch):
    """Truncation flags outside RF_TRUNC_RELATIVE | RF_TRUNC_ANALYTIC, and an analytic
    threshold of 0, are rejected before any work."""
    import ctypes
    import paper_2511_12894_gb300 as P
    cfg = workload.config(1, n_override=1 << 12, k_override=1)
    ref, nb = cfg.groups[0]
    rf = _rf(cfg)
    ip = torch.tensor(workload.inv_psd(cfg), device="cuda")
    h = ctypes.c_void_p()
    for flags, thr in [(8, 1e-3), (-1, 1e-3), (3, 0.0)]:
        st = P._lib.rf_build_ratio_kernels(rf.handle, P._templates([ref]), P._templates(nb), len(nb),
                                           ctypes.c_void_p(ip.data_ptr()), thr, flags, 0, ctypes.byref(h), None)
        assert st == P.RF_EINVAL and not h.value


def test_build_ratio_kernels_f32_long(torch):
    cfg = _small_f32_cfg(1 << 17, 6)
    ref = cfg.groups[0][0]
    nb = workload.duration_lattice(ref, cfg.f_low, 8, 0.3, 2.0, np.random.default_rng(3), n_eta=1)
    cfg = replace(cfg, groups=((ref, nb),))
    ip = workload.inv_psd(cfg)
    rf = _rf(cfg)
    kern = rf.build_ratio_kernels(ref, nb, torch.tensor(ip, device="cuda"), 1e-3)
    pk = ratio.build_ratio_kernels(ref, nb, cfg.n, cfg.fs, cfg.f_low, cfg.f_high, cfg.pn_order, ip, 1e-3)
    assert np.array_equal(kern.lag0, pk.lag0) and np.array_equal(kern.length, pk.length)
    taps = kern.taps().cpu().numpy()
    assert _relerr(taps, pk.taps.astype(np.complex64)) < 1e-6
    assert pk.length.max() > 1000


def test_build_special_cases(torch):
    """Same template, a whole-sample time shift and a phase offset: the shifted
    template's kernel is the reference kernel moved by the shift."""
    cfg = workload.config(1, n_override=1 << 13, k_override=1)
    ref = cfg.groups[0][0]
    ip = workload.inv_psd(cfg)
    rf = _rf(cfg)
    tg = [ref, replace(ref, tc=37 / cfg.fs), replace(ref, phic=0.9)]
    kern = rf.build_ratio_kernels(ref, tg, torch.tensor(ip, device="cuda"), 1e-3)
    pk = ratio.build_ratio_kernels(ref, tg, cfg.n, cfg.fs, cfg.f_low, cfg.f_high, cfg.pn_order, ip, 1e-3)
    assert np.array_equal(kern.lag0, pk.lag0) and np.array_equal(kern.length, pk.length)
    # the shifted template's kernel is the same kernel moved by -37 lags
    assert kern.lag0[1] == kern.lag0[0] - 37 and kern.length[1] == kern.length[0]


# ---------------------------------------------------------------- reconstruction

def _random_kernels(rng, n, lengths, lags, dtype):
    taps = []
    for L in lengths:
        c = (rng.standard_normal(L) + 1j * rng.standard_normal(L)) / np.sqrt(max(L, 1))
        taps.append(c)
    t = np.concatenate(taps) if taps else np.zeros(0, complex)
    if dtype == "f32":
        t = t.astype(np.complex64).astype(np.complex128)
    return t


@pytest.mark.parametrize("dtype", ["f64", "f32"])
def test_reconstruct_direct_edge_lengths(torch, dtype):
    """L in {0,1,2,31,32,33,255,256,257,n}, lags of both signs and wrapping, k uneven."""
    n = 1 << 12
    rng = np.random.default_rng(4)
    lengths = [0, 1, 2, 31, 32, 33, 255, 256, 257, 1000, n, 7, 600, 513, 64, 65, 3]
    lags = [0, 5, -3, n // 2, -(n // 2) + 1, 100, -1, 0, 37, -700, 0, n // 2 - 3, -5, 1999, -2048 + 1, 11, -n // 4]
    cfgd = workload.config(1, n_override=n, k_override=1)
    if dtype == "f32":
        cfgd = replace(cfgd, dtype="f32")
    rf = _rf(cfgd)
    z = rng.standard_normal(n) + 1j * rng.standard_normal(n)
    if dtype == "f32":
        z = z.astype(np.complex64).astype(np.complex128)
    taps = _random_kernels(rng, n, lengths, lags, dtype)
    # FP32 sums of L random unit-variance terms: rounding grows like sqrt(L) (two-level
    # summation in chunks of 256 taps); the FP32-equivalent bar 2e-6 holds up to ~1000 taps
    tol = lambda L: TOL[dtype] * (max(1.0, np.sqrt(L / 1024.0)) if dtype == "f32" else 1.0)
    kern = rf.kernels_import(lags, lengths, taps)
    zt = torch.tensor(z.astype(np.complex128 if dtype == "f64" else np.complex64), device="cuda")
    out = rf.reconstruct(zt, kern, "direct").cpu().numpy()
    off = np.concatenate([[0], np.cumsum(lengths)])
    for j in range(len(lengths)):
        zo = reconstruct.reconstruct_direct(z, lags[j], taps[off[j]:off[j + 1]])
        scale = max(np.abs(zo).max(), 1e-30)
        err = np.abs(out[j] - zo).max() / scale if lengths[j] else np.abs(out[j]).max()
        assert err < (tol(lengths[j]) if lengths[j] else 1e-30), (j, lengths[j], err)
    # fused window peaks against the oracle's peaks of the same series
    for W in (1, 3, 1000, 1024, 4096):
        P, A = rf.reconstruct_winmax(zt, kern, W, "direct")
        P, A = P.cpu().numpy(), A.cpu().numpy()
        for j in range(len(lengths)):
            zo = reconstruct.reconstruct_direct(z, lags[j], taps[off[j]:off[j + 1]])
            Po, Ao = reconstruct.window_peaks(zo, W)
            scale = max(Po.max(), 1e-30)
            # peaks are stored as float32: add its rounding
            bound = (4 * tol(lengths[j]) + 2.0 ** -23) * scale + 1e-30
            assert np.abs(P[j] - Po).max() <= bound
            mag2 = zo.real ** 2 + zo.imag ** 2
            _argmax_ok(mag2, A[j], Ao, W, 8 * tol(lengths[j]) * scale)


def test_reconstruct_matches_oracle_cfg1_full(torch):
    """The FP64 small workload end to end at its full size (n = 65536, 16 neighbours)."""
    cfg = workload.config(1)
    ref, nb = cfg.groups[0]
    ip = workload.inv_psd(cfg)
    x = data.strain(cfg)
    rf = _rf(cfg)
    ipt = torch.tensor(ip, device="cuda")
    z, _ = rf.mf_reference(torch.tensor(x, device="cuda"), ipt, [ref])
    kern = rf.build_ratio_kernels(ref, nb, ipt, cfg.threshold)
    out = rf.reconstruct(z[0], kern, "direct").cpu().numpy()
    P, A = rf.reconstruct_winmax(z[0], kern, cfg.window, "direct")
    P, A = P.cpu().numpy(), A.cpu().numpy()
    zo, _ = mf.matched_filter(x, ip, cfg.n, cfg.fs, cfg.f_low, cfg.f_high, ref.m1, ref.m2, cfg.pn_order)
    pk = ratio.build_ratio_kernels(ref, nb, cfg.n, cfg.fs, cfg.f_low, cfg.f_high, cfg.pn_order, ip, cfg.threshold)
    assert np.array_equal(kern.lag0, pk.lag0) and np.array_equal(kern.length, pk.length)
    for j in range(len(nb)):
        zh = reconstruct.reconstruct_direct(zo, *pk.kernel(j))
        assert _relerr(out[j], zh) < TOL["f64"]
        Po, Ao = reconstruct.window_peaks(zh, cfg.window)
        assert np.abs(P[j] - Po).max() <= 1e-6 * Po.max()     # peaks are stored as float32
        _argmax_ok(zh.real ** 2 + zh.imag ** 2, A[j], Ao, cfg.window, 1e-9 * Po.max())
    # the injected neighbour is found at its arrival sample
    inj = cfg.injections[0]
    w = inj.sample // cfg.window
    assert A[inj.template_index, w] == inj.sample


def test_winmax_series(torch):
    cfg = workload.config(1, n_override=1 << 14, k_override=1)
    rf = _rf(replace(cfg, dtype="f32"))
    rng = np.random.default_rng(9)
    z = (rng.standard_normal((3, cfg.n)) + 1j * rng.standard_normal((3, cfg.n))).astype(np.complex64)
    z[1, 100:110] = 5.0  # ties inside one window
    P, A = rf.winmax(torch.tensor(z, device="cuda"), 1000)
    P, A = P.cpu().numpy(), A.cpu().numpy()
    for r in range(3):
        zz = z[r].astype(np.complex128)
        Po, Ao = reconstruct.window_peaks(z[r], 1000)
        assert np.abs(P[r] - Po).max() <= 1e-6 * Po.max()
        _argmax_ok(np.abs(zz) ** 2, A[r], Ao, 1000, 1e-5 * Po.max())
    assert A[1, 0] == 100


# ---------------------------------------------------------------- overlap-save

_OS_N = 1 << 15


@pytest.fixture(scope="module")
def os_case():
    """Random z and kernels whose lengths sit around every partition length tested (Lp - 1,
    Lp, Lp + 1, 2 Lp + 7), above n/2, and zero; lags of both signs and wrapping; with the
    oracle's direct sums, computed once for every layout."""
    n = _OS_N
    rng = np.random.default_rng(1515)
    lengths = [1, 2, 31, 63, 64, 65, 135, 255, 256, 257, 519, 1023, 1024, 1025, 2055, 2047, 2048, 2049,
               4095, 4096, 4097, 8199, 8191, 8192, 8193, 16391, n // 2 + 3, 0]
    lags = [int(v) for v in rng.integers(-n // 2 + 1, n // 2 + 1, len(lengths))]
    lags[:4] = [0, -5, n // 2, -(n // 2) + 1]
    z = (rng.standard_normal(n) + 1j * rng.standard_normal(n)).astype(np.complex64)
    taps = [((rng.standard_normal(L) + 1j * rng.standard_normal(L)) / np.sqrt(max(L, 1))).astype(np.complex64)
            for L in lengths]
    zo = [reconstruct.reconstruct_direct(z.astype(np.complex128), lags[j], taps[j].astype(np.complex128))
          for j in range(len(lengths))]
    return z, lengths, lags, taps, zo


@pytest.mark.parametrize("B,Lp", [(512, 256), (512, 128), (512, 64), (1024, 512), (8192, 4096), (8192, 2048),
                                  (8192, 1024), (16384, 8192), (16384, 4096), (16384, 2048), (32768, 16384),
                                  (32768, 8192)])
def test_reconstruct_os_edge_lengths(torch, os_case, B, Lp):
    """Overlap-save with block B and partitions of Lp taps (hop B - Lp, which does not divide
    n for Lp < B/2, so the last block is partial) against the oracle's direct sum; window
    peaks for windows down to 1 sample."""
    z, lengths, lags, taps, zo = os_case
    n = _OS_N
    cfg = replace(workload.config(1, n_override=n, k_override=1), dtype="f32")
    rf = _rf(cfg)
    kern = rf.kernels_import(lags, lengths, np.concatenate(taps))
    kern.prepare(B, Lp)
    assert kern.os_layout() == (B, Lp)
    zt = torch.tensor(z, device="cuda")
    out = rf.reconstruct(zt, kern, "os").cpu().numpy()
    for j, L in enumerate(lengths):
        if L == 0:
            assert np.abs(out[j]).max() == 0.0
            continue
        assert _relerr(out[j], zo[j]) < TOL["f32"], (B, Lp, j, L)
    for W in (1, 3, 1000, 2048, n):
        P, A = rf.reconstruct_winmax(zt, kern, W, "os")
        P, A = P.cpu().numpy(), A.cpu().numpy()
        for j, L in enumerate(lengths):
            Po, Ao = reconstruct.window_peaks(zo[j], W)
            if L == 0:
                assert np.all(P[j] == 0)
                continue
            assert np.abs(P[j] - Po).max() <= 4 * TOL["f32"] * Po.max(), (B, Lp, W, j)
            _argmax_ok(zo[j].real ** 2 + zo[j].imag ** 2, A[j], Ao, W, 8 * TOL["f32"] * Po.max())


@pytest.mark.parametrize("cuts,blocks,parts", [([0, 1000], [4096, 16384], [1024, 4096]),
                                               ([0, 2000, 8000], [4096, 16384, 32768], [1024, 4096, 16384]),
                                               ([0, 64, 2048, 8192], [1024, 512, 8192, 16384],
                                                [128, 256, 2048, 8192])])
def test_reconstruct_os_length_buckets(torch, os_case, cuts, blocks, parts):
    """A layout per kernel-length bucket (one segment transform and launch per bucket) gives
    the oracle's direct sums in the original row order, and the same window peaks."""
    z, lengths, lags, taps, zo = os_case
    n = _OS_N
    cfg = replace(workload.config(1, n_override=n, k_override=1), dtype="f32")
    rf = _rf(cfg)
    kern = rf.kernels_import(lags, lengths, np.concatenate(taps))
    kern.prepare_buckets(cuts, blocks, parts)
    assert kern.os_buckets() == list(zip(cuts, blocks, parts))
    zt = torch.tensor(z, device="cuda")
    out = rf.reconstruct(zt, kern, "os").cpu().numpy()
    for j, L in enumerate(lengths):
        if L == 0:
            assert np.abs(out[j]).max() == 0.0
            continue
        assert _relerr(out[j], zo[j]) < TOL["f32"], (cuts, j, L)
    P, A = rf.reconstruct_winmax(zt, kern, 1000, "os")
    P, A = P.cpu().numpy(), A.cpu().numpy()
    for j, L in enumerate(lengths):
        if L == 0:
            continue
        Po, Ao = reconstruct.window_peaks(zo[j], 1000)
        assert np.abs(P[j] - Po).max() <= 4 * TOL["f32"] * Po.max()
        _argmax_ok(zo[j].real ** 2 + zo[j].imag ** 2, A[j], Ao, 1000, 8 * TOL["f32"] * Po.max())
    with pytest.raises(Exception):
        kern.prepare_buckets([5, 100], [4096, 4096], [1024, 1024])      # first cut must be 0
    with pytest.raises(Exception):
        kern.prepare_buckets([0, 100], [4096, 4096], [1024, 3000])      # partition not B/2, B/4, B/8


@pytest.mark.parametrize("long_part", [8192, 16384])
def test_batched_length_buckets_match_per_group(torch, long_part):
    """The persistent batched launch runs one pass per layout bucket and writes the same rows
    as the per-group bucketed reconstruction (the long bucket on 32768-point blocks: on CTA
    pairs at Q = 4, on one CTA per block at Q = 2)."""
    cfg = _batch_cfg()
    ip = torch.tensor(workload.inv_psd(cfg), device="cuda")
    x = torch.tensor(data.strain(cfg), dtype=torch.float32, device="cuda")
    rf = _rf(cfg)
    refs = [g[0] for g in cfg.groups]
    z, _ = rf.mf_reference(x, ip, refs)
    kerns = [rf.build_ratio_kernels(r, nb, ip, cfg.threshold) for r, nb in cfg.groups]
    allL = np.concatenate([k.length for k in kerns])
    cut = int(np.median(allL)) + 1
    for k in kerns:
        k.prepare_buckets([0, cut], [4096, 32768], [1024, long_part])
    W = cfg.window
    P, A = rf.reconstruct_batched([z[g] for g in range(len(refs))], kerns, W)
    row = 0
    for g, k in enumerate(kerns):
        Pg, Ag = rf.reconstruct_winmax(z[g], k, W, "os")
        assert torch.equal(P[row:row + k.k], Pg) and torch.equal(A[row:row + k.k], Ag)
        row += k.k


def _cfg2_long(n=1 << 17, k=8, dmax=4.0):
    cfg = workload.config(2, n_override=n, k_override=k)
    ref = cfg.groups[0][0]
    nb = workload.duration_lattice(ref, cfg.f_low, k, 0.3, dmax, np.random.default_rng(3), n_eta=1)
    inj = (workload.Injection(2, 0, n // 3, 15.0),)
    return replace(cfg, groups=((ref, nb),), injections=inj)


def test_reconstruct_os_paper_shaped_kernels(torch):
    """Reconstruct-only: the oracle's z_ref and kernels (rounded to complex64) through
    overlap-save, against the oracle's FP64 direct sum of the same rounded inputs; and the
    whole GPU path (matched filter, builder, overlap-save) against the FP64 oracle."""
    cfg = _cfg2_long()
    ref, nb = cfg.groups[0]
    ip = workload.inv_psd(cfg)
    x = data.strain(cfg)
    zo_ref, _ = mf.matched_filter(x, ip, cfg.n, cfg.fs, cfg.f_low, cfg.f_high, ref.m1, ref.m2, cfg.pn_order)
    pk = ratio.build_ratio_kernels(ref, nb, cfg.n, cfg.fs, cfg.f_low, cfg.f_high, cfg.pn_order, ip, cfg.threshold)
    assert pk.length.max() > 4096          # several partitions at B = 8192
    rf = _rf(cfg)
    z32 = zo_ref.astype(np.complex64)
    kern = rf.kernels_import(pk.lag0, pk.length, pk.taps.astype(np.complex64))
    zh = [reconstruct.reconstruct_direct(z32.astype(np.complex128), pk.kernel(j)[0],
                                         pk.kernel(j)[1].astype(np.complex64)) for j in range(len(nb))]
    for B, Lp in ((2048, 1024), (8192, 4096), (8192, 2048), (16384, 2048)):
        kern.prepare(B, Lp)
        out = rf.reconstruct(torch.tensor(z32, device="cuda"), kern, "os").cpu().numpy()
        for j in range(len(nb)):
            assert _relerr(out[j], zh[j]) < TOL["f32"], (B, Lp, j)
    # the modelled layout choice is one of the allowed layouts
    kern.prepare()
    B, Lp = kern.os_layout()
    assert B in (512, 1024, 2048, 4096, 8192, 16384) and B <= cfg.n and Lp in (B // 2, B // 4, B // 8)
    # whole path
    ipt = torch.tensor(ip, device="cuda")
    zg, _ = rf.mf_reference(torch.tensor(x, dtype=torch.float32, device="cuda"), ipt, [ref])
    kg = rf.build_ratio_kernels(ref, nb, ipt, cfg.threshold)
    assert np.array_equal(kg.lag0, pk.lag0) and np.array_equal(kg.length, pk.length)
    out = rf.reconstruct(zg[0], kg, "auto").cpu().numpy()
    P, A = rf.reconstruct_winmax(zg[0], kg, cfg.window, "auto")
    P, A = P.cpu().numpy(), A.cpu().numpy()
    for j in range(len(nb)):
        zh = reconstruct.reconstruct_direct(zo_ref, *pk.kernel(j))
        assert _relerr(out[j], zh) < TOL["f32"], j
        Po, Ao = reconstruct.window_peaks(zh, cfg.window)
        assert np.abs(P[j] - Po).max() <= 4 * TOL["f32"] * Po.max()
        _argmax_ok(zh.real ** 2 + zh.imag ** 2, A[j], Ao, cfg.window, 8 * TOL["f32"] * Po.max())
    inj = cfg.injections[0]
    assert A[inj.template_index, inj.sample // cfg.window] == inj.sample


def test_full_size_paper_workload_sampled(torch):
    """The benchmark's workload at full size (n = 2^20, 256 neighbours) in the launch
    configuration the benchmark times; checked on sampled outputs computed one by one by
    the oracle, and by properties of the window peaks that hold at any size."""
    cfg = workload.config(2)
    ref, nb = cfg.groups[0]
    ip = workload.inv_psd(cfg)
    x = data.strain(cfg)
    rf = _rf(cfg)
    ipt = torch.tensor(ip, device="cuda")
    # as the benchmark runs it: stored reference filter, autotuned layout, AUTO reconstruction
    filt, _ = rf.reference_filters(ipt, [ref])
    zg = rf.mf_filtered(torch.tensor(x, dtype=torch.float32, device="cuda"), filt)
    kern = rf.build_ratio_kernels(ref, nb, ipt, cfg.threshold)
    rf.autotune([zg[0]], [kern], cfg.window, allow_split=True)
    P, A = rf.reconstruct_winmax(zg[0], kern, cfg.window, "auto")
    P, A = P.cpu().numpy(), A.cpu().numpy()
    zo_ref, _ = mf.matched_filter(x, ip, cfg.n, cfg.fs, cfg.f_low, cfg.f_high, ref.m1, ref.m2, cfg.pn_order)
    assert _relerr(zg[0].cpu().numpy(), zo_ref) < TOL["f32"]
    rng = np.random.default_rng(0)
    order = np.argsort(kern.length)
    sample = [int(order[0]), int(order[len(order) // 2]), int(order[-1])]
    pk = ratio.build_ratio_kernels(ref, [nb[j] for j in sample], cfg.n, cfg.fs, cfg.f_low, cfg.f_high,
                                   cfg.pn_order, ip, cfg.threshold)
    for q, j in enumerate(sample):
        assert kern.lag0[j] == pk.lag0[q] and kern.length[j] == pk.length[q]
        m0, c = pk.kernel(q)
        # the reported peak equals the oracle's value at the reported index ...
        wins = rng.choice(P.shape[1], 24, replace=False)
        vals = reconstruct.reconstruct_at(zo_ref, m0, c, A[j, wins])
        assert np.abs(P[j, wins] - np.abs(vals) ** 2).max() <= 4 * TOL["f32"] * P[j].max()
        # ... and no sampled sample of those windows exceeds it
        for w in wins[:6]:
            idx = w * cfg.window + rng.choice(cfg.window, 48, replace=False)
            v = np.abs(reconstruct.reconstruct_at(zo_ref, m0, c, idx)) ** 2
            assert np.all(v <= P[j, w] + 4 * TOL["f32"] * P[j].max())
    # the injections are recovered at their arrival samples
    for inj in cfg.injections:
        w = inj.sample // cfg.window
        assert abs(int(A[inj.template_index, w]) - inj.sample) <= 1


def test_long_segment_2p23_sampled(torch):
    """The long-duration workload's segment (n = 2^23, f_low = 5 Hz) for one reference and two
    neighbours 40-120 s away in duration (kernels of tens of thousands of taps): z_ref on sampled indices by the defining sum of
    Eq. 2, and the reconstructed window peaks at sampled windows by the defining sum of Eq. 8
    over the library's own z_ref and taps."""
    base = workload.config(5, k_override=2)
    ref = base.groups[0][0]
    nb = workload.duration_lattice(ref, base.f_low, 2, 40.0, 120.0, np.random.default_rng(55), n_eta=1,
                                   eta_range=(0.24, 0.25), mrange=(2.0, 3.0))
    cfg = replace(base, groups=((ref, nb),) + base.groups[1:])
    n, fs, W = cfg.n, cfg.fs, cfg.window
    ip = workload.inv_psd(cfg)
    x = data.strain(cfg)
    rf = _rf(cfg)
    ipt = torch.tensor(ip, device="cuda")
    filt, _ = rf.reference_filters(ipt, [ref])
    zg = rf.mf_filtered(torch.tensor(x, dtype=torch.float32, device="cuda"), filt)
    kern = rf.build_ratio_kernels(ref, nb, ipt, 3e-5)    # the benchmark's relative threshold
    assert kern.length.max() > 1 << 15                    # many partitions at any layout
    rf.autotune([zg[0]], [kern], W)
    P, A = rf.reconstruct_winmax(zg[0], kern, W, "auto")
    P, A = P.cpu().numpy(), A.cpu().numpy()
    z = zg[0].cpu().numpy().astype(np.complex128)
    rng = np.random.default_rng(5)
    # z_ref against Eq. 2 on sampled indices (the data spectrum as constructed)
    xf = workload.noise_spectrum(cfg, 0) + data.injection_spectrum(cfg, ip)
    ipb = mf.band_limited_inv_psd(ip, n, fs, cfg.f_low, cfg.f_high)
    h = mf.template(n, fs, ref.m1, ref.m2, cfg.pn_order)
    idx = rng.choice(n, 8, replace=False)
    zs = mf.snr_at(xf, h, ipb, n, fs, idx)
    assert np.abs(z[idx] - zs).max() <= 4 * TOL["f32"] * np.abs(z).max()
    # reconstruction against Eq. 8 on sampled windows
    taps = kern.taps().cpu().numpy().astype(np.complex128)
    for j in range(kern.k):
        c = taps[kern.offset[j]:kern.offset[j + 1]]
        wins = rng.choice(P.shape[1], 6, replace=False)
        vals = reconstruct.reconstruct_at(z, int(kern.lag0[j]), c, A[j, wins])
        assert np.abs(P[j, wins] - np.abs(vals) ** 2).max() <= 4 * TOL["f32"] * P[j].max()
        for w in wins[:2]:
            ii = w * W + rng.choice(min(W, n - w * W), 16, replace=False)
            v = np.abs(reconstruct.reconstruct_at(z, int(kern.lag0[j]), c, ii)) ** 2
            assert np.all(v <= P[j, w] + 4 * TOL["f32"] * P[j].max())


# ---------------------------------------------------------------- batched form

def _batch_cfg(n=1 << 15):
    """Three references of the batched workload with uneven neighbour counts."""
    base = workload.config(4, n_override=n, k_override=24)
    rng = np.random.default_rng(44)
    groups = []
    for g, k in enumerate((2, 5, 3)):
        ref = base.groups[g][0]
        nb = workload.duration_lattice(ref, base.f_low, k, 0.05, 3.0, rng, eta_range=(0.235, 0.25), n_eta=1)
        groups.append((ref, nb))
    return replace(base, groups=tuple(groups), injections=(workload.Injection(1, 1, n // 2, 12.0),))


def test_reconstruct_batched_matches_per_group_and_oracle(torch):
    cfg = _batch_cfg()
    ip = workload.inv_psd(cfg)
    x = data.strain(cfg)
    rf = _rf(cfg)
    ipt = torch.tensor(ip, device="cuda")
    refs = [g[0] for g in cfg.groups]
    z, _ = rf.mf_reference(torch.tensor(x, dtype=torch.float32, device="cuda"), ipt, refs)
    kerns = [rf.build_ratio_kernels(r, nb, ipt, cfg.threshold) for r, nb in cfg.groups]
    W = cfg.window
    P, A = rf.reconstruct_batched([z[g] for g in range(len(refs))], kerns, W)
    P2, A2 = rf.reconstruct_batched([z[g] for g in range(len(refs))], kerns, W)   # cached plan
    assert torch.equal(P, P2) and torch.equal(A, A2)
    row = 0
    for g, (ref, nb) in enumerate(cfg.groups):
        Pg, Ag = rf.reconstruct_winmax(z[g], kerns[g], W, "os")
        assert torch.equal(P[row:row + len(nb)], Pg) and torch.equal(A[row:row + len(nb)], Ag)
        zo, _ = mf.matched_filter(x, ip, cfg.n, cfg.fs, cfg.f_low, cfg.f_high, ref.m1, ref.m2, cfg.pn_order)
        pk = ratio.build_ratio_kernels(ref, nb, cfg.n, cfg.fs, cfg.f_low, cfg.f_high, cfg.pn_order, ip,
                                       cfg.threshold)
        for j in range(len(nb)):
            zh = reconstruct.reconstruct_direct(zo, *pk.kernel(j))
            Po, Ao = reconstruct.window_peaks(zh, W)
            Pj, Aj = P[row + j].cpu().numpy(), A[row + j].cpu().numpy()
            assert np.abs(Pj - Po).max() <= 4 * TOL["f32"] * Po.max()
            _argmax_ok(zh.real ** 2 + zh.imag ** 2, Aj, Ao, W, 8 * TOL["f32"] * Po.max())
        row += len(nb)
    # a re-prepared kernel set (other block size) invalidates the cached plan
    for k in kerns:
        k.prepare(2048)
    P3, A3 = rf.reconstruct_batched([z[g] for g in range(len(refs))], kerns, W)
    assert torch.allclose(P3, P, rtol=4 * TOL["f32"], atol=4 * TOL["f32"] * P.max().item())


@pytest.mark.parametrize("algo,prec", [("direct", "native"), ("gemm", "bf16x6")])
def test_reconstruct_batched_other_forms_match_per_group(torch, algo, prec):
    """The batched entry with the direct or tensor-core form writes, group after group, the
    same rows as the per-group calls."""
    cfg = _batch_cfg()
    ip = torch.tensor(workload.inv_psd(cfg), device="cuda")
    x = torch.tensor(data.strain(cfg), dtype=torch.float32, device="cuda")
    rf = _rf(cfg)
    refs = [g[0] for g in cfg.groups]
    z, _ = rf.mf_reference(x, ip, refs)
    kerns = [rf.build_ratio_kernels(r, nb, ip, cfg.threshold) for r, nb in cfg.groups]
    W = cfg.window
    P, A = rf.reconstruct_batched([z[g] for g in range(len(refs))], kerns, W, algo, prec=prec)
    row = 0
    for g, k in enumerate(kerns):
        Pg, Ag = rf.reconstruct_winmax(z[g], k, W, algo, prec=prec)
        assert torch.equal(P[row:row + k.k], Pg) and torch.equal(A[row:row + k.k], Ag)
        row += k.k
    assert row == P.shape[0]


@pytest.mark.parametrize("algo,prec", [("os", "native"), ("direct", "native"), ("gemm", "bf16x6")])
def test_reconstruct_batched_with_an_empty_group(torch, algo, prec):
    """A reference without dependents (a one-template set of a structured bank) between two
    groups: no rows of its own, the other groups' rows as in their own calls."""
    cfg = _batch_cfg()
    groups = (cfg.groups[0], (cfg.groups[1][0], ()), cfg.groups[2])
    cfg = replace(cfg, groups=groups, injections=())
    ip = torch.tensor(workload.inv_psd(cfg), device="cuda")
    x = torch.tensor(data.strain(cfg), dtype=torch.float32, device="cuda")
    rf = _rf(cfg)
    refs = [g[0] for g in cfg.groups]
    z, _ = rf.mf_reference(x, ip, refs)
    kerns = [rf.build_ratio_kernels(r, nb, ip, cfg.threshold) for r, nb in cfg.groups]
    assert kerns[1].k == 0
    W = cfg.window
    P, A = rf.reconstruct_batched([z[g] for g in range(len(refs))], kerns, W, algo, prec=prec)
    assert P.shape[0] == kerns[0].k + kerns[2].k
    row = 0
    for g, k in enumerate(kerns):
        if k.k:
            Pg, Ag = rf.reconstruct_winmax(z[g], k, W, algo, prec=prec)
            assert torch.equal(P[row:row + k.k], Pg) and torch.equal(A[row:row + k.k], Ag)
        row += k.k


def test_stream_winmax_equals_the_segment_calls(torch):
    """Streaming over a strain 2.5 segment hops long: every window equals the one the
    segment whose interior holds it gives through the per-segment calls (stored-filter matched
    filter, reference peaks, batched reconstruction), argmax shifted to stream indices; the
    stream's first window comes from a segment starting guard samples before the data."""
    cfg = _batch_cfg()
    n, W = cfg.n, 2048
    guard = 2 * W
    hop = n - 2 * guard
    total = 5 * hop // 2 // W * W
    rng = np.random.default_rng(51)
    x = rng.standard_normal(total).astype(np.float32)
    ip = torch.tensor(workload.inv_psd(cfg), device="cuda")
    rf = _rf(cfg)
    refs = [g[0] for g in cfg.groups]
    filt, _ = rf.reference_filters(ip, refs)
    kerns = [rf.build_ratio_kernels(r, nb, ip, cfg.threshold) for r, nb in cfg.groups]
    rm, ra, nm, na = rf.stream_winmax(x, filt, kerns, W, guard)
    nwt = total // W
    assert rm.shape == (len(refs), nwt) and nm.shape == (sum(k.k for k in kerns), nwt)
    seen = np.zeros(nwt, bool)
    q = 0
    while q * hop < nwt * W:
        s0 = q * hop - guard
        seg = np.zeros(n, np.float32)
        a, b = max(0, s0), min(total, s0 + n)
        seg[a - s0:b - s0] = x[a:b]
        z = rf.mf_filtered(torch.tensor(seg, device="cuda"), filt)
        Pr, Ar = rf.winmax(z, W)
        Pn, An = rf.reconstruct_batched([z[g] for g in range(len(refs))], kerns, W)
        for wl in range(guard // W, (n - guard) // W):
            w = (s0 + wl * W) // W
            if 0 <= w < nwt:
                assert not seen[w]
                seen[w] = True
                assert np.array_equal(rm[:, w], Pr[:, wl].cpu().numpy())
                assert np.array_equal(ra[:, w], s0 + Ar[:, wl].cpu().numpy().astype(np.int64))
                assert np.array_equal(nm[:, w], Pn[:, wl].cpu().numpy())
                assert np.array_equal(na[:, w], s0 + An[:, wl].cpu().numpy().astype(np.int64))
        q += 1
    assert seen.all() and q == 3


def test_batched_step_captures_in_a_cuda_graph(torch):
    """After a warm-up call, the whole online step (matched filter of every reference,
    reference peaks, batched reconstruction) replays from a CUDA graph with the same result."""
    cfg = _batch_cfg()
    ip = torch.tensor(workload.inv_psd(cfg), device="cuda")
    x = torch.tensor(data.strain(cfg), dtype=torch.float32, device="cuda")
    rf = _rf(cfg)
    refs = [g[0] for g in cfg.groups]
    kerns = [rf.build_ratio_kernels(r, nb, ip, cfg.threshold) for r, nb in cfg.groups]
    G, n, W = len(refs), cfg.n, cfg.window
    nw = -(-n // W)
    z = torch.empty((G, n), dtype=torch.complex64, device="cuda")
    sg = torch.empty(G, dtype=torch.float64, device="cuda")
    rows = sum(k.k for k in kerns)
    P = torch.empty((rows, nw), dtype=torch.float32, device="cuda")
    A = torch.empty((rows, nw), dtype=torch.int32, device="cuda")
    Pr = torch.empty((G, nw), dtype=torch.float32, device="cuda")
    Ar = torch.empty((G, nw), dtype=torch.int32, device="cuda")
    rf.reserve(rows)

    def step():
        rf.mf_reference(x, ip, refs, z_out=z, sigma_out=sg)
        rf.winmax(z, W, max_out=Pr, arg_out=Ar)
        rf.reconstruct_batched([z[g] for g in range(G)], kerns, W, max_out=P, arg_out=A)

    s = torch.cuda.Stream()
    s.wait_stream(torch.cuda.current_stream())
    with torch.cuda.stream(s):
        step()
    torch.cuda.current_stream().wait_stream(s)
    torch.cuda.synchronize()
    P0, A0, Pr0 = P.clone(), A.clone(), Pr.clone()
    P.zero_(); A.zero_(); Pr.zero_()
    graph = torch.cuda.CUDAGraph()
    with torch.cuda.graph(graph):
        step()
    graph.replay()
    torch.cuda.synchronize()
    assert torch.equal(P, P0) and torch.equal(A, A0) and torch.equal(Pr, Pr0)


# ---------------------------------------------------------------- tensor-core direct form

# Error bars of the split-BF16 products relative to max|z| (x = x0 + x1 + x2, u = 2^-9 the BF16
# unit roundoff of each term): the dropped products are O(u) for BF16, O(u^2) for x3, and O(u^3)
# for x6/x9, where the FP32 accumulation (about 1e-7 of the running sum) dominates.  3xTF32
# (u = 2^-11 per TF32 term, two terms) drops x1 y1 and both split residuals, 3 u^2 = 7e-7 of
# |x||y| per product at most.
GEMM_TOL = {"bf16": 2e-2, "bf16x3": 2e-4, "bf16x6": 2e-6, "bf16x9": 2e-6, "3xtf32": 2e-6}


@pytest.mark.parametrize("dtype", ["f32", "f64"])
def test_reconstruct_gemm_edge_lengths(torch, dtype):
    n = 1 << 13
    rng = np.random.default_rng(17)
    lengths = [1, 2, 15, 16, 17, 100, 255, 256, 257, 384, 0, 500, 31, 1000, 600]
    lags = [0, -5, 37, n // 2, -(n // 2) + 1, 100, -1000, 3, 2000, -2, 5, 11, -n // 4, -400, 4000]
    cfg = replace(workload.config(1, n_override=n, k_override=1), dtype=dtype)
    rf = _rf(cfg)
    cdt = np.complex64 if dtype == "f32" else np.complex128
    z = (rng.standard_normal(n) + 1j * rng.standard_normal(n)).astype(cdt)
    taps = [((rng.standard_normal(L) + 1j * rng.standard_normal(L)) / np.sqrt(max(L, 1))).astype(cdt)
            for L in lengths]
    kern = rf.kernels_import(lags, lengths, np.concatenate(taps))
    zt = torch.tensor(z, device="cuda")
    zo = [reconstruct.reconstruct_direct(z.astype(np.complex128), lags[j], taps[j].astype(np.complex128))
          for j in range(len(lengths))]
    errs = {}
    for prec, tol in GEMM_TOL.items():
        out = rf.reconstruct(zt, kern, "gemm", prec=prec).cpu().numpy()
        rf.device_status()
        worst = 0.0
        for j, L in enumerate(lengths):
            if L == 0:
                assert np.abs(out[j]).max() == 0.0
                continue
            worst = max(worst, _relerr(out[j], zo[j]))
        errs[prec] = worst
        assert worst < tol, (prec, worst)
        P, A = rf.reconstruct_winmax(zt, kern, 1000, "gemm", prec=prec)
        P, A = P.cpu().numpy(), A.cpu().numpy()
        for j, L in enumerate(lengths):
            if L == 0:
                continue
            Po, Ao = reconstruct.window_peaks(zo[j], 1000)
            assert np.abs(P[j] - Po).max() <= 4 * tol * Po.max()
            _argmax_ok(zo[j].real ** 2 + zo[j].imag ** 2, A[j], Ao, 1000, 8 * tol * Po.max())
    # each extra set of products improves the result; two TF32 terms resolve about 2^-22
    assert errs["bf16x3"] < errs["bf16"] / 10 and errs["bf16x6"] < errs["bf16x3"] / 10
    assert errs["3xtf32"] < errs["bf16x3"] / 10


def test_reconstruct_gemm_precision_form_workload(torch):
    """The precision-form workload: the FP64 small configuration's data and bank through the
    tensor-core form, every split precision against the FP64 oracle."""
    cfg = workload.config(3)
    ref, nb = cfg.groups[0]
    ip = workload.inv_psd(cfg)
    x = data.strain(cfg)
    rf = _rf(cfg)
    ipt = torch.tensor(ip, device="cuda")
    z, _ = rf.mf_reference(torch.tensor(x, device="cuda"), ipt, [ref])
    kern = rf.build_ratio_kernels(ref, nb, ipt, cfg.threshold)
    zo, _ = mf.matched_filter(x, ip, cfg.n, cfg.fs, cfg.f_low, cfg.f_high, ref.m1, ref.m2, cfg.pn_order)
    pk = ratio.build_ratio_kernels(ref, nb, cfg.n, cfg.fs, cfg.f_low, cfg.f_high, cfg.pn_order, ip, cfg.threshold)
    zh = [reconstruct.reconstruct_direct(zo, *pk.kernel(j)) for j in range(len(nb))]
    for prec, tol in GEMM_TOL.items():
        out = rf.reconstruct(z[0], kern, "gemm", prec=prec).cpu().numpy()
        worst = max(_relerr(out[j], zh[j]) for j in range(len(nb)))
        assert worst < tol, (prec, worst)
    P, A = rf.reconstruct_winmax(z[0], kern, cfg.window, "gemm", prec="bf16x6")
    inj = cfg.injections[0]
    assert A[inj.template_index, inj.sample // cfg.window].item() == inj.sample


# Output tiles stacked along N for sets of at most 16 neighbours: the widest stack whose MMA of
# the leading A term fits N = 256 (S x 32 columns per B term) and whose product-order column
# groups fit tensor memory (bf16x9 keeps one group per product, 9 x 32 x S <= 512).
GEMM_SHIFTS = {"bf16": 8, "bf16x3": 4, "bf16x6": 2, "bf16x9": 1, "3xtf32": 4}


@pytest.mark.parametrize("n", [512, 1 << 12])
def test_reconstruct_gemm_stacked_tiles(torch, n):
    """Few neighbours with kernels longer than a tile: the output-shift stack, including a
    segment shorter than one stacked super-tile (n = 512 < 8 x 128), against the oracle."""
    rng = np.random.default_rng(29)
    lengths = [300, 129, 5, 257]
    lags = [0, -n // 2 + 1, 17, n // 3]
    cfg = replace(workload.config(1, n_override=n, k_override=1), dtype="f32")
    rf = _rf(cfg)
    z = (rng.standard_normal(n) + 1j * rng.standard_normal(n)).astype(np.complex64)
    taps = [((rng.standard_normal(L) + 1j * rng.standard_normal(L)) / np.sqrt(L)).astype(np.complex64)
            for L in lengths]
    kern = rf.kernels_import(lags, lengths, np.concatenate(taps))
    zt = torch.tensor(z, device="cuda")
    zo = [reconstruct.reconstruct_direct(z.astype(np.complex128), lags[j], taps[j].astype(np.complex128))
          for j in range(len(lengths))]
    for prec, tol in GEMM_TOL.items():
        out = rf.reconstruct(zt, kern, "gemm", prec=prec).cpu().numpy()
        lay = kern.gemm_layout()
        assert lay["prec"] == prec and lay["nj"] == 16 and lay["shifts"] == GEMM_SHIFTS[prec], lay
        assert lay["kc"] * lay["nck"] == lay["lp"] + 128 * (lay["shifts"] - 1) and lay["lp"] >= 300
        worst = max(_relerr(out[j], zo[j]) for j in range(len(lengths)))
        assert worst < tol, (prec, worst)
        P, A = rf.reconstruct_winmax(zt, kern, 100, "gemm", prec=prec)
        P, A = P.cpu().numpy(), A.cpu().numpy()
        for j in range(len(lengths)):
            Po, Ao = reconstruct.window_peaks(zo[j], 100)
            assert np.abs(P[j] - Po).max() <= 4 * tol * Po.max()
            _argmax_ok(zo[j].real ** 2 + zo[j].imag ** 2, A[j], Ao, 100, 8 * tol * Po.max())


def test_reconstruct_gemm_short_kernels_small_set(torch):
    """At most 16 neighbours whose kernels fit one tile take the widest groups without stacked
    tiles; results against the oracle."""
    n = 1 << 12
    rng = np.random.default_rng(31)
    lengths = [1, 64, 128, 100, 7]
    lags = [3, -9, 0, 200, -1000]
    cfg = replace(workload.config(1, n_override=n, k_override=1), dtype="f32")
    rf = _rf(cfg)
    z = (rng.standard_normal(n) + 1j * rng.standard_normal(n)).astype(np.complex64)
    taps = [((rng.standard_normal(L) + 1j * rng.standard_normal(L)) / np.sqrt(L)).astype(np.complex64)
            for L in lengths]
    kern = rf.kernels_import(lags, lengths, np.concatenate(taps))
    zt = torch.tensor(z, device="cuda")
    zo = [reconstruct.reconstruct_direct(z.astype(np.complex128), lags[j], taps[j].astype(np.complex128))
          for j in range(len(lengths))]
    for prec, tol in GEMM_TOL.items():
        out = rf.reconstruct(zt, kern, "gemm", prec=prec).cpu().numpy()
        lay = kern.gemm_layout()
        assert lay["shifts"] == 1 and lay["nj"] > 16, lay
        worst = max(_relerr(out[j], zo[j]) for j in range(len(lengths)))
        assert worst < tol, (prec, worst)


def test_reconstruct_gemm_wide_groups(torch):
    """More neighbours than one 16-wide group: the widest tensor-core tiles (all split terms of
    a group side by side in N) against the oracle, with a ragged last group."""
    n = 1 << 12
    rng = np.random.default_rng(23)
    k = 101
    lengths = list(rng.integers(1, 300, k))
    lags = list(rng.integers(-n // 2 + 1, n // 2, k))
    cfg = replace(workload.config(1, n_override=n, k_override=1), dtype="f32")
    rf = _rf(cfg)
    z = (rng.standard_normal(n) + 1j * rng.standard_normal(n)).astype(np.complex64)
    taps = [((rng.standard_normal(L) + 1j * rng.standard_normal(L)) / np.sqrt(L)).astype(np.complex64)
            for L in lengths]
    kern = rf.kernels_import(lags, lengths, np.concatenate(taps))
    zt = torch.tensor(z, device="cuda")
    zo = [reconstruct.reconstruct_direct(z.astype(np.complex128), int(lags[j]), taps[j].astype(np.complex128))
          for j in range(k)]
    for prec, tol in GEMM_TOL.items():
        out = rf.reconstruct(zt, kern, "gemm", prec=prec).cpu().numpy()
        worst = max(_relerr(out[j], zo[j]) for j in range(k))
        assert worst < tol, (prec, worst)
    P, A = rf.reconstruct_winmax(zt, kern, 512, "gemm", prec="bf16x6")
    P, A = P.cpu().numpy(), A.cpu().numpy()
    for j in range(0, k, 7):
        Po, Ao = reconstruct.window_peaks(zo[j], 512)
        assert np.abs(P[j] - Po).max() <= 4 * GEMM_TOL["bf16x6"] * Po.max()
        _argmax_ok(zo[j].real ** 2 + zo[j].imag ** 2, A[j], Ao, 512, 8 * GEMM_TOL["bf16x6"] * Po.max())


def test_bounded_wait_timeout_is_reported_and_context_survives(torch):
    """A device-side wait that runs out (a barrier nothing arrives on, short limit) is
    reported as RF_ETIMEOUT by the next status call, cleared, and the context keeps working."""
    from paper_2511_12894_gb300 import RF_ETIMEOUT, RFError
    cfg = _small_f32_cfg(1 << 12, 2)
    rf = _rf(cfg)
    rf.device_status()                       # clean to begin with
    rf.selftest_bounded_wait()
    with pytest.raises(RFError) as e:
        rf.device_status()
    assert e.value.status == RF_ETIMEOUT
    rf.device_status()                       # cleared
    ref = cfg.groups[0][0]
    ip = workload.inv_psd(cfg)
    x = data.strain(cfg)
    z, _ = rf.mf_reference(torch.tensor(x, dtype=torch.float32, device="cuda"), torch.tensor(ip, device="cuda"), [ref])
    zo, _ = mf.matched_filter(x, ip, cfg.n, cfg.fs, cfg.f_low, cfg.f_high, ref.m1, ref.m2, cfg.pn_order)
    assert _relerr(z[0].cpu().numpy(), zo) < TOL["f32"]


def test_autotune_records_the_fastest_form_and_auto_follows_it(torch):
    """The autotuner times overlap-save layouts and buckets (single-pass and two-phase), the
    tensor-core form, mixed forms and the direct sum on a batch, records the fastest, and AUTO
    then gives the same rows as that form called explicitly; on an FP64 grid without split
    precisions only the exact direct sum competes."""
    cfg = _batch_cfg()
    ip = torch.tensor(workload.inv_psd(cfg), device="cuda")
    x = torch.tensor(data.strain(cfg), dtype=torch.float32, device="cuda")
    rf = _rf(cfg)
    refs = [g[0] for g in cfg.groups]
    z, _ = rf.mf_reference(x, ip, refs)
    kerns = [rf.build_ratio_kernels(r, nb, ip, cfg.threshold) for r, nb in cfg.groups]
    W = cfg.window
    zs = [z[g] for g in range(len(refs))]
    table = rf.autotune(zs, kerns, W, allow_split=True, max_os=3)
    assert len(table) >= 3 and all(e["ms"] > 0 for e in table)
    assert sum(e["algo"] == "os" and e["cut"] == 0 for e in table) == 3       # single layouts
    assert all(e["block2"] and e["part2"] for e in table if e["cut"])          # two-bucket variants
    assert {e["algo"] for e in table} <= {"os", "os_bins", "gemm", "direct"}
    win = table[0]
    assert win["ms"] == min(e["ms"] for e in table)
    # a bucketed winner (overlap-save, two-phase or mixed) is prepared bucket by bucket
    bucketed = bool(win["cut"]) or win["algo"] in ("os", "os_bins")
    if bucketed:
        want = [(0, win["block"], win["part"])]
        forms = [(win["algo"], win["prec"])]
        if win["cut"]:
            want.append((win["cut"], win["block2"], win["part2"]))
            forms.append((win["algo2"], "native"))
        if win["cut3"]:
            want.append((win["cut3"], win["block3"], win["part3"]))
            forms.append((win["algo3"], "native"))
        assert all(k.os_buckets() == want and k.bucket_forms() == forms for k in kerns)
    P, A = rf.reconstruct_batched(zs, kerns, W)                       # AUTO -> the tuned form
    P2, A2 = rf.reconstruct_batched(zs, kerns, W, "os" if bucketed else win["algo"],
                                    prec="native" if bucketed else win["prec"])
    assert torch.equal(P, P2) and torch.equal(A, A2)
    # FP64 grid, exact forms only
    c1 = workload.config(1, n_override=1 << 13, k_override=3)
    r1 = _rf(c1)
    ref, nb = c1.groups[0]
    ip1 = torch.tensor(workload.inv_psd(c1), device="cuda")
    z1, _ = r1.mf_reference(torch.tensor(data.strain(c1), device="cuda"), ip1, [ref])
    k1 = r1.build_ratio_kernels(ref, nb, ip1, c1.threshold)
    t1 = r1.autotune([z1[0]], [k1], c1.window)
    assert [e["algo"] for e in t1] == ["direct"]
