"""Parity with the FP64 oracle at the sizes the benchmark runs.

The batched workload at full size (64 references, about 16k neighbours, n = 2^20), the
long-duration workload (n = 2^23, f_low = 5 Hz, 128 x 128, kernels on per-neighbour build
grids), streaming over data longer than one segment, and the tensor-core form at kernels of
up to 4096 taps.  The oracle cannot compute every output at these sizes, so each check takes
sampled rows and windows: the kernel spans exactly, the taps to their FP32 rounding (FP64
builds to the rounding of their phases), the reported window peak against the oracle's
direct sum of Eq. 8 at the reported index (2e-6 of the row's max|z|, on |z|), no sampled
output of a window above the reported peak, and the argmax where the window's top two
values differ by more than the error bound (elsewhere any index within it).
"""
from dataclasses import replace

import numpy as np
import pytest

import workload
from oracle import data, mf, ratio, reconstruct

pytestmark = pytest.mark.gpu

TOL32 = 2e-6
# |c32 - c64| for an FP64 value rounded to complex64: half an ulp per part
F32_ROUND = 2.0 ** -24 * np.sqrt(2.0)


@pytest.fixture(scope="module")
def torch():
    import torch as t
    if not t.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2511_12894_gb300 import build
    build.build()
    return t


def _rf(cfg, dtype=None):
    from paper_2511_12894_gb300 import RatioFilter
    return RatioFilter.from_config(cfg if dtype is None else replace(cfg, dtype=dtype))


def _fp64_phase_bound(cfg, ref):
    """Relative bound on FP64 taps: the phases reach |Psi| ~ 1e5 rad at the lowest build
    frequency (f_low - df_low), and dPsi = Psi_j - Psi_ref carries a few ulp(|Psi|) of absolute
    rounding on each side, which the kernel inherits as a relative error; never below 1e-12."""
    from oracle import taylorf2
    f = np.array([max(cfg.f_low - min(cfg.df_low_max, cfg.f_low / 2), 1e-3)])
    psi = float(np.abs(taylorf2.phase(f, ref.m1, ref.m2, cfg.pn_order, 0.0, 0.0)).max())
    return max(1e-12, 64 * 2.0 ** -52 * psi)


def _check_taps(kern, j, c_oracle, tol64=1e-12):
    c = kern.taps()[int(kern.offset[j]):int(kern.offset[j + 1])].cpu().numpy().astype(np.complex128)
    assert c.shape == c_oracle.shape
    scale = np.abs(c_oracle).max()
    assert np.all(np.abs(c - c_oracle) <= F32_ROUND * np.abs(c_oracle) + tol64 * scale)


def _check_row_peaks(P, A, zo, m0, c, W, rng, nwin=8, nprobe=3, per_win=32):
    """Peaks of one row against the oracle's direct sum at sampled windows."""
    n = zo.shape[0]
    nw = P.shape[0]
    zmax = np.sqrt(P.max())
    wins = rng.choice(nw, min(nw, nwin), replace=False)
    vals = np.abs(reconstruct.reconstruct_at(zo, m0, c, A[wins].astype(np.int64)))
    assert np.all((A[wins] >= wins * W) & (A[wins] < np.minimum(n, (wins + 1) * W)))
    err = np.abs(np.sqrt(P[wins]) - vals).max()
    assert err <= TOL32 * zmax, (err / zmax)
    for w in wins[:nprobe]:
        idx = w * W + rng.choice(min(W, n - w * W), per_win, replace=False)
        v = np.abs(reconstruct.reconstruct_at(zo, m0, c, idx))
        assert np.all(v <= np.sqrt(P[w]) + TOL32 * zmax)
    return err / zmax


def _window_argmax_ok(P, A, zo, m0, c, w, W, zmax):
    """The whole window by the oracle: the peak and, outside near-ties, its index."""
    n = zo.shape[0]
    idx = np.arange(w * W, min(n, (w + 1) * W), dtype=np.int64)
    v = np.abs(reconstruct.reconstruct_at(zo, m0, c, idx)) ** 2
    order = np.argsort(v)
    assert abs(np.sqrt(P[w]) - np.sqrt(v[order[-1]])) <= TOL32 * zmax
    bound = 4.0 * TOL32 * zmax * np.sqrt(v[order[-1]])
    if v[order[-1]] - v[order[-2]] > bound:
        assert A[w] == idx[order[-1]]
    else:
        assert v[A[w] - w * W] >= v[order[-1]] - bound


def test_batched_full_size_64_references(torch):
    """The batched workload at full size in one persistent launch per length bucket (the
    autotuner's layouts for it): sampled rows of the first, a middle and the last group (the
    shortest, median and longest kernel and the group's last row, so the row offsets of the
    whole work list are exercised) against oracle-built kernels and the oracle's z_ref."""
    cfg = workload.config(4)
    G = len(cfg.groups)
    assert G == 64 and sum(len(nb) for _, nb in cfg.groups) > 15000
    refs = [g[0] for g in cfg.groups]
    ip = workload.inv_psd(cfg)
    x = data.strain(cfg)
    rf = _rf(cfg)
    ipt = torch.tensor(ip, device="cuda")
    filt, _ = rf.reference_filters(ipt, refs)
    zg = rf.mf_filtered(torch.tensor(x, dtype=torch.float32, device="cuda"), filt)
    kerns = [rf.build_ratio_kernels(r, nb, ipt, 3e-5) for r, nb in cfg.groups]
    for k in kerns:
        k.prepare_buckets([0, 2048], [4096, 16384], [1024, 4096])
    P, A = rf.reconstruct_batched([zg[g] for g in range(G)], kerns, cfg.window)
    P, A = P.cpu().numpy(), A.cpu().numpy()
    row0 = np.cumsum([0] + [k.k for k in kerns])
    assert P.shape[0] == row0[-1]
    rng = np.random.default_rng(64)
    worst = 0.0
    for g in (0, G // 2, G - 1):
        ref, nb = cfg.groups[g]
        kern = kerns[g]
        zo, _ = mf.matched_filter(x, ip, cfg.n, cfg.fs, cfg.f_low, cfg.f_high, ref.m1, ref.m2, cfg.pn_order)
        assert np.abs(zg[g].cpu().numpy() - zo).max() <= TOL32 * np.abs(zo).max()
        order = np.argsort(kern.length)
        sample = sorted({int(order[0]), int(order[len(order) // 2]), int(order[-1]), kern.k - 1})
        pk = ratio.build_ratio_kernels(ref, [nb[j] for j in sample], cfg.n, cfg.fs, cfg.f_low, cfg.f_high,
                                       cfg.pn_order, ip, 3e-5)
        for q, j in enumerate(sample):
            assert kern.lag0[j] == pk.lag0[q] and kern.length[j] == pk.length[q]
            m0, c = pk.kernel(q)
            _check_taps(kern, j, c)
            r = row0[g] + j
            worst = max(worst, _check_row_peaks(P[r], A[r], zo, m0, c, cfg.window, rng))
    assert worst <= TOL32


def test_long_segment_full_size_oracle_kernels(torch):
    """The long-duration workload (n = 2^23, 128 references x 128 neighbours) as the benchmark
    runs it: kernels on per-neighbour build grids, two overlap-save buckets, the batched launch
    over all 16,384 rows.  For sampled neighbours of two groups the FP64 builder's spans equal
    the oracle's and its taps agree to the FP64 rounding of phases of 1e5 rad (a few 1e-9 of
    the largest tap; 1e-12 where the phases are small); the FP32 build's taps are their FP32
    rounding; the window peaks match the oracle's direct sum on its own z_ref; an injection's
    window has the oracle's peak and argmax."""
    cfg = workload.config(5)
    G = len(cfg.groups)
    refs = [g[0] for g in cfg.groups]
    ip = workload.inv_psd(cfg)
    x = data.strain(cfg)
    rf = _rf(cfg)
    ipt = torch.tensor(ip, device="cuda")
    filt, _ = rf.reference_filters(ipt, refs)
    zg = rf.mf_filtered(torch.tensor(x, dtype=torch.float32, device="cuda"), filt)
    kerns = [rf.build_ratio_kernels(r, nb, ipt, 3e-5, n_build=-1) for r, nb in cfg.groups]
    for k in kerns:
        k.prepare_buckets([0, 8192], [16384, 16384], [4096, 8192])
    P, A = rf.reconstruct_batched([zg[g] for g in range(G)], kerns, cfg.window)
    P, A = P.cpu().numpy(), A.cpu().numpy()
    row0 = np.cumsum([0] + [k.k for k in kerns])
    rf64 = _rf(cfg, "f64")
    rng = np.random.default_rng(23)
    inj_groups = sorted({inj.group for inj in cfg.injections})
    for g in (inj_groups[0], G - 1):
        ref, nb = cfg.groups[g]
        kern = kerns[g]
        tol64 = _fp64_phase_bound(cfg, ref)
        zo, _ = mf.matched_filter(x, ip, cfg.n, cfg.fs, cfg.f_low, cfg.f_high, ref.m1, ref.m2, cfg.pn_order)
        order = np.argsort(kern.length)
        sample = sorted({int(order[0]), int(order[len(order) // 2]), int(order[-1])})
        inj_here = [inj for inj in cfg.injections if inj.group == g and inj.template_index >= 0]
        sample = sorted(set(sample) | {inj.template_index for inj in inj_here[:1]})
        pk = ratio.build_ratio_kernels(ref, [nb[j] for j in sample], cfg.n, cfg.fs, cfg.f_low, cfg.f_high,
                                       cfg.pn_order, ip, 3e-5, n_build=-1)
        k64 = rf64.build_ratio_kernels(ref, [nb[j] for j in sample], ipt, 3e-5, n_build=-1)
        t64 = k64.taps().cpu().numpy()
        assert np.array_equal(k64.lag0, pk.lag0) and np.array_equal(k64.length, pk.length)
        for q, j in enumerate(sample):
            m0, c = pk.kernel(q)
            c64 = t64[int(k64.offset[q]):int(k64.offset[q + 1])]
            assert np.abs(c64 - c).max() <= tol64 * np.abs(c).max()
            assert kern.lag0[j] == pk.lag0[q] and kern.length[j] == pk.length[q]
            _check_taps(kern, j, c, tol64)
            r = row0[g] + j
            _check_row_peaks(P[r], A[r], zo, m0, c, cfg.window, rng, nwin=6, nprobe=2, per_win=16)
        for inj in inj_here[:1]:
            q = sample.index(inj.template_index)
            m0, c = pk.kernel(q)
            r = row0[g] + inj.template_index
            w = inj.sample // cfg.window
            _window_argmax_ok(P[r], A[r], zo, m0, c, w, cfg.window, np.sqrt(P[r].max()))
            assert abs(int(A[r, w]) - inj.sample) <= 1
        k64.free()


def test_stream_winmax_matches_the_oracle(torch):
    """Streaming over data 2.5 segment hops long against the oracle: every window of the stream
    is the window peak of the oracle's direct sum (Eq. 8) on the oracle's matched filter of the
    segment whose interior holds the window (data outside the stream zero), for the references
    (Eq. 2) and their neighbours."""
    base = workload.config(4, n_override=1 << 15, k_override=24)
    rng = np.random.default_rng(52)
    groups = []
    for g, k in enumerate((3, 2)):
        ref = base.groups[g][0]
        nb = workload.duration_lattice(ref, base.f_low, k, 0.05, 2.0, rng, eta_range=(0.235, 0.25), n_eta=1)
        groups.append((ref, nb))
    cfg = replace(base, groups=tuple(groups), injections=())
    n, W = cfg.n, 2048
    guard = 2 * W
    hop = n - 2 * guard
    total = 5 * hop // 2 // W * W
    x = rng.standard_normal(total).astype(np.float32)
    ip = workload.inv_psd(cfg)
    ipt = torch.tensor(ip, device="cuda")
    rf = _rf(cfg)
    refs = [g[0] for g in cfg.groups]
    filt, _ = rf.reference_filters(ipt, refs)
    kerns = [rf.build_ratio_kernels(r, nb, ipt, cfg.threshold) for r, nb in cfg.groups]
    rm, ra, nm, na = rf.stream_winmax(x, filt, kerns, W, guard)
    nwt = total // W
    pks = [ratio.build_ratio_kernels(r, list(nb), n, cfg.fs, cfg.f_low, cfg.f_high, cfg.pn_order, ip,
                                     cfg.threshold) for r, nb in cfg.groups]
    for g, pk in enumerate(pks):
        assert np.array_equal(pk.lag0, kerns[g].lag0) and np.array_equal(pk.length, kerns[g].length)
    # oracle: the series of every template on every segment, each window from its segment
    ref_P = np.zeros((len(refs), nwt))
    ref_A = np.zeros((len(refs), nwt), dtype=np.int64)
    nb_P = np.zeros((nm.shape[0], nwt))
    nb_A = np.zeros((nm.shape[0], nwt), dtype=np.int64)
    series_ref, series_nb = {}, {}
    q = 0
    while q * hop < nwt * W:
        s0 = q * hop - guard
        seg = np.zeros(n)
        a, b = max(0, s0), min(total, s0 + n)
        seg[a - s0:b - s0] = x[a:b]
        row = 0
        for g, (ref, nb) in enumerate(cfg.groups):
            zo, _ = mf.matched_filter(seg, ip, n, cfg.fs, cfg.f_low, cfg.f_high, ref.m1, ref.m2, cfg.pn_order)
            zs = [reconstruct.reconstruct_direct(zo, *pks[g].kernel(j)) for j in range(len(nb))]
            for wl in range(guard // W, (n - guard) // W):
                w = (s0 + wl * W) // W
                if not 0 <= w < nwt:
                    continue
                sl = slice(wl * W, (wl + 1) * W)
                m2 = np.abs(zo[sl]) ** 2
                ref_P[g, w], ref_A[g, w] = m2.max(), s0 + wl * W + int(np.argmax(m2))
                series_ref[(g, w)] = m2
                for j, zj in enumerate(zs):
                    m2 = np.abs(zj[sl]) ** 2
                    nb_P[row + j, w], nb_A[row + j, w] = m2.max(), s0 + wl * W + int(np.argmax(m2))
                    series_nb[(row + j, w)] = m2
            row += len(nb)
        q += 1
    assert q == 3
    for P, A, Po, Ao, series in ((rm, ra, ref_P, ref_A, series_ref), (nm, na, nb_P, nb_A, series_nb)):
        for r in range(P.shape[0]):
            zmax = np.sqrt(Po[r].max())
            assert np.abs(np.sqrt(P[r]) - np.sqrt(Po[r])).max() <= TOL32 * zmax
            for w in range(nwt):
                m2 = np.sort(series[(r, w)])
                bound = 4.0 * TOL32 * zmax * np.sqrt(m2[-1])
                if m2[-1] - m2[-2] > bound:
                    assert A[r, w] == Ao[r, w], (r, w)
                else:
                    assert series[(r, w)][A[r, w] - w * W] >= m2[-1] - bound


GEMM_TOL_LONG = {"bf16x6": 2e-6, "3xtf32": 2e-6}


@pytest.mark.parametrize("prec", ["bf16x6", "3xtf32"])
def test_reconstruct_gemm_kernels_up_to_4096_taps(torch, prec):
    """The tensor-core form on kernels of 1000 to 4096 taps (several K chunks per tile, ragged
    last chunk, signed first lags) against the oracle's direct sum, series and window peaks."""
    n = 1 << 14
    rng = np.random.default_rng(4096)
    lengths = [1000, 1023, 2047, 2048, 2049, 3000, 4095, 4096]
    lags = [0, -7, 301, -(n // 2) + 1, n // 2, 1234, -4000, 77]
    cfg = workload.config(2, n_override=n, k_override=1)
    rf = _rf(cfg)
    z = (rng.standard_normal(n) + 1j * rng.standard_normal(n)).astype(np.complex64)
    taps = [((rng.standard_normal(L) + 1j * rng.standard_normal(L)) / np.sqrt(L)).astype(np.complex64)
            for L in lengths]
    kern = rf.kernels_import(lags, lengths, np.concatenate(taps))
    zt = torch.tensor(z, device="cuda")
    out = rf.reconstruct(zt, kern, "gemm", prec=prec).cpu().numpy()
    rf.device_status()
    P, A = rf.reconstruct_winmax(zt, kern, 2048, "gemm", prec=prec)
    P, A = P.cpu().numpy(), A.cpu().numpy()
    tol = GEMM_TOL_LONG[prec]
    for j, L in enumerate(lengths):
        zo = reconstruct.reconstruct_direct(z.astype(np.complex128), lags[j], taps[j].astype(np.complex128))
        assert np.abs(out[j] - zo).max() <= tol * np.abs(zo).max(), (L, np.abs(out[j] - zo).max() / np.abs(zo).max())
        Po, Ao = reconstruct.window_peaks(zo, 2048)
        zmax = np.sqrt(Po.max())
        assert np.abs(np.sqrt(P[j]) - np.sqrt(Po)).max() <= tol * zmax
        m2 = zo.real ** 2 + zo.imag ** 2
        for w in range(Po.shape[0]):
            seg = np.sort(m2[w * 2048:(w + 1) * 2048])
            bound = 4.0 * tol * zmax * np.sqrt(seg[-1])
            if seg[-1] - seg[-2] > bound:
                assert A[j, w] == Ao[w]
            else:
                assert m2[A[j, w]] >= seg[-1] - bound
    kern.free()
