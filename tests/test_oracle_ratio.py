"""Pins of the oracle ratio kernels: exact identities (Eqs. 7-8), special cases,
window closed form (Eq. 9), App. A envelope and tail bounds, truncation."""
import itertools
import math
from dataclasses import replace

import numpy as np
import pytest

import workload
from oracle import bounds, data, mf, ratio, reconstruct
from workload import Template


def _setup(n=1 << 14, k=4):
    cfg = workload.config(1, n_override=n, k_override=k)
    ip = workload.inv_psd(cfg)
    x = data.strain(cfg)
    ref, nb = cfg.groups[0]
    z_ref, _ = mf.matched_filter(x, ip, cfg.n, cfg.fs, cfg.f_low, cfg.f_high, ref.m1, ref.m2, cfg.pn_order)
    return cfg, ip, x, ref, nb, z_ref


def _full_mf(cfg, ip, x, t):
    z, _ = mf.matched_filter(x, ip, cfg.n, cfg.fs, cfg.f_low, cfg.f_high, t.m1, t.m2, cfg.pn_order, t.tc, t.phic)
    return z


def test_window_closed_form():
    f_low, f_high, dl, dh = 40.0, 459.0, 3.0, 53.0
    f = np.array([f_low - dl, f_low - dl / 2, f_low, 100.0, f_high, f_high + dh / 2, f_high + dh, 0.0, 600.0])
    w = ratio.window(f, f_low, f_high, dl, dh)
    assert np.allclose(w, [0.0, 0.5, 1.0, 1.0, 1.0, 0.5, 0.0, 0.0, 0.0], atol=1e-15)
    # continuity and monotonic tapers
    g = np.linspace(f_low - dl, f_low, 101)
    assert np.all(np.diff(ratio.window(g, f_low, f_high, dl, dh)) >= -1e-15)
    g = np.linspace(f_high, f_high + dh, 101)
    assert np.all(np.diff(ratio.window(g, f_low, f_high, dl, dh)) <= 1e-15)


@pytest.mark.parametrize("side", ["low", "high"])
def test_window_tapers_are_raised_cosines(side):
    """Eq. (9)'s tapers are raised cosines: flat at both ends of the taper (a linear ramp is
    not), steepest at the midpoint with slope pi / (2 df), and point-symmetric about it."""
    f_low, f_high, dl, dh = 40.0, 459.0, 3.0, 53.0
    a, d = (f_low - dl, dl) if side == "low" else (f_high, dh)
    w = lambda f: ratio.window(np.asarray(f, dtype=np.float64), f_low, f_high, dl, dh)
    h = 1e-5 * d
    slope = lambda f: (w(f + h) - w(f - h)) / (2 * h)
    for end in (a + 1e-4 * d, a + d - 1e-4 * d):
        assert abs(slope(end)) < 1e-3 / d
    x = np.linspace(a + 0.01 * d, a + 0.99 * d, 999)
    s = np.abs(slope(x))
    assert abs(s.max() - math.pi / (2 * d)) < 1e-6 / d
    assert abs(x[np.argmax(s)] - (a + d / 2)) < 2e-3 * d
    u = np.linspace(0.0, d, 37)
    assert np.allclose(w(a + u) + w(a + d - u), 1.0, rtol=0, atol=1e-14)


def test_df_low_rule_newtonian_closed_form():
    """Eq. (10) at Newtonian order: t(f) = -(5/256) Mc^(-5/3) (pi f)^(-8/3), so
    |dt'(f_low)| = (8/3)(5/256) pi^(-8/3) f_low^(-11/3) |Mc_t^(-5/3) - Mc_ref^(-5/3)|; the
    5 Hz cap and the f_low/2 guard bound it, and equal templates take the cap."""
    ref = Template(1.6, 1.5)
    for tgt, f_low in [(Template(1.62, 1.5), 20.0), (Template(1.4, 1.35), 30.0), (Template(2.0, 1.2), 40.0)]:
        mc = lambda t: (t.m1 * t.m2) ** 0.6 / (t.m1 + t.m2) ** 0.2 * workload.MSUN_S
        dtp = 8.0 / 3.0 * 5.0 / 256.0 * math.pi ** (-8.0 / 3.0) * f_low ** (-11.0 / 3.0) * \
            abs(mc(tgt) ** (-5.0 / 3.0) - mc(ref) ** (-5.0 / 3.0))
        want = 1.0 / math.sqrt(dtp)
        got = ratio.df_low_rule(ref, tgt, 0, f_low, df_low_max=1e9)
        assert abs(got / min(want, 0.5 * f_low) - 1.0) < 1e-12
        assert ratio.df_low_rule(ref, tgt, 0, f_low, df_low_max=0.1) == 0.1
    assert ratio.df_low_rule(ref, ref, 7, 20.0, df_low_max=5.0) == 5.0
    assert ratio.df_low_rule(ref, ref, 7, 4.0, df_low_max=5.0) == 2.0


def test_untruncated_identity_reproduces_full_matched_filter():
    """Eqs. (7)-(8): with the whole circular kernel, reconstruction equals direct MF."""
    cfg, ip, x, ref, nb, z_ref = _setup()
    for t in nb[:3]:
        K, _ = ratio.kernel_spectrum(ref, t, cfg.n, cfg.fs, cfg.f_low, cfg.f_high, cfg.pn_order, ip)
        rho = ratio.kernel_full(K, cfg.n)
        zf = _full_mf(cfg, ip, x, t)
        # circular convolution by FFT of the full kernel (exact identity check)
        zh = np.fft.ifft(np.fft.fft(z_ref) * np.fft.fft(rho))
        assert np.abs(zh - zf).max() / np.abs(zf).max() < 1e-12


def test_untruncated_identity_direct_sum_small():
    cfg, ip, x, ref, nb, z_ref = _setup(n=1 << 11, k=2)
    t = nb[1]
    K, _ = ratio.kernel_spectrum(ref, t, cfg.n, cfg.fs, cfg.f_low, cfg.f_high, cfg.pn_order, ip)
    rho = ratio.kernel_full(K, cfg.n)
    zh = reconstruct.reconstruct_direct(z_ref, 0, rho)
    zf = _full_mf(cfg, ip, x, t)
    assert np.abs(zh - zf).max() / np.abs(zf).max() < 1e-12


def test_special_cases_identity_shift_phase():
    cfg, ip, x, ref, nb, z_ref = _setup()
    n = cfg.n
    # same template: z unchanged
    for tgt, expect in [
        (ref, z_ref),
        (replace(ref, tc=37 / cfg.fs), np.roll(z_ref, -37)),        # z^[i] = z_ref[i + 37]
        (replace(ref, tc=-5 / cfg.fs), np.roll(z_ref, 5)),
        (replace(ref, phic=0.9), z_ref * np.exp(-0.9j)),
    ]:
        K, _ = ratio.kernel_spectrum(ref, tgt, n, cfg.fs, cfg.f_low, cfg.f_high, cfg.pn_order, ip, df_low=4.0)
        rho = ratio.kernel_full(K, n)
        zh = np.fft.ifft(np.fft.fft(z_ref) * np.fft.fft(rho))
        assert np.abs(zh - expect).max() / np.abs(z_ref).max() < 1e-12


def test_kernel_parseval():
    cfg, ip, x, ref, nb, z_ref = _setup()
    K, _ = ratio.kernel_spectrum(ref, nb[0], cfg.n, cfg.fs, cfg.f_low, cfg.f_high, cfg.pn_order, ip)
    rho = ratio.kernel_full(K, cfg.n)
    assert abs(np.sum(np.abs(rho) ** 2) / (np.sum(np.abs(K) ** 2) / cfg.n) - 1) < 1e-12


def _long_pair():
    """A pair with a long kernel (f_low = 20 Hz, 3.5PN), as in the paper's figures."""
    n, fs = 1 << 17, 1024.0
    ref = Template(1.6, 1.5)
    tgt = Template(1.64, 1.48)
    return n, fs, 20.0, fs / 2 - 53.0, ref, tgt


def test_kernel_envelope_follows_stationary_phase():
    """Eq. (A11): inside the support |rho[m]| ~ dt / sqrt(|dt'(f*)|) with dt(f*) = -m dt."""
    n, fs, fl, fh, ref, tgt = _long_pair()
    ip = np.ones(n // 2 + 1)
    K, dfl = ratio.kernel_spectrum(ref, tgt, n, fs, fl, fh, 7, ip)
    rho = ratio.kernel_full(K, n)
    d_lo = bounds.delta_t(np.array([fl]), ref, tgt, 7)[0]
    d_hi = bounds.delta_t(np.array([fh]), ref, tgt, 7)[0]
    lo, hi = sorted([-d_lo, -d_hi])                     # lag-time support [lo, hi]
    assert hi - lo > 1.0                                  # a long kernel
    m = np.arange(int(math.ceil((lo + 0.2 * (hi - lo)) * fs)), int((hi - 0.2 * (hi - lo)) * fs))
    env = bounds.stationary_envelope(m / fs, ref, tgt, 7, fl, fh, 1 / fs)
    got = np.abs(rho[m % n])
    ok = np.isfinite(env)
    # local RMS over 64 lags removes the SPA interference ripple
    k = 64
    ratio_ = np.sqrt(np.convolve(got[ok] ** 2, np.ones(k) / k, "valid")) / np.convolve(env[ok], np.ones(k) / k, "valid")
    assert np.median(ratio_) == pytest.approx(1.0, abs=0.1)
    # and most energy lies in the stationary support
    sup = np.arange(int(lo * fs) - 64, int(hi * fs) + 64)
    assert np.sum(np.abs(rho[sup % n]) ** 2) / np.sum(np.abs(rho) ** 2) > 0.99


def _wide_pair():
    """1.4 + 1.4 against 2 + 2 Msun: a 72 s duration difference and a high-frequency time
    offset of 17 ms (17 lags), so the high tail's centre is resolved."""
    n, fs = 1 << 17, 1024.0
    return n, fs, 20.0, fs / 2 - 53.0, Template(1.4, 1.4), Template(2.0, 2.0)


@pytest.mark.parametrize("pair", [_long_pair, _wide_pair])
def test_kernel_tails_below_appendix_bounds_and_window_shortens_them(pair):
    """Eqs. (A9)-(A10): tails beyond the support decay below the bounds (x2 slack
    for the one-sided vs 2 Re form), and reach them within a small factor: the bounds
    are the tails' leading-order envelope (three integrations by parts over the
    raised-cosine taper).  Without the window (df = 0) the tails are longer (Fig. 2)."""
    n, fs, fl, fh, ref, tgt = pair()
    ip = np.ones(n // 2 + 1)
    K, dfl = ratio.kernel_spectrum(ref, tgt, n, fs, fl, fh, 7, ip)
    rho = ratio.kernel_full(K, n)
    d_lo = bounds.delta_t(np.array([fl]), ref, tgt, 7)[0]
    d_hi = bounds.delta_t(np.array([fh]), ref, tgt, 7)[0]
    # low-frequency end of the support is at lag time -d_lo; go 2..10 / df_low beyond it
    sgn = np.sign(-d_lo - (-d_hi))
    t_lo = -d_lo + sgn * np.linspace(2.0 / dfl, 10.0 / dfl, 200)
    b_lo = bounds.low_tail_bound(t_lo, ref, tgt, 7, fl, dfl, 1 / fs)
    got_lo = np.abs(rho[np.round(t_lo * fs).astype(int) % n])
    assert np.all(got_lo <= 2.0 * b_lo + 1e-12)
    assert np.max(got_lo / b_lo) > 0.4
    t_hi = -d_hi - sgn * np.linspace(2.0 / 53.0, 10.0 / 53.0, 50)
    b_hi = bounds.high_tail_bound(t_hi, ref, tgt, 7, fh, 53.0, 1 / fs)
    got_hi = np.abs(rho[np.round(t_hi * fs).astype(int) % n])
    assert np.all(got_hi <= 2.0 * b_hi + 1e-12)
    assert np.max(got_hi / b_hi) > 0.4
    # the unwindowed kernel has a longer tail at the same lags
    K0, _ = ratio.kernel_spectrum(ref, tgt, n, fs, fl, fh, 7, ip, df_low=0.0, df_high=0.0)
    rho0 = ratio.kernel_full(K0, n)
    got0 = np.abs(rho0[np.round(t_lo * fs).astype(int) % n])
    assert np.median(got0) > 5 * np.median(got_lo)
    _, L_win, _ = ratio.truncate(rho, 1e-3)
    _, L_raw, _ = ratio.truncate(rho0, 1e-3)
    assert L_raw > L_win


def _brute_arc(mask):
    n = mask.size
    best = None
    for L in range(0, n + 1):
        for m0 in range(n):
            cover = np.zeros(n, bool)
            cover[(m0 + np.arange(L)) % n] = True
            if np.all(cover[mask]):
                sl = ratio.signed_lag(m0, n)
                if best is None or L < best[1] or (L == best[1] and sl < ratio.signed_lag(best[0], n)):
                    best = (m0, L)
        if best is not None:
            return best
    return best


def test_minimal_arc_brute_force():
    rng = np.random.default_rng(11)
    for n in (1, 2, 3, 5, 8, 9, 16):
        for _ in range(60):
            mask = rng.random(n) < rng.uniform(0.05, 0.6)
            if not mask.any():
                mask[rng.integers(0, n)] = True
            assert ratio.minimal_arc(mask) == _brute_arc(mask), (n, mask)
    # explicit ties: two kept lags diametrically opposite
    mask = np.zeros(8, bool)
    mask[[1, 5]] = True
    assert ratio.minimal_arc(mask) == _brute_arc(mask) == (5, 5)   # start -3 beats start 1
    mask = np.zeros(8, bool)
    mask[[0, 4]] = True
    assert ratio.minimal_arc(mask) == _brute_arc(mask) == (0, 5)   # start 0 beats start +4 (n/2 maps to +n/2)


def test_truncation_keeps_threshold_region_and_is_monotone():
    cfg, ip, x, ref, nb, z_ref = _setup(n=1 << 15, k=2)
    t = nb[0]
    K, _ = ratio.kernel_spectrum(ref, t, cfg.n, cfg.fs, cfg.f_low, cfg.f_high, cfg.pn_order, ip)
    rho = ratio.kernel_full(K, cfg.n)
    zf = _full_mf(cfg, ip, x, t)
    errs, Ls = [], []
    for thr in (1e-2, 1e-3, 1e-4, 1e-5):
        m0, L, c = ratio.truncate(rho, thr)
        kept = (m0 + np.arange(L)) % cfg.n
        outside = np.setdiff1d(np.arange(cfg.n), kept)
        assert np.all(np.abs(rho[outside]) < thr * np.abs(rho).max())
        assert np.array_equal(c, rho[kept])
        zh = reconstruct.reconstruct_direct(z_ref, m0, c)
        errs.append(np.abs(zh - zf).max() / np.abs(zf).max())
        Ls.append(L)
    assert all(a > b for a, b in zip(errs, errs[1:]))
    assert all(a < b for a, b in zip(Ls, Ls[1:]))
    # Sec. II.D / abstract: O(1e-4)-level agreement once truncated at 1e-3
    assert errs[1] < 5e-3


def test_truncation_degenerate_inputs():
    assert ratio.truncate(np.zeros(16, complex), 1e-3)[:2] == (0, 0)
    d = np.zeros(16, complex)
    d[15] = 2.0
    m0, L, c = ratio.truncate(d, 1e-3)
    assert (m0, L) == (-1, 1) and c[0] == 2.0
    m0, L, c = ratio.truncate(np.ones(16, complex), 1e-3)
    assert L == 16


def test_coarse_build_grid_reproduces_the_data_grid_kernels():
    """Built on the rule's coarser grid, every kernel keeps the span of the data-grid kernel
    (the paper's exact object) and its taps to 1e-7 of their maximum; a grid equal to the
    data grid reproduces it exactly; the rule's grid is a power of two below n that grows
    with the duration difference."""
    n = 1 << 16
    cfg = workload.config(1, n_override=n, k_override=4)
    ref = cfg.groups[0][0]
    nb = list(cfg.groups[0][1]) + list(workload.duration_lattice(ref, cfg.f_low, 4, 0.2, 3.0,
                                                                  np.random.default_rng(9), n_eta=1,
                                                                  mrange=(1.0, 4.5)))
    ip = workload.inv_psd(cfg)
    args = (ref, nb, n, cfg.fs, cfg.f_low, cfg.f_high, cfg.pn_order, ip, 1e-4)
    fine = ratio.build_ratio_kernels(*args)
    same = ratio.build_ratio_kernels(*args, n_build=n)
    assert np.array_equal(fine.taps, same.taps) and np.array_equal(fine.lag0, same.lag0)
    coarse = ratio.build_ratio_kernels(*args, n_build=-1)
    assert np.all(coarse.grid < n) and np.all((coarse.grid & (coarse.grid - 1)) == 0)
    assert len(np.unique(coarse.grid)) > 1
    for j in range(len(nb)):
        assert coarse.lag0[j] == fine.lag0[j] and coarse.length[j] == fine.length[j]
        cf, cc = fine.kernel(j)[1], coarse.kernel(j)[1]
        assert np.abs(cc - cf).max() <= 1e-7 * np.abs(cf).max()
    # longer kernels get grids at least as large
    order = np.argsort(fine.length)
    assert np.all(np.diff(coarse.grid[order]) >= 0)


@pytest.mark.parametrize("cfg_id,js", [(1, [0, 7, 15]), (2, [0, 5, 200])])
def test_analytic_span_follows_the_kernel(cfg_id, js):
    """Analytic truncation (Sec. II.D with the App. A expressions): the kept lags contain the
    stationary region between the window edges' times, outside them the kernel's |r| stays
    within a small factor of the threshold amplitude (the Eqs. (A9)-(A10) bounds hold far from
    the edges only), and the span is of the order of the numeric arc at the same threshold;
    absolute thresholds (the paper's 1e-3 / s, and 1e-2 / s) and a small relative one, where
    the tails reach well past the edges (the bounds are asymptotic: at a relative 1e-3 the
    reach beyond a sharp high-frequency edge is under two taper widths and the near sidelobes
    exceed it)."""
    cfg = workload.config(cfg_id)
    ref, nb = cfg.groups[0]
    ip = workload.inv_psd(cfg)
    for rel, thr in [(True, 3e-5), (False, 1e-3), (False, 1e-2)]:
        for j in js:
            t = nb[j]
            a = ratio.build_ratio_kernels(ref, [t], cfg.n, cfg.fs, cfg.f_low, cfg.f_high, cfg.pn_order, ip, thr, rel,
                                          n_build=-1, analytic=True)
            nbg = int(a.grid[0])
            d = ratio.df_low_rule(ref, t, cfg.pn_order, cfg.f_low, cfg.df_low_max)
            K, _ = ratio.kernel_spectrum(ref, t, cfg.n, cfg.fs, cfg.f_low, cfg.f_high, cfg.pn_order, ip, n_build=nbg)
            rho = ratio.kernel_full(K, nbg)
            norm = ratio.norm_ratio(ref, t, cfg.n, cfg.fs, cfg.f_low, cfg.f_high, cfg.pn_order, ip)
            r = 2.0 * cfg.fs * np.abs(rho) / norm                 # |r| envelope (1/s)
            amp = thr * r.max() if rel else thr
            m0, L = int(a.lag0[0]), int(a.length[0])
            kept = np.zeros(nbg, bool)
            kept[(m0 + np.arange(L)) % nbg] = True
            # the stationary region -dt(f) for f in [f_low, f_high]
            fe = np.array([cfg.f_low, cfg.f_high])
            c = -bounds.delta_t(fe, ref, t, cfg.pn_order) * cfg.fs
            stat = np.arange(int(np.ceil(c.min())), int(np.floor(c.max())) + 1)
            assert kept[stat % nbg].all()
            # outside: below a few times the threshold amplitude (the bounds are asymptotic;
            # a span on the wrong side or without the tails leaves 1e3 and more)
            assert r[~kept].max() < 4.0 * amp, (cfg_id, j, rel, thr, r[~kept].max() / amp)
            # of the order of the numeric arc at the same threshold
            _, Ln, _ = ratio.truncate(rho * (1.0 if rel else 2.0 * cfg.fs / norm), thr, rel)
            assert 0.5 * Ln <= L <= 2.0 * Ln, (cfg_id, j, rel, thr, L, Ln)
            # the taps are the kernel itself on the kept lags
            np.testing.assert_array_equal(a.taps, rho[(m0 + np.arange(L)) % nbg])


def test_real_kernel_form_equals_the_complex_one_before_truncation():
    """The paper's real kernel 2 Re rho against the complex one-sided rho (Eq. 8): z_ref has
    no negative-frequency content, so untruncated they give the same series to rounding;
    truncated at the same threshold they differ, by less than the truncation error itself."""
    cfg = workload.config(1, n_override=1 << 13, k_override=3)
    ref, nb = cfg.groups[0]
    ip = workload.inv_psd(cfg)
    x = data.strain(cfg)
    z, _ = mf.matched_filter(x, ip, cfg.n, cfg.fs, cfg.f_low, cfg.f_high, ref.m1, ref.m2, cfg.pn_order)
    for t in nb:
        zc = reconstruct.reconstruct_direct(z, *ratio.build_ratio_kernels(
            ref, [t], cfg.n, cfg.fs, cfg.f_low, cfg.f_high, cfg.pn_order, ip, 0.0).kernel(0))
        zr = reconstruct.reconstruct_direct(z, *ratio.build_ratio_kernels(
            ref, [t], cfg.n, cfg.fs, cfg.f_low, cfg.f_high, cfg.pn_order, ip, 0.0, real=True).kernel(0))
        assert np.abs(zr - zc).max() <= 1e-12 * np.abs(zc).max()
        zt = reconstruct.reconstruct_direct(z, *ratio.build_ratio_kernels(
            ref, [t], cfg.n, cfg.fs, cfg.f_low, cfg.f_high, cfg.pn_order, ip, 1e-3, real=True).kernel(0))
        zct = reconstruct.reconstruct_direct(z, *ratio.build_ratio_kernels(
            ref, [t], cfg.n, cfg.fs, cfg.f_low, cfg.f_high, cfg.pn_order, ip, 1e-3).kernel(0))
        e_real, e_cplx = np.abs(zt - zc).max(), np.abs(zct - zc).max()
        assert 0 < e_real < 20 * max(e_cplx, 1e-12 * np.abs(zc).max())


def test_analytic_span_is_tight_to_the_kernel_tails():
    """The App. A tail bounds (Eqs. A9-A10) are the tails' leading-order envelope, not a loose
    bound.  The raised-cosine taper's second derivative jumps by pi^2 / (2 df^2) at each of its
    two ends; three integrations by parts give |q| ~ 1 / (16 pi df^2 |t - c|^3) per end, and the
    two ends together with |r| = 2 |q| give R / (4 pi df^2 |t - c|^3).  So the analytic span
    (where that bound meets the threshold amplitude) slightly exceeds the numeric arc of the
    kernel at the same amplitude.  A bound constant off by 2, or a relative amplitude taken on
    |rho| instead of |r| = 2 fs |rho| / (N_ref / N) (complex form) or |r| = fs |2 Re rho| /
    (N_ref / N) (real form), moves the span by 2^(1/3)."""
    for real in (False, True):
        groups = {"relative": [], "absolute": []}
        for cfg_id, js in [(1, [0, 7, 15]), (2, [0, 5, 100, 200, 255])]:
            cfg = workload.config(cfg_id)
            ref, nb = cfg.groups[0]
            ip = workload.inv_psd(cfg)
            for rel, thr in [(True, 3e-5), (True, 1e-4), (False, 1e-3), (False, 1e-2)]:
                for j in js:
                    t = nb[j]
                    a = ratio.build_ratio_kernels(ref, [t], cfg.n, cfg.fs, cfg.f_low, cfg.f_high, cfg.pn_order, ip,
                                                  thr, rel, n_build=-1, analytic=True, real=real)
                    nbg = int(a.grid[0])
                    K, _ = ratio.kernel_spectrum(ref, t, cfg.n, cfg.fs, cfg.f_low, cfg.f_high, cfg.pn_order, ip,
                                                 n_build=nbg)
                    rho = ratio.kernel_full(K, nbg)
                    norm = ratio.norm_ratio(ref, t, cfg.n, cfg.fs, cfg.f_low, cfg.f_high, cfg.pn_order, ip)
                    # |r| in 1/s, from the taps of either form
                    taps, scale = ((2.0 * rho.real).astype(complex), cfg.fs / norm) if real else \
                        (rho, 2.0 * cfg.fs / norm)
                    _, Ln, _ = ratio.truncate(taps * (1.0 if rel else scale), thr, rel)
                    q = int(a.length[0]) / Ln
                    assert 0.95 <= q <= 1.4, (real, cfg_id, j, rel, thr, q)
                    groups["relative" if rel else "absolute"].append(q)
        for name, qs in groups.items():
            assert 1.0 <= float(np.median(qs)) <= 1.25, (real, name, sorted(qs))


def test_analytic_span_covers_the_level_set_of_the_bounds():
    """The analytic span by brute force (Sec. II.D with Eqs. A9-A10).  On a fine time grid, the
    lag times where the bound of one of the four taper ends, R / (4 pi df_e^2 |t - c_e|^3) with
    c_e = -dt(f_e) and R = 1 for this family, reaches the amplitude, together with the region
    between the ends, form one interval.  The span covers it, rounded out to whole lags: at
    most one lag more on each side."""
    cfg = workload.config(2)
    ref, nb = cfg.groups[0]
    fs, n = cfg.fs, cfg.n
    h = 0.02 / fs                                   # brute-force time step: a fiftieth of a lag
    for j in (0, 100, 255):
        t = nb[j]
        d = ratio.df_low_rule(ref, t, cfg.pn_order, cfg.f_low, cfg.df_low_max)
        fe = np.array([cfg.f_low - d, cfg.f_low, cfg.f_high, cfg.f_high + cfg.df_high])
        dfe = np.array([d, d, cfg.df_high, cfg.df_high])
        c = -bounds.delta_t(fe, ref, t, cfg.pn_order)
        for amp in (1e-3, 1e-2, 0.3):
            m0, L = bounds.analytic_span(ref, t, cfg.pn_order, cfg.f_low, cfg.f_high, d, cfg.df_high, fs, n, amp)
            reach = (1.0 / (4.0 * math.pi * dfe.min() ** 2 * amp)) ** (1.0 / 3.0) + 1.0
            tt = np.arange(c.min() - reach, c.max() + reach, h)
            b = np.max(1.0 / (4.0 * math.pi * dfe[:, None] ** 2 * np.abs(tt[None, :] - c[:, None]) ** 3), axis=0)
            inside = (b >= amp) | ((tt >= c.min()) & (tt <= c.max()))
            lo, hi = tt[inside].min() * fs, tt[inside].max() * fs     # in lags
            assert m0 <= lo + h * fs and m0 + L - 1 >= hi - h * fs, (j, amp, m0, L, lo, hi)
            assert m0 > lo - 1.0 - h * fs and m0 + L - 1 < hi + 1.0 + h * fs, (j, amp, m0, L, lo, hi)
