"""Pins of the oracle matched filter: zero-noise optimal SNR, noise statistics,
and the strain/spectrum conventions against library transforms."""
from dataclasses import replace

import numpy as np

import workload
from oracle import data, mf
from workload import Injection


def _cfg(n=1 << 14):
    return workload.config(1, n_override=n)


def test_zero_noise_injection_peaks_at_optimal_snr():
    """Eqs. (2)-(3): the exact template at an integer arrival sample gives |z| = rho_opt there."""
    cfg = _cfg()
    ref, nb = cfg.groups[0]
    for s, snr in [(1234, 12.0), (cfg.n - 77, 8.0)]:
        c = replace(cfg, injections=(Injection(3, 0, s, snr),))
        x = data.strain(c, noise=False)
        t = nb[3]
        z, N = mf.matched_filter(x, workload.inv_psd(c), c.n, c.fs, c.f_low, c.f_high, t.m1, t.m2, c.pn_order)
        assert int(np.argmax(np.abs(z))) == s
        assert abs(abs(z[s]) - snr) < 1e-11
        # phase of z at the peak is zero for phi_c = 0 (template matched exactly)
        assert abs(np.angle(z[s])) < 1e-10


def test_noise_only_mean_power_is_two():
    """Eq. (3) normalisation: E|z|^2 = 2 in Gaussian noise with the one-sided PSD."""
    cfg = replace(_cfg(1 << 15), injections=())
    ref = cfg.groups[0][0]
    ip = workload.inv_psd(cfg)
    means, res = [], []
    for r in range(32):
        x = data.strain(cfg, realisation=r, injections=False)
        z, _ = mf.matched_filter(x, ip, cfg.n, cfg.fs, cfg.f_low, cfg.f_high, ref.m1, ref.m2, cfg.pn_order)
        means.append(np.mean(np.abs(z) ** 2))
        res.append(np.mean(z.real))
    assert abs(np.mean(means) - 2.0) < 0.05
    assert abs(np.mean(res)) < 0.05


def test_strain_conventions_against_library():
    """x = irfft(x~) / dt and x~ = dt * rfft(x), the continuous-FT normalisation of Eq. (1)."""
    cfg = _cfg(1 << 12)
    xf = workload.noise_spectrum(cfg) + 0.0
    x = data.spectrum_to_strain(xf, cfg.n, cfg.fs)
    assert np.allclose(x, np.fft.irfft(xf, cfg.n) * cfg.fs, rtol=0, atol=1e-12 * np.abs(x).max())
    back = mf.data_spectrum(x, cfg.fs)
    assert np.allclose(back, np.fft.rfft(x) / cfg.fs, rtol=0, atol=1e-12 * np.abs(back).max())
    assert np.allclose(back, xf, rtol=0, atol=1e-9 * np.abs(xf).max())


def test_band_limit_zeroes_outside_band():
    """Eq. (4): data outside [f_low, f_high] do not reach z."""
    cfg = replace(_cfg(1 << 12), injections=())
    ref = cfg.groups[0][0]
    ip = workload.inv_psd(cfg)
    f = mf.freqs(cfg.n, cfg.fs)
    xf = np.where((f < cfg.f_low) | (f > cfg.f_high), 1.0 + 0.5j, 0.0)
    x = data.spectrum_to_strain(xf, cfg.n, cfg.fs)
    z, _ = mf.matched_filter(x, ip, cfg.n, cfg.fs, cfg.f_low, cfg.f_high, ref.m1, ref.m2, cfg.pn_order)
    assert np.abs(z).max() < 1e-9


def test_sigma_closed_form_flat_psd():
    """N^2 = 4 df sum |h|^2 / S: for |h| = f^-7/6 and unit flat PSD it is a plain sum."""
    n, fs = 1 << 12, 1024.0
    f = mf.freqs(n, fs)
    h = mf.template(n, fs, 1.4, 1.3, 2)
    ipb = np.where((f >= 30) & (f <= 300), 1.0, 0.0)
    fb = f[ipb > 0]
    expect = np.sqrt(4 * (fs / n) * np.sum(fb ** (-7 / 3)))
    assert abs(mf.sigma(h, ipb, fs / n) / expect - 1) < 1e-13


def test_snr_at_equals_the_series_at_those_samples():
    """The sampled form of Eq. 2 agrees with the transform-based series (a different route:
    per-sample sums with exact integer phase reduction against the radix-2 inverse FFT)."""
    cfg = workload.config(1, n_override=1 << 12, k_override=2)
    ip = workload.inv_psd(cfg)
    x = data.strain(cfg)
    ref = cfg.groups[0][0]
    n, fs = cfg.n, cfg.fs
    xf = mf.data_spectrum(x, fs)
    ipb = mf.band_limited_inv_psd(ip, n, fs, cfg.f_low, cfg.f_high)
    h = mf.template(n, fs, ref.m1, ref.m2, cfg.pn_order)
    z, _ = mf.snr_series(xf, h, ipb, n, fs)
    idx = np.array([0, 1, 17, n // 2, n - 1, 2049])
    zs = mf.snr_at(xf, h, ipb, n, fs, idx)
    assert np.abs(zs - z[idx]).max() <= 1e-10 * np.abs(z).max()


def test_band_includes_both_edge_bins():
    """Eq. (4): 1/S is zero outside the closed band [f_low, f_high]; when both edges fall on
    grid bins, those bins are kept and their outer neighbours are not."""
    n, fs = 1 << 12, 1024.0
    df = fs / n
    f_low, f_high = 160 * df, 1800 * df
    ipb = mf.band_limited_inv_psd(np.ones(n // 2 + 1), n, fs, f_low, f_high)
    assert ipb[160] == 1.0 and ipb[1800] == 1.0
    assert ipb[159] == 0.0 and ipb[1801] == 0.0
    assert np.count_nonzero(ipb) == 1800 - 160 + 1
