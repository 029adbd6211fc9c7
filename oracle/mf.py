"""Matched filtering (oracle; test infrastructure only).

Sec. II.A.  With the one-sided grid f_k = k df, df = 1/T, k = 0..n/2:

* data spectrum (Eq. 1, discretised):  x~_k = dt * sum_j x[j] exp(-2 pi i j k / n);
* band limitation (Eq. 4):  S_n = +inf outside [f_low, f_high], i.e. the
  inverse PSD is zero there (both band edges included);
* normalisation (Eq. 3):  N^2 = 4 df sum_k |h~_k|^2 / S_k;
* complex SNR (Eqs. 2, 6):
      z[i] = (4 df / N) sum_{k=0}^{n/2} x~_k conj(h~_k) / S_k exp(+2 pi i i k / n).
"""
from __future__ import annotations

import numpy as np

from . import fft as _fft
from . import taylorf2


def freqs(n: int, fs: float) -> np.ndarray:
    return np.arange(n // 2 + 1, dtype=np.float64) * (fs / n)


def band_mask(n: int, fs: float, f_low: float, f_high: float) -> np.ndarray:
    f = freqs(n, fs)
    return (f >= f_low) & (f <= f_high)


def band_limited_inv_psd(inv_psd: np.ndarray, n: int, fs: float, f_low: float, f_high: float) -> np.ndarray:
    """Eq. (4): 1/S_n set to zero outside [f_low, f_high]."""
    return np.where(band_mask(n, fs, f_low, f_high), np.asarray(inv_psd, dtype=np.float64), 0.0)


def data_spectrum(x: np.ndarray, fs: float) -> np.ndarray:
    """One-sided x~_k, k = 0..n/2 (Eq. 1 with dt = 1/fs)."""
    x = np.asarray(x, dtype=np.float64)
    n = x.shape[-1]
    return (_fft.fft(x) / fs)[..., : n // 2 + 1]


def template(n: int, fs: float, m1: float, m2: float, pn_order: int, tc: float = 0.0,
             phic: float = 0.0) -> np.ndarray:
    """h~ at the one-sided bins (Eq. A1); 0 at DC."""
    return taylorf2.template_fd(freqs(n, fs), m1, m2, pn_order, tc, phic)


def sigma(h: np.ndarray, inv_psd_band: np.ndarray, df: float) -> float:
    """N of Eq. (3) (inv_psd_band already band limited)."""
    return float(np.sqrt(4.0 * df * np.sum(np.abs(h) ** 2 * inv_psd_band)))


def snr_series(xf: np.ndarray, h: np.ndarray, inv_psd_band: np.ndarray, n: int, fs: float):
    """Complex SNR z[i], i = 0..n-1 (Eq. 2), and N (Eq. 3)."""
    df = fs / n
    N = sigma(h, inv_psd_band, df)
    spec = np.zeros(n, dtype=np.complex128)
    spec[: n // 2 + 1] = (4.0 * df / N) * xf * np.conj(h) * inv_psd_band
    return _fft.ifft_unnormalised(spec), N


def snr_at(xf: np.ndarray, h: np.ndarray, inv_psd_band: np.ndarray, n: int, fs: float,
           idx: np.ndarray) -> np.ndarray:
    """z[i] of Eq. (2) for the sample indices ``idx`` only, each by the defining sum over the
    one-sided bins (for segments too long to transform in the oracle)."""
    df = fs / n
    N = sigma(h, inv_psd_band, df)
    w = (4.0 * df / N) * np.asarray(xf) * np.conj(h) * inv_psd_band
    out = np.empty(len(idx), dtype=np.complex128)
    for q, i in enumerate(np.asarray(idx, dtype=np.int64)):
        # exp(2 pi i i k / n) with the product i k reduced modulo n exactly (integers)
        ph = ((int(i) * np.arange(w.shape[0], dtype=np.int64)) % n).astype(np.float64) * (2.0 * np.pi / n)
        out[q] = np.sum(w * (np.cos(ph) + 1j * np.sin(ph)))
    return out


def matched_filter(x: np.ndarray, inv_psd: np.ndarray, n: int, fs: float, f_low: float, f_high: float,
                   m1: float, m2: float, pn_order: int, tc: float = 0.0, phic: float = 0.0):
    """Full matched filter of real data x with one template: (z, N)."""
    xf = data_spectrum(x, fs)
    ipb = band_limited_inv_psd(inv_psd, n, fs, f_low, f_high)
    h = template(n, fs, m1, m2, pn_order, tc, phic)
    return snr_series(xf, h, ipb, n, fs)
