"""Ratio kernels (oracle; test infrastructure only).

Sec. II.B-II.D and App. A.

* Eq. (5)/(A3)-(A4): r~(f) = h~(f) / h~_ref(f) = R(f) exp(-i dPsi(f)),
  R = B / B_ref, dPsi = Psi - Psi_ref.
* Eq. (7): z = (N_ref / N) * inverse transform of z~_ref * conj(r~).  On the
  discrete one-sided grid the kernel spectrum is therefore
      K~_k = (N_ref / N) W(f_k) conj(r~(f_k)) = (N_ref / N) R(f_k) W(f_k) exp(+i dPsi(f_k)),
  and the kernel is rho[m] = (1/n) sum_{k=0}^{n/2} K~_k exp(+2 pi i k m / n),
  so that z[i] = sum_m rho[m] z_ref[(i - m) mod n] (Eq. 8, circular form).
* Eq. (9): window W(f), cosine tapers on (f_low - df_low, f_low) and
  (f_high, f_high + df_high), 1 on [f_low, f_high], 0 elsewhere.
* Eq. (10): df_low = 1 / sqrt(|d tau'(f_low)|), capped at 5 Hz; with a common
  coalescence time d tau' = -d t', so |d tau'| = |dPsi''| / (2 pi).  A further
  cap df_low <= f_low / 2 keeps the taper at positive frequency (a reading for
  low f_low, where the paper is silent).
* Sec. II.D: keep the region where |rho| is above threshold.  Reading: the
  threshold is relative, thr * max|rho|, decided on squared magnitudes
  |rho|^2 >= thr^2 max|rho|^2 in FP64; the kept region is the shortest
  circular arc [m0, m0 + L) that covers every above-threshold lag (sub-threshold
  lags inside it are kept); ties go to the arc whose start, mapped to
  (-n/2, n/2], is smallest.
* Sec. II.D with App. A, analytic truncation (optional): the kept lags come from the
  App. A expressions instead of the kernel's magnitudes (bounds.analytic_span); parity
  pinned against the computed kernels' tails where the bounds are asymptotic.
* Real-kernel form (optional; the paper's own, Eq. 8 with r(t) = 2 Re of the Eq. (A5)
  integrand of App. A): taps 2 Re rho[m], truncated on |2 Re rho|.  z_ref has no negative-
  frequency content, so before truncation the conjugate half of 2 Re rho multiplies zeros and
  the result equals the complex kernel's; after truncation the two differ.
* Sec. II.D, build grid: the kernels may be built on a coarser frequency grid
  f_k = k fs / n_b (n_b a power of two <= n) as long as 1/df of that grid exceeds
  the kernel's duration; rho is then the n_b-point inverse transform (the same
  (1/n_b) normalisation, so both approximate dt r(t)) and lags are signed on the
  n_b circle.  The rule (a reading: the paper asks only for a grid longer than
  the duration difference) takes the smallest power of two of at least four
  times the lag extent between the window edges' time offsets (Eq. A2) plus the
  low taper's spread 4 fs / df_low.  N_ref / N stays on the data grid.
"""
from __future__ import annotations

import math
from dataclasses import dataclass
from typing import List, Sequence, Tuple

import numpy as np

from . import bounds
from . import fft as _fft
from . import taylorf2
from .mf import band_limited_inv_psd, freqs, sigma


def window(f: np.ndarray, f_low: float, f_high: float, df_low: float, df_high: float) -> np.ndarray:
    """W(f) of Eq. (9)."""
    f = np.asarray(f, dtype=np.float64)
    w = np.zeros_like(f)
    lo = (f > f_low - df_low) & (f < f_low)
    if df_low > 0:
        w[lo] = 0.5 * (1.0 + np.cos(np.pi * (f[lo] - f_low) / df_low))
    mid = (f >= f_low) & (f <= f_high)
    w[mid] = 1.0
    hi = (f > f_high) & (f < f_high + df_high)
    if df_high > 0:
        w[hi] = 0.5 * (1.0 - np.cos(np.pi * (f[hi] - (f_high + df_high)) / df_high))
    return w


def df_low_rule(ref, tgt, pn_order: int, f_low: float, df_low_max: float) -> float:
    """Eq. (10) with the 5 Hz cap and the f_low/2 guard."""
    d2 = taylorf2.d2phase(np.array([f_low]), tgt.m1, tgt.m2, pn_order)[0] - \
        taylorf2.d2phase(np.array([f_low]), ref.m1, ref.m2, pn_order)[0]
    dtp = abs(d2) / (2.0 * math.pi)
    rule = 1.0 / math.sqrt(dtp) if dtp > 0 else math.inf
    return min(df_low_max, 0.5 * f_low, rule)


def norm_ratio(ref, tgt, n: int, fs: float, f_low: float, f_high: float, pn_order: int,
               inv_psd: np.ndarray) -> float:
    """N_ref / N (Eq. 3) on the data grid of n samples."""
    f = freqs(n, fs)
    ipb = band_limited_inv_psd(inv_psd, n, fs, f_low, f_high)
    df = fs / n
    h_ref = taylorf2.template_fd(f, ref.m1, ref.m2, pn_order, ref.tc, ref.phic)
    h_tgt = taylorf2.template_fd(f, tgt.m1, tgt.m2, pn_order, tgt.tc, tgt.phic)
    return sigma(h_ref, ipb, df) / sigma(h_tgt, ipb, df)


def kernel_spectrum(ref, tgt, n: int, fs: float, f_low: float, f_high: float, pn_order: int,
                    inv_psd: np.ndarray, df_low_max: float = 5.0, df_high: float = 53.0,
                    df_low: float = None, n_build: int = None) -> Tuple[np.ndarray, float]:
    """K~_k, k = 0..n_b/2 (Eq. 7 with the Eq. 9 window) on the build grid f_k = k fs / n_b
    (n_b = n_build, default n); N_ref / N (Eq. 3) on the data grid of n samples.  Returns
    (K~, df_low)."""
    nb = n if n_build is None else n_build
    if df_low is None:
        df_low = df_low_rule(ref, tgt, pn_order, f_low, df_low_max)
    norm = norm_ratio(ref, tgt, n, fs, f_low, f_high, pn_order, inv_psd)   # N_ref / N
    fb = freqs(nb, fs)
    w = window(fb, f_low, f_high, df_low, df_high)
    sup = w > 0
    dpsi = taylorf2.phase(fb[sup], tgt.m1, tgt.m2, pn_order, tgt.tc, tgt.phic) - \
        taylorf2.phase(fb[sup], ref.m1, ref.m2, pn_order, ref.tc, ref.phic)
    R = taylorf2.amplitude(fb[sup]) / taylorf2.amplitude(fb[sup])   # B / B_ref (same law)
    K = np.zeros(nb // 2 + 1, dtype=np.complex128)
    K[sup] = norm * R * w[sup] * np.exp(1j * dpsi)
    return K, df_low


def build_grid_rule(ref, tgt, n: int, fs: float, f_low: float, f_high: float, pn_order: int,
                    df_low: float, df_high: float = 53.0) -> int:
    """Build grid of a kernel (Sec. II.D: 1/df of the build grid must exceed the duration
    difference).  The kernel lives between the lags of the time offsets at the window edges,
    dt(f) = (Psi_tgt'(f) - Psi_ref'(f)) / (2 pi) (Eq. A2) at f_low - df_low and
    f_high + df_high, widened by the taper's spread 4 fs / df_low; the grid is the smallest
    power of two of at least four times that extent, capped at n."""
    fe = np.array([f_low - df_low, f_high + df_high])
    d = (taylorf2.dphase(fe, tgt.m1, tgt.m2, pn_order) - taylorf2.dphase(fe, ref.m1, ref.m2, pn_order)) / (2 * math.pi)
    extent = float(np.abs(d).max()) * fs + 4.0 * fs / df_low
    nb = 16
    while nb < 4.0 * extent and nb < n:
        nb *= 2
    return min(nb, n)


def kernel_full(K: np.ndarray, n: int) -> np.ndarray:
    """rho[m], m = 0..n-1: (1/n) times the unnormalised inverse DFT of the
    one-sided K~ (zero at k > n/2)."""
    spec = np.zeros(n, dtype=np.complex128)
    spec[: n // 2 + 1] = K
    return _fft.ifft_unnormalised(spec) / n


def signed_lag(m: int, n: int) -> int:
    """Map a lag in [0, n) to (-n/2, n/2]."""
    return m if m <= n // 2 else m - n


def minimal_arc(mask: np.ndarray) -> Tuple[int, int]:
    """Shortest circular arc [m0, m0+L) covering every True; (m0 in [0,n), L).

    Ties between equally short arcs go to the smallest signed start.
    An all-False mask gives (0, 0).
    """
    n = mask.shape[0]
    s = np.flatnonzero(mask)
    if s.size == 0:
        return 0, 0
    if s.size == 1:
        return int(s[0]), 1
    nxt = np.concatenate([s[1:], [s[0] + n]])
    gaps = nxt - s - 1                       # below-threshold run after each kept lag
    gmax = gaps.max()
    cands = [int(nxt[a] % n) for a in np.flatnonzero(gaps == gmax)]
    m0 = min(cands, key=lambda m: signed_lag(m, n))
    return m0, int(n - gmax)


def truncate(rho: np.ndarray, thr: float, relative: bool = True) -> Tuple[int, int, np.ndarray]:
    """Sec. II.D: (m0 signed, L, taps c[l] = rho[(m0 + l) mod n])."""
    n = rho.shape[0]
    mag2 = rho.real ** 2 + rho.imag ** 2
    amax2 = mag2.max() if n else 0.0
    if amax2 == 0.0:
        return 0, 0, np.zeros(0, dtype=np.complex128)
    cut2 = thr * thr * (amax2 if relative else 1.0)
    m0, L = minimal_arc(mag2 >= cut2)
    taps = rho[(m0 + np.arange(L)) % n]
    return signed_lag(m0, n), L, taps


@dataclass
class PackedKernels:
    """Truncated kernels of one reference group, packed back to back."""
    n: int
    lag0: np.ndarray      # int64 [K] signed first lag m0
    length: np.ndarray    # int64 [K]
    offset: np.ndarray    # int64 [K+1]
    taps: np.ndarray      # complex128 [offset[-1]]
    df_low: np.ndarray    # float64 [K]
    grid: np.ndarray = None  # int64 [K] build grid (lags are signed on it)

    def kernel(self, j: int) -> Tuple[int, np.ndarray]:
        return int(self.lag0[j]), self.taps[self.offset[j]:self.offset[j + 1]]


def build_ratio_kernels(ref, targets: Sequence, n: int, fs: float, f_low: float, f_high: float,
                        pn_order: int, inv_psd: np.ndarray, thr: float, relative: bool = True,
                        df_low_max: float = 5.0, df_high: float = 53.0, n_build: int = 0,
                        analytic: bool = False, real: bool = False) -> PackedKernels:
    """Kernel spectrum -> full kernel -> threshold truncation, per target.

    n_build: 0 builds on the data grid (n lags); a power of two builds every kernel on that
    grid; -1 takes build_grid_rule per target.  Lags are signed on the build grid.
    analytic: the kept lags come from the App. A expressions (bounds.analytic_span) instead
    of the kernel's own magnitudes; a relative threshold is then taken on the kernel's peak
    of |r| = 2 fs |rho| / (N_ref / N), an absolute one is a threshold amplitude on |r| in 1/s.
    real: the real-kernel form, taps 2 Re rho (imaginary parts zero), truncated on their
    magnitude (numeric) or on the same analytic span."""
    lag0: List[int] = []
    length: List[int] = []
    taps: List[np.ndarray] = []
    dfl: List[float] = []
    grids: List[int] = []
    for t in targets:
        d = df_low_rule(ref, t, pn_order, f_low, df_low_max)
        nb = n if n_build == 0 else (n_build if n_build > 0 else
                                     build_grid_rule(ref, t, n, fs, f_low, f_high, pn_order, d, df_high))
        K, _ = kernel_spectrum(ref, t, n, fs, f_low, f_high, pn_order, inv_psd, df_low_max, df_high, d, nb)
        rho = kernel_full(K, nb)
        if real:
            rho = (2.0 * rho.real).astype(np.complex128)
        if analytic:
            # |r| = 2 fs |rho| / (N_ref / N) for the complex kernel, fs |2 Re rho| / (N_ref / N) real
            peak = float(np.abs(rho).max()) if nb else 0.0
            amp = thr * (1.0 if real else 2.0) * fs * peak / \
                norm_ratio(ref, t, n, fs, f_low, f_high, pn_order, inv_psd) if relative else thr
            if amp <= 0.0:
                m0, L, c = 0, 0, np.zeros(0, dtype=np.complex128)
            else:
                m0, L = bounds.analytic_span(ref, t, pn_order, f_low, f_high, d, df_high, fs, nb, amp)
                c = rho[(m0 + np.arange(L)) % nb]
        else:
            m0, L, c = truncate(rho, thr, relative)
        lag0.append(m0)
        length.append(L)
        taps.append(c)
        dfl.append(d)
        grids.append(nb)
    offset = np.concatenate([[0], np.cumsum(length)]).astype(np.int64)
    return PackedKernels(n, np.array(lag0, np.int64), np.array(length, np.int64), offset,
                         np.concatenate(taps) if taps else np.zeros(0, np.complex128), np.array(dfl),
                         np.array(grids, np.int64))
