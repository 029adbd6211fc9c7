"""Target SNR reconstruction and window peaks (oracle; test infrastructure only).

Eq. (8) in discrete circular form, with the truncated kernel (Sec. II.D):
    z^[i] = sum_{l=0}^{L-1} c[l] z_ref[(i - m0 - l) mod n],   c[l] = rho[(m0 + l) mod n].
Computed directly, O(n L), never through an FFT.

Per-window peak (the product read in Sec. IV): for windows of W samples,
    P[w] = max_{i in [wW, (w+1)W)} |z^[i]|^2,   A[w] = smallest i attaining it.
"""
from __future__ import annotations

import numpy as np


def reconstruct_direct(z_ref: np.ndarray, m0: int, taps: np.ndarray) -> np.ndarray:
    """Full series z^ (complex128, length n) by the defining sum."""
    z_ref = np.asarray(z_ref, dtype=np.complex128)
    out = np.zeros_like(z_ref)
    for l, c in enumerate(np.asarray(taps, dtype=np.complex128)):
        # np.roll(a, s)[i] = a[(i - s) mod n]
        out += c * np.roll(z_ref, m0 + l)
    return out


def reconstruct_at(z_ref: np.ndarray, m0: int, taps: np.ndarray, idx: np.ndarray) -> np.ndarray:
    """z^[i] for the sample indices ``idx`` only, each by the defining sum."""
    z_ref = np.asarray(z_ref, dtype=np.complex128)
    n = z_ref.shape[0]
    taps = np.asarray(taps, dtype=np.complex128)
    idx = np.asarray(idx, dtype=np.int64)
    out = np.empty(idx.shape[0], dtype=np.complex128)
    l = np.arange(taps.shape[0], dtype=np.int64)
    for q, i in enumerate(idx):
        out[q] = np.sum(taps * z_ref[(i - m0 - l) % n])
    return out


def window_peaks(z: np.ndarray, W: int):
    """(P, A): per-window max |z|^2 and its smallest index; the last window may be short."""
    z = np.asarray(z)
    n = z.shape[0]
    nw = (n + W - 1) // W
    mag2 = (z.real.astype(np.float64) ** 2 + z.imag.astype(np.float64) ** 2)
    P = np.empty(nw, dtype=np.float64)
    A = np.empty(nw, dtype=np.int64)
    for w in range(nw):
        seg = mag2[w * W: min(n, (w + 1) * W)]
        a = int(np.argmax(seg))          # first occurrence of the maximum
        P[w] = seg[a]
        A[w] = w * W + a
    return P, A
