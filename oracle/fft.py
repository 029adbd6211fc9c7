"""Radix-2 discrete Fourier transform (oracle; test infrastructure only).

Convention (Eq. 1 discretised): the forward transform is
    X[k] = sum_j x[j] exp(-2 pi i j k / n),
the inverse (unnormalised) transform is
    x[j] = sum_k X[k] exp(+2 pi i j k / n).
Continuous-FT normalisation (a~(f_k) = dt * X[k]) is applied by the callers.

Textbook iterative Cooley-Tukey: bit-reversal permutation, then log2(n)
stages of size-2 butterflies with twiddles exp(-+2 pi i m / size).  Each
stage is vectorised over its butterflies with numpy, which is only a faster
way to run the same butterflies; no other restructuring.
"""
from __future__ import annotations

import numpy as np


def _bit_reverse_indices(n: int) -> np.ndarray:
    bits = n.bit_length() - 1
    idx = np.arange(n, dtype=np.int64)
    rev = np.zeros(n, dtype=np.int64)
    for b in range(bits):
        rev |= ((idx >> b) & 1) << (bits - 1 - b)
    return rev


def _transform(x: np.ndarray, sign: float) -> np.ndarray:
    a = np.asarray(x, dtype=np.complex128)
    n = a.shape[-1]
    if n == 0:
        return a.copy()
    if n & (n - 1):
        raise ValueError("oracle FFT needs a power-of-two length")
    a = a[..., _bit_reverse_indices(n)].copy()
    size = 2
    while size <= n:
        half = size // 2
        m = np.arange(half)
        w = np.exp(sign * 2j * np.pi * m / size)          # twiddles of this stage
        a = a.reshape(a.shape[:-1] + (n // size, size))
        top = a[..., :half].copy()
        bot = a[..., half:] * w
        a[..., :half] = top + bot
        a[..., half:] = top - bot
        a = a.reshape(a.shape[:-2] + (n,))
        size *= 2
    return a


def fft(x: np.ndarray) -> np.ndarray:
    """Forward DFT along the last axis (sign -1)."""
    return _transform(x, -1.0)


def ifft_unnormalised(x: np.ndarray) -> np.ndarray:
    """Inverse DFT along the last axis without the 1/n factor (sign +1)."""
    return _transform(x, +1.0)


def dft_naive(x: np.ndarray, sign: float = -1.0) -> np.ndarray:
    """O(n^2) DFT by the defining sum; used only to pin ``fft`` on small n."""
    x = np.asarray(x, dtype=np.complex128)
    n = x.shape[-1]
    j = np.arange(n)
    # reduce j*k mod n exactly in integers before forming the angle
    jk = np.outer(j, j) % n
    mat = np.exp(sign * 2j * np.pi * np.arange(n) / n)[jk]
    return x @ mat.T
