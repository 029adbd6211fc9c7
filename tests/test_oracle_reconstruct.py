"""Pins of the oracle's direct convolution and window peaks by brute force and
by a library FFT convolution."""
import numpy as np

from oracle import reconstruct


def test_direct_matches_fft_circular_convolution():
    rng = np.random.default_rng(5)
    n = 512
    z = rng.standard_normal(n) + 1j * rng.standard_normal(n)
    for m0, L in [(0, 1), (3, 17), (-40, 33), (250, 255), (-256, 512)]:
        c = rng.standard_normal(L) + 1j * rng.standard_normal(L)
        rho = np.zeros(n, complex)
        rho[(m0 + np.arange(L)) % n] = c
        expect = np.fft.ifft(np.fft.fft(z) * np.fft.fft(rho))
        got = reconstruct.reconstruct_direct(z, m0, c)
        assert np.abs(got - expect).max() < 1e-11
        idx = np.array([0, 1, n // 2, n - 1])
        assert np.abs(reconstruct.reconstruct_at(z, m0, c, idx) - expect[idx]).max() < 1e-11


def test_direct_brute_force_tiny():
    z = np.array([1 + 2j, -1j, 3.0, 0.5 - 0.5j])
    c = np.array([2.0, 1j])
    m0 = -1
    n = 4
    expect = [sum(c[l] * z[(i - m0 - l) % n] for l in range(2)) for i in range(n)]
    assert np.allclose(reconstruct.reconstruct_direct(z, m0, c), expect, atol=1e-15)


def test_window_peaks_brute_force_with_ties_and_ragged_tail():
    rng = np.random.default_rng(2)
    for n, W in [(10, 3), (16, 4), (7, 7), (5, 8), (33, 8)]:
        z = np.round(rng.standard_normal(n) * 2) + 1j * np.round(rng.standard_normal(n) * 2)
        P, A = reconstruct.window_peaks(z, W)
        assert P.size == -(-n // W)
        for w in range(P.size):
            seg = [z[i].real ** 2 + z[i].imag ** 2 for i in range(w * W, min(n, (w + 1) * W))]
            best = max(seg)
            first = w * W + seg.index(best)
            assert P[w] == best and A[w] == first
