"""Pins of the oracle's radix-2 FFT against the defining DFT sum and identities."""
import numpy as np
import pytest

from oracle import fft


@pytest.mark.parametrize("p", range(0, 13))
def test_fft_matches_naive_dft(p):
    n = 1 << p
    rng = np.random.default_rng(p)
    x = rng.standard_normal(n) + 1j * rng.standard_normal(n)
    ref = fft.dft_naive(x, -1.0)
    got = fft.fft(x)
    scale = max(1.0, np.abs(ref).max())
    assert np.abs(got - ref).max() / scale < 1e-12
    ref_i = fft.dft_naive(x, +1.0)
    got_i = fft.ifft_unnormalised(x)
    assert np.abs(got_i - ref_i).max() / scale < 1e-12


def test_fft_matches_library_large():
    rng = np.random.default_rng(7)
    x = rng.standard_normal(1 << 16) + 1j * rng.standard_normal(1 << 16)
    assert np.allclose(fft.fft(x), np.fft.fft(x), rtol=0, atol=1e-9)
    assert np.allclose(fft.ifft_unnormalised(x), np.fft.ifft(x) * x.size, rtol=0, atol=1e-9)


def test_parseval_and_round_trip():
    rng = np.random.default_rng(3)
    n = 1 << 14
    x = rng.standard_normal(n) + 1j * rng.standard_normal(n)
    X = fft.fft(x)
    assert abs(np.sum(np.abs(X) ** 2) / n - np.sum(np.abs(x) ** 2)) / np.sum(np.abs(x) ** 2) < 1e-13
    back = fft.ifft_unnormalised(X) / n
    assert np.abs(back - x).max() < 1e-13


def test_fft_delta_and_tone():
    n = 256
    d = np.zeros(n, complex)
    d[5] = 1.0
    k = np.arange(n)
    assert np.allclose(fft.fft(d), np.exp(-2j * np.pi * 5 * k / n), atol=1e-14)
    tone = np.exp(2j * np.pi * 17 * k / n)
    X = fft.fft(tone)
    assert abs(X[17] - n) < 1e-11 and np.abs(np.delete(X, 17)).max() < 1e-11


def test_fft_rejects_non_power_of_two():
    with pytest.raises(ValueError):
        fft.fft(np.ones(6))
