"""The index algebra of the two-pass four-step FFT (the matched filter's transforms at
n = 2^18 .. 2^24), checked on the host: with j = N2 a + b and k = k1 + N1 k2, column DFTs of N1
points, the inter-pass twiddle w_n^(b k1) (formed as the kernel forms it: two small tables,
w_n^(b ltid) e^u with e = w_n^(b NT) and the powers of e by products), row DFTs of N2 points and
the transposed store give the DFT of Eq. 1.  numpy's FFT serves as the reference transform.
"""
import numpy as np
import pytest


def _tables(n):
    lo = (int(np.log2(n)) + 1) // 2
    m_lo = np.arange(1 << lo)
    m_hi = np.arange(n >> lo) << lo
    return lo, np.exp(-2j * np.pi * m_lo / n), np.exp(-2j * np.pi * m_hi / n)


def _twiddles(n, n1, n2, dtype):
    """w_n^(b k1) for every column b and bin k1, as the column pass forms them: k1 = ltid + NT u
    with NT = N1 / 16; w = w_n^(b ltid) e^u, e, e^2, e^4, e^8 from the tables, e^3, e^5..e^7 by
    products, e^(u + 8) = e^u e^8; every product rounded to dtype."""
    lo, t_lo, t_hi = _tables(n)
    t_lo, t_hi = t_lo.astype(dtype), t_hi.astype(dtype)
    nt = n1 // 16
    b = np.arange(n2)[:, None]
    ltid = np.arange(nt)[None, :]
    tab = lambda m: (t_lo[m & ((1 << lo) - 1)] * t_hi[m >> lo]).astype(dtype)
    b0 = tab(b * ltid)
    e1, e2, e4, e8 = (tab(b * (s * nt)) for s in (1, 2, 4, 8))
    pows = {0: np.ones_like(e1), 1: e1, 2: e2, 3: (e2 * e1).astype(dtype), 4: e4, 5: (e4 * e1).astype(dtype),
            6: (e4 * e2).astype(dtype), 7: (e4 * (e2 * e1).astype(dtype)).astype(dtype)}
    w = np.empty((n2, n1), dtype=dtype)
    for u in range(8):
        wu = b0 if u == 0 else (b0 * pows[u]).astype(dtype)
        w8 = (wu * e8).astype(dtype)
        w[:, ltid[0] + nt * u] = wu
        w[:, ltid[0] + nt * (u + 8)] = w8
    return w


@pytest.mark.parametrize("logn", [18, 19, 20])
@pytest.mark.parametrize("sign", [-1, +1])
def test_four_step_decomposition(logn, sign):
    n = 1 << logn
    n1 = 1 << (logn // 2)
    n2 = n // n1
    rng = np.random.default_rng(logn)
    x = rng.standard_normal(n) + 1j * rng.standard_normal(n)
    w = _twiddles(n, n1, n2, np.complex128)
    if sign > 0:
        w = np.conj(w)
    a = x.reshape(n1, n2)                                       # a[a_, b] = x[N2 a_ + b]
    y = np.fft.fft(a, axis=0) if sign < 0 else np.fft.ifft(a, axis=0) * n1   # columns: bin k1
    y = y * w.T                                                 # w_n^(b k1)
    zz = np.fft.fft(y, axis=1) if sign < 0 else np.fft.ifft(y, axis=1) * n2   # rows: bin k2
    out = np.empty(n, complex)
    out[(np.arange(n1)[:, None] + n1 * np.arange(n2)[None, :]).ravel()] = zz.ravel()
    ref = np.fft.fft(x) if sign < 0 else np.fft.ifft(x) * n
    assert np.abs(out - ref).max() <= 1e-12 * np.abs(ref).max()


def test_twiddle_powers_in_fp32_stay_within_a_few_ulp():
    """The FP32 twiddles the column pass forms (table products and powers) against exact ones:
    within 8 FP32 ulp of a unit-modulus value."""
    logn = 20
    n = 1 << logn
    n1 = 1 << (logn // 2)
    n2 = n // n1
    w32 = _twiddles(n, n1, n2, np.complex64).astype(np.complex128)
    b = np.arange(n2)[:, None]
    k1 = np.arange(n1)[None, :]
    exact = np.exp(-2j * np.pi * ((b * k1) % n) / n)
    assert np.abs(w32 - exact).max() <= 8 * 2.0 ** -24
