"""Synthetic strain with injections (oracle; test infrastructure only).

Sec. III.B: coloured Gaussian noise plus injected inspirals, each scaled so
that its optimal SNR in zero noise (matched with itself) is the requested
value.  The seeded noise draws and injection parameters come from the shared
``workload`` module; the injected waveforms use this oracle's own templates.

An injection of template h arriving at sample s is a h~(f) with t_c = s dt,
restricted to [f_low, f_high], with a = rho_opt / N (Eq. 3).  The real strain
is x[j] = (1/(n dt)) sum_{k=0}^{n-1} x~_k exp(+2 pi i j k / n) with the
Hermitian continuation x~_{n-k} = conj(x~_k).
"""
from __future__ import annotations

import numpy as np

import workload
from . import fft as _fft
from .mf import band_limited_inv_psd, freqs, sigma, template


def injection_spectrum(cfg, inv_psd: np.ndarray) -> np.ndarray:
    n, fs = cfg.n, cfg.fs
    ipb = band_limited_inv_psd(inv_psd, n, fs, cfg.f_low, cfg.f_high)
    band = ipb > 0
    out = np.zeros(n // 2 + 1, dtype=np.complex128)
    for inj in cfg.injections:
        ref, nbrs = cfg.groups[inj.group]
        t = ref if inj.template_index < 0 else nbrs[inj.template_index]
        h = template(n, fs, t.m1, t.m2, cfg.pn_order, tc=inj.sample / fs)
        a = inj.snr / sigma(h, ipb, fs / n)
        out += np.where(band, a * h, 0.0)
    return out


def spectrum_to_strain(xf: np.ndarray, n: int, fs: float) -> np.ndarray:
    full = np.zeros(n, dtype=np.complex128)
    full[: n // 2 + 1] = xf
    full[n // 2 + 1:] = np.conj(xf[1: n // 2][::-1])
    return (_fft.ifft_unnormalised(full).real * fs / n)


def strain(cfg, realisation: int = 0, noise: bool = True, injections: bool = True) -> np.ndarray:
    """Real strain x (float64, or float32-rounded for the FP32 configurations)."""
    ip = workload.inv_psd(cfg)
    xf = np.zeros(cfg.n // 2 + 1, dtype=np.complex128)
    if noise:
        xf = xf + workload.noise_spectrum(cfg, realisation)
    if injections:
        xf = xf + injection_spectrum(cfg, ip)
    x = spectrum_to_strain(xf, cfg.n, cfg.fs)
    if cfg.dtype == "f32":
        x = x.astype(np.float32).astype(np.float64)
    return x
