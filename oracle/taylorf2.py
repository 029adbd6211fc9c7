"""Stationary-phase inspiral templates (oracle; test infrastructure only).

App. A, Eq. (A1): h~(f) = B(f) exp(-i Psi(f)) for f > 0, with Eq. (A2):
Psi'(f) = 2 pi t(f).  The template family is TaylorF2 (cited in Sec. II.B):

  Psi(f) = 2 pi f t_c - phi_c - pi/4 + 3 / (128 eta v^5) * sum_k alpha_k v^k,
  v = (pi M f)^(1/3),  M = total mass in seconds,

with the non-spinning post-Newtonian coefficients alpha_0..alpha_7 of
Buonanno, Iyer, Ochsner, Pan & Sathyaprakash (2009); pn_order = 2 keeps
alpha_0 and alpha_2 (1PN), pn_order = 7 keeps all (3.5PN).  The amplitude is
B(f) = f^(-7/6) with unit scale: every SNR is normalised by N (Eq. 3), so the
scale cancels.

t(f) and Psi''(f) are the analytic derivatives of the series, taken term by
term through dv/df = v / (3 f).
"""
from __future__ import annotations

import math
from typing import Tuple

import numpy as np

MSUN_S = 4.925491025543576e-6
EULER_GAMMA = 0.5772156649015329
V_LSO = 1.0 / math.sqrt(6.0)


def _coeffs(eta: float, pn_order: int) -> Tuple[dict, float, float]:
    """Constant parts of alpha_k, plus the coefficients of the two log terms.

    alpha_5(v) = a5 (1 + 3 ln(v / v_lso));  alpha_6(v) = a6 - (6848/21) ln(4 v).
    Returns ({k: alpha_k constant part}, a5_log_coeff, a6_log_coeff) where the
    log pieces are a5 * 3 ln(v/v_lso) and -(6848/21) ln(4v).
    """
    pi = math.pi
    a = {0: 1.0}
    a5log = 0.0
    a6log = 0.0
    if pn_order >= 2:
        a[2] = 3715.0 / 756.0 + 55.0 * eta / 9.0
    if pn_order >= 3:
        a[3] = -16.0 * pi
    if pn_order >= 4:
        a[4] = 15293365.0 / 508032.0 + 27145.0 * eta / 504.0 + 3085.0 * eta ** 2 / 72.0
    if pn_order >= 5:
        a5 = pi * (38645.0 / 756.0 - 65.0 * eta / 9.0)
        a[5] = a5
        a5log = 3.0 * a5
    if pn_order >= 6:
        a[6] = (11583231236531.0 / 4694215680.0 - 6848.0 * EULER_GAMMA / 21.0 - 640.0 * pi ** 2 / 3.0
                + (-15737765635.0 / 3048192.0 + 2255.0 * pi ** 2 / 12.0) * eta
                + 76055.0 * eta ** 2 / 1728.0 - 127825.0 * eta ** 3 / 1296.0)
        a6log = -6848.0 / 21.0
    if pn_order >= 7:
        a[7] = pi * (77096675.0 / 254016.0 + 378515.0 * eta / 1512.0 - 74045.0 * eta ** 2 / 756.0)
    return a, a5log, a6log


def _masses(m1: float, m2: float) -> Tuple[float, float]:
    mt = m1 + m2
    return mt * MSUN_S, m1 * m2 / mt ** 2


def series(v: np.ndarray, eta: float, pn_order: int) -> Tuple[np.ndarray, np.ndarray, np.ndarray]:
    """g(v) = sum_k alpha_k(v) v^(k-5) and its first two v-derivatives."""
    a, a5log, a6log = _coeffs(eta, pn_order)
    v = np.asarray(v, dtype=np.float64)
    g = np.zeros_like(v)
    g1 = np.zeros_like(v)
    g2 = np.zeros_like(v)
    for k, ak in a.items():
        p = k - 5
        g += ak * v ** p
        g1 += ak * p * v ** (p - 1)
        g2 += ak * p * (p - 1) * v ** (p - 2)
    if a5log:
        # a5log * ln(v/v_lso) * v^0
        g += a5log * np.log(v / V_LSO)
        g1 += a5log / v
        g2 += -a5log / v ** 2
    if a6log:
        # a6log * ln(4 v) * v^1
        g += a6log * np.log(4.0 * v) * v
        g1 += a6log * (np.log(4.0 * v) + 1.0)
        g2 += a6log / v
    return g, g1, g2


def phase(f: np.ndarray, m1: float, m2: float, pn_order: int, tc: float = 0.0, phic: float = 0.0) -> np.ndarray:
    """Psi(f) in radians (FP64), f > 0."""
    M, eta = _masses(m1, m2)
    f = np.asarray(f, dtype=np.float64)
    v = np.cbrt(math.pi * M * f)
    g, _, _ = series(v, eta, pn_order)
    return 2.0 * math.pi * f * tc - phic - math.pi / 4.0 + 3.0 / (128.0 * eta) * g


def dphase(f: np.ndarray, m1: float, m2: float, pn_order: int, tc: float = 0.0) -> np.ndarray:
    """Psi'(f) = 2 pi t(f)  (Eq. A2)."""
    M, eta = _masses(m1, m2)
    f = np.asarray(f, dtype=np.float64)
    v = np.cbrt(math.pi * M * f)
    _, g1, _ = series(v, eta, pn_order)
    # d/df = (v / (3 f)) d/dv and v / (3 f) = pi M / (3 v^2)
    return 2.0 * math.pi * tc + (math.pi * M / (128.0 * eta)) * g1 / v ** 2


def d2phase(f: np.ndarray, m1: float, m2: float, pn_order: int) -> np.ndarray:
    """Psi''(f) = 2 pi t'(f)  (Eq. A2)."""
    M, eta = _masses(m1, m2)
    f = np.asarray(f, dtype=np.float64)
    v = np.cbrt(math.pi * M * f)
    _, g1, g2 = series(v, eta, pn_order)
    dv_df = math.pi * M / (3.0 * v ** 2)
    return (math.pi * M / (128.0 * eta)) * (g2 / v ** 2 - 2.0 * g1 / v ** 3) * dv_df


def time_of_frequency(f, m1, m2, pn_order, tc=0.0):
    """t(f) = Psi'(f) / (2 pi)  (Eq. A2)."""
    return dphase(f, m1, m2, pn_order, tc) / (2.0 * math.pi)


def amplitude(f: np.ndarray) -> np.ndarray:
    """B(f) = f^(-7/6) (unit scale; Eq. A1)."""
    f = np.asarray(f, dtype=np.float64)
    return f ** (-7.0 / 6.0)


def template_fd(f: np.ndarray, m1, m2, pn_order, tc=0.0, phic=0.0) -> np.ndarray:
    """h~(f) = B(f) exp(-i Psi(f)) for f > 0 (Eq. A1); 0 at f <= 0."""
    f = np.asarray(f, dtype=np.float64)
    out = np.zeros(f.shape, dtype=np.complex128)
    pos = f > 0
    psi = phase(f[pos], m1, m2, pn_order, tc, phic)
    out[pos] = amplitude(f[pos]) * np.exp(-1j * psi)
    return out
