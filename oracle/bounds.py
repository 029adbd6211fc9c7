"""App. A approximations of the ratio kernel (oracle; test infrastructure only).

With the discrete kernel rho[m] = (1/n) sum_k K~_k exp(2 pi i k m / n) and
K~ = W exp(+i dPsi) (unit R), rho[m] ~ dt * q(-m dt) with
q(t) = int W R exp(2 pi i f t - i dPsi(f)) df, the complex integrand of Eq. (A5)
(the paper's r(t) is 2 Re q(t)).  The stationary point of the lag-m term is
where dt(f) = -m dt, dt(f) = t(f) - t_ref(f).

* Eq. (A11) (stationary region): |q| ~ R / sqrt(|dt'(f*)|), so
  |rho[m]| ~ dt * R / sqrt(|dt'(f*)|).
* Eq. (A9) (low side):  |q| <= R / (4 pi df_low^2 |dt(f_low) - t|^3).
* Eq. (A10) (high side): |q| <= R / (4 pi df_high^2 |t - dt(f_high)|^3).

Analytic truncation (Sec. II.D: the kept region is found from the App. A expressions).
Reading: the windowed band's stationary points run from the outer end of the low taper,
f_low - df_low, to the outer end of the high one, f_high + df_high (inside a taper the
amplitude is the stationary one times W, and where dt' is large the taper alone spans a good
part of a second); the ends of each taper (f_low - df_low and f_low with df_low, f_high and
f_high + df_high with df_high) add endpoint contributions that decay on both sides of their
times as the Eq. (A9)/(A10) bound R(f_e) / (4 pi df_e^2 |t - dt(f_e)|^3) on |r| (the low taper
is narrow, so its tail reaches past the high edge as well).  With a threshold amplitude A on
|r| the kept lag times are the union of [c_e - d_e, c_e + d_e] over the four taper ends,
c_e = -dt(f_e) on the kernel's axis and d_e = (R(f_e) / (4 pi df_e^2 A))^(1/3): the interval
from the smallest c_e - d_e to the largest c_e + d_e, which contains the stationary region
(dt monotonic).  A relative threshold takes A = thr max|r|, with |r| = 2 |q| = 2 fs |rho| /
(N_ref / N) the kernel's own peak; an absolute one takes A = thr in 1/s (the paper's threshold
amplitude).  Lags: floor and ceil of the end times times fs; a span as long as the grid keeps
the whole grid from lag 0.
"""
from __future__ import annotations

import math

import numpy as np

from . import taylorf2


def delta_t(f, ref, tgt, pn_order):
    """dt(f) = t(f) - t_ref(f) (App. A)."""
    return taylorf2.time_of_frequency(f, tgt.m1, tgt.m2, pn_order, tgt.tc) - \
        taylorf2.time_of_frequency(f, ref.m1, ref.m2, pn_order, ref.tc)


def delta_t_prime(f, ref, tgt, pn_order):
    """dt'(f) = dPsi''(f) / (2 pi)."""
    return (taylorf2.d2phase(f, tgt.m1, tgt.m2, pn_order) -
            taylorf2.d2phase(f, ref.m1, ref.m2, pn_order)) / (2.0 * math.pi)


def stationary_envelope(lags_s: np.ndarray, ref, tgt, pn_order, f_low, f_high, dt_s) -> np.ndarray:
    """Eq. (A11) amplitude at lag times t = m dt: dt / sqrt(|dt'(f*)|) with
    dt(f*) = -t, for lags whose f* lies in (f_low, f_high); NaN elsewhere."""
    f = np.linspace(f_low, f_high, 20001)
    d = delta_t(f, ref, tgt, pn_order)
    order = np.argsort(d)
    target = -np.asarray(lags_s, dtype=np.float64)
    fstar = np.interp(target, d[order], f[order], left=np.nan, right=np.nan)
    out = np.full(target.shape, np.nan)
    ok = np.isfinite(fstar)
    out[ok] = dt_s / np.sqrt(np.abs(delta_t_prime(fstar[ok], ref, tgt, pn_order)))
    return out


def low_tail_bound(lags_s, ref, tgt, pn_order, f_low, df_low, dt_s):
    """Eq. (A9) converted to |rho|: dt / (4 pi df_low^2 |dt(f_low) + m dt|^3)."""
    d0 = delta_t(np.array([f_low]), ref, tgt, pn_order)[0]
    return dt_s / (4.0 * math.pi * df_low ** 2 * np.abs(d0 + np.asarray(lags_s)) ** 3)


def high_tail_bound(lags_s, ref, tgt, pn_order, f_high, df_high, dt_s):
    """Eq. (A10) converted to |rho|: dt / (4 pi df_high^2 |m dt + dt(f_high)|^3)."""
    d1 = delta_t(np.array([f_high]), ref, tgt, pn_order)[0]
    return dt_s / (4.0 * math.pi * df_high ** 2 * np.abs(np.asarray(lags_s) + d1) ** 3)


def analytic_span(ref, tgt, pn_order, f_low, f_high, df_low, df_high, fs, nb, amp) -> tuple:
    """Kept lags of the analytic truncation at threshold amplitude ``amp`` on |r| (1/s):
    (m0 signed on the nb circle, L).  An infinite amplitude keeps the edge lags only."""
    fe = np.array([f_low - df_low, f_low, f_high, f_high + df_high])
    t_e = (taylorf2.dphase(fe, tgt.m1, tgt.m2, pn_order) - taylorf2.dphase(fe, ref.m1, ref.m2, pn_order)) / \
        (2.0 * math.pi)
    R_e = taylorf2.amplitude(fe) / taylorf2.amplitude(fe)          # B / B_ref (same law)
    dfe = np.array([df_low, df_low, df_high, df_high])
    d_e = np.cbrt(R_e / (4.0 * math.pi * dfe * dfe * amp))
    c_e = -t_e
    lo = float(np.min(c_e - d_e))
    hi = float(np.max(c_e + d_e))
    if not (math.ceil(hi * fs) - math.floor(lo * fs) + 1.0 < nb):   # the whole grid, from lag 0
        return 0, int(nb)
    m_lo = math.floor(lo * fs)
    m_hi = math.ceil(hi * fs)
    m0 = m_lo % nb
    return (m0 if m0 <= nb // 2 else m0 - nb), int(m_hi - m_lo + 1)
