"""Pins of the oracle's template phase against closed forms and its own calculus."""
import json
import math
import os

import numpy as np
import pytest

from oracle import taylorf2, ratio
from workload import MSUN_S, Template, _masses_from_mchirp_eta

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")


def _chirp_time_closed_form(m1, m2, f, order):
    """Textbook chirp time: tau0 (Newtonian) and tau0 * (1 + 4/3 (743/336 + 11 eta / 4) v^2) (1PN)."""
    M = (m1 + m2) * MSUN_S
    eta = m1 * m2 / (m1 + m2) ** 2
    mc = M * eta ** 0.6
    tau0 = 5.0 / 256.0 * (math.pi * f) ** (-8.0 / 3.0) * mc ** (-5.0 / 3.0)
    if order == 0:
        return tau0
    v2 = (math.pi * M * f) ** (2.0 / 3.0)
    return tau0 * (1.0 + 4.0 / 3.0 * (743.0 / 336.0 + 11.0 * eta / 4.0) * v2)


def test_newtonian_and_1pn_chirp_time():
    for m1, m2, f in [(1.4, 1.4, 10.0), (2.8, 2.8, 40.0), (3.0, 1.0, 20.0)]:
        t0 = -taylorf2.time_of_frequency(np.array([f]), m1, m2, pn_order=0)[0]
        t1 = -taylorf2.time_of_frequency(np.array([f]), m1, m2, pn_order=2)[0]
        assert abs(t0 / _chirp_time_closed_form(m1, m2, f, 0) - 1) < 1e-13
        assert abs(t1 / _chirp_time_closed_form(m1, m2, f, 1) - 1) < 1e-13
    # the well-known ~1000 s of a 1.4+1.4 binary from 10 Hz at leading order
    assert 990 < _chirp_time_closed_form(1.4, 1.4, 10.0, 0) < 1010


@pytest.mark.parametrize("pn", [2, 7])
def test_derivatives_match_finite_differences(pn):
    m1, m2 = 1.9, 1.3
    f = np.array([15.0, 20.0, 45.0, 130.0, 600.0])
    h = 1e-3 * f
    psi = lambda g: taylorf2.phase(g, m1, m2, pn, tc=0.3, phic=0.7)
    d1_fd = (-psi(f + 2 * h) + 8 * psi(f + h) - 8 * psi(f - h) + psi(f - 2 * h)) / (12 * h)
    d1 = taylorf2.dphase(f, m1, m2, pn, tc=0.3)
    assert np.max(np.abs(d1_fd / d1 - 1)) < 1e-7
    dp = lambda g: taylorf2.dphase(g, m1, m2, pn, tc=0.3)
    d2_fd = (-dp(f + 2 * h) + 8 * dp(f + h) - 8 * dp(f - h) + dp(f - 2 * h)) / (12 * h)
    d2 = taylorf2.d2phase(f, m1, m2, pn)
    assert np.max(np.abs(d2_fd / d2 - 1)) < 1e-7


def test_tc_and_phic_enter_linearly():
    f = np.linspace(20, 900, 50)
    base = taylorf2.phase(f, 1.5, 1.2, 7)
    shifted = taylorf2.phase(f, 1.5, 1.2, 7, tc=2.5, phic=0.4)
    assert np.allclose(shifted - base, 2 * np.pi * f * 2.5 - 0.4, rtol=0, atol=1e-8)


def test_amplitude_law_and_sign():
    f = np.array([30.0, 60.0])
    h = taylorf2.template_fd(f, 1.4, 1.4, 7)
    assert np.allclose(np.abs(h), f ** (-7 / 6), rtol=1e-14)
    # h = B exp(-i Psi): the phase of h is -Psi mod 2 pi
    psi = taylorf2.phase(f, 1.4, 1.4, 7)
    assert np.allclose(np.angle(h * np.exp(1j * psi)), 0.0, atol=1e-9)


def test_fig1_fig2_printed_values():
    """Fig. 1: ~300 s templates; Fig. 2: df_low = 1.92 Hz for that pair (Eq. 10)."""
    g = json.load(open(os.path.join(GOLDEN, "fig2_dflow.json")))
    r = Template(*_masses_from_mchirp_eta(g["reference_mchirp_msun"], 0.25))
    t = Template(*_masses_from_mchirp_eta(g["target_mchirp_msun"], 0.25))
    tau = -taylorf2.time_of_frequency(np.array([g["f_low_hz"]]), r.m1, r.m2, 7)[0]
    assert 0.8 * g["printed_duration_s"] < tau < 1.1 * g["printed_duration_s"]
    d = ratio.df_low_rule(r, t, 7, g["f_low_hz"], df_low_max=1e9)
    # chirp masses given to ~3 digits admit df_low in about [1.5, 1.9]; the rule's
    # scale (square root, 2 pi) is pinned to 20% by the printed 1.92 Hz
    assert abs(d / g["printed_df_low_hz"] - 1) < 0.2
    # masses within the caption's rounding reproduce the printed value closely
    r2 = Template(*_masses_from_mchirp_eta(0.8745, 0.25))
    t2 = Template(*_masses_from_mchirp_eta(0.8707, 0.25))
    assert abs(ratio.df_low_rule(r2, t2, 7, 20.0, 1e9) - g["printed_df_low_hz"]) < 0.1


# --- independent pin of the 3.5PN phase: the energy-balance law --------------------------
#
# The stationary-phase template's t(f) obeys dt/dv = -E'(v) / F(v) (energy balance, with
# v = (pi M f)^(1/3)): binding energy E = -(eta M v^2 / 2) e(v) and gravitational-wave flux
# F = (32/5) eta^2 v^10 phi(v), both non-spinning post-Newtonian series published in
# Blanchet, Living Rev. Relativ. 17, 2 (2014), energy to 3PN and flux to 3.5PN.  TaylorF2
# integrates the ratio re-expanded to relative order v^7, so
#   dt/dv = (5 M / (32 eta)) v^-9 * sum_{k<=7} c_k v^k
# with ln v held as a parameter in the expansion; no integration constant enters dt/dv, so
# every phase coefficient alpha_2..alpha_7 (log terms included) is fixed by it.


def _energy_flux_series(v, eta):
    """c_0..c_7 of (1 + 2 e2 v^2 + 3 e4 v^4 + 4 e6 v^6) / phi(v), ln v taken at this v,
    and the coefficient of ln v inside c_6."""
    pi = math.pi
    e2 = -3.0 / 4.0 - eta / 12.0
    e4 = -27.0 / 8.0 + 19.0 / 8.0 * eta - eta ** 2 / 24.0
    e6 = (-675.0 / 64.0 + (34445.0 / 576.0 - 205.0 / 96.0 * pi ** 2) * eta - 155.0 / 96.0 * eta ** 2
          - 35.0 / 5184.0 * eta ** 3)
    num = [1.0, 0.0, 2 * e2, 0.0, 3 * e4, 0.0, 4 * e6, 0.0]
    den = [1.0, 0.0,
           -1247.0 / 336.0 - 35.0 / 12.0 * eta,
           4.0 * pi,
           -44711.0 / 9072.0 + 9271.0 / 504.0 * eta + 65.0 / 18.0 * eta ** 2,
           (-8191.0 / 672.0 - 583.0 / 24.0 * eta) * pi,
           (6643739519.0 / 69854400.0 + 16.0 / 3.0 * pi ** 2 - 1712.0 / 105.0 * 0.5772156649015329
            - 856.0 / 105.0 * math.log(16.0 * v * v)
            + (-134543.0 / 7776.0 + 41.0 / 48.0 * pi ** 2) * eta - 94403.0 / 3024.0 * eta ** 2
            - 775.0 / 324.0 * eta ** 3),
           (-16285.0 / 504.0 + 214745.0 / 1728.0 * eta + 193385.0 / 3024.0 * eta ** 2) * pi]
    c = []
    for k in range(8):  # power-series division num / den, den[0] = 1
        c.append(num[k] - sum(den[j] * c[k - j] for j in range(1, k + 1)))
    # ln v enters only through den[6] * c_0: -(856/105) * 2 ln v, with the opposite sign in c_6
    c6_log = 1712.0 / 105.0 * c[0]
    return c, c6_log


_PN_CASES = [(0.25, 2.8), (0.2, 4.0), (0.1875, 4.0), (0.1, 3.0)]  # (eta, total mass in Msun)
_PN_V = [0.05, 0.1, 0.2, 0.3]


def _component_masses(eta, mt):
    m1 = mt * (1.0 + math.sqrt(1.0 - 4.0 * eta)) / 2.0
    return m1, mt - m1


def _energy_balance_errors():
    """Largest relative misfit of the oracle's t'(v) and t(v) against the energy-balance series."""
    worst_d, worst_t = 0.0, 0.0
    for eta, mt in _PN_CASES:
        m1, m2 = _component_masses(eta, mt)
        M = mt * MSUN_S
        scale = 5.0 * M / (32.0 * eta)
        for v in _PN_V:
            f = np.array([v ** 3 / (math.pi * M)])
            c, c6_log = _energy_flux_series(v, eta)
            # dt/dv from Psi'' = 2 pi (dt/dv)(dv/df), dv/df = pi M / (3 v^2)
            dtdv = taylorf2.d2phase(f, m1, m2, 7)[0] / (2.0 * math.pi) / (math.pi * M / (3.0 * v * v))
            want_d = scale * sum(c[k] * v ** (k - 9) for k in range(8))
            worst_d = max(worst_d, abs(dtdv / want_d - 1.0))
            # t(v) - t_c = integral from infinity of dt/dv: each c_k u^(k-9) gives c_k v^(k-8)/(k-8);
            # the ln u inside c_6 adds -c6_log / (4 v^2) (from the integral of u^-3 ln u)
            t = taylorf2.time_of_frequency(f, m1, m2, 7, tc=0.0)[0]
            want_t = scale * (sum(c[k] * v ** (k - 8) / (k - 8) for k in range(8)) - c6_log / (4.0 * v * v))
            worst_t = max(worst_t, abs(t / want_t - 1.0))
    return worst_d, worst_t


def test_phase_follows_the_energy_balance_of_the_pn_energy_and_flux():
    """Every 3.5PN coefficient of the oracle's Psi (Sec. II.B template family; Eq. A2 for
    t = Psi' / 2 pi) against the energy and flux series of an independent source."""
    worst_d, worst_t = _energy_balance_errors()
    assert worst_d < 1e-12
    assert worst_t < 1e-12


@pytest.mark.parametrize("k", [2, 3, 4, 5, 6, 7, "log5", "log6"])
def test_energy_balance_pin_detects_a_changed_coefficient(monkeypatch, k):
    """A mistake planted in one phase coefficient of the oracle (relative 1e-6) fails the pin."""
    orig = taylorf2._coeffs

    def planted(eta, pn_order):
        a, a5log, a6log = orig(eta, pn_order)
        a = dict(a)
        if k == "log5":
            a5log *= 1.0 + 1e-6
        elif k == "log6":
            a6log *= 1.0 + 1e-6
        else:
            a[k] *= 1.0 + 1e-6
        return a, a5log, a6log

    monkeypatch.setattr(taylorf2, "_coeffs", planted)
    worst_d, worst_t = _energy_balance_errors()
    if k == 5:
        # the constant part of alpha_5 is a constant phase (it sets no t(f)): by design
        # invisible to the pin, as it is to |z|
        assert worst_d < 1e-12 and worst_t < 1e-12
    else:
        assert max(worst_d, worst_t) > 1e-10
