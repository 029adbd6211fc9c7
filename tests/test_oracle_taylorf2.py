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
