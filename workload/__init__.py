"""Seeded synthetic inputs for the ratio-filter hot path.

This module is shared by the FP64 oracle and by the CUDA path.  It holds no
step of the method itself: no template phase, no matched filter, no ratio
kernel.  It only produces

* the five workload configurations (grid, band, bank recipe, injection recipe),
* the one-sided noise PSD ``S_n(f)`` (an input of the method, Sec. II.A),
* seeded standard-normal draws for the coloured noise,
* seeded template-bank parameters (component masses, coalescence time/phase),
* seeded injection parameters (which template, arrival sample, optimal SNR).

Turning these into a strain time series needs the template model, so that is
done by each side with its own code (``oracle.data`` for the oracle; the
library's own template routine for the CUDA path).

Seeds are ``1000 * config + stream`` (stream 0 noise, 1 bank, 2 injections).
"""
from __future__ import annotations

from dataclasses import dataclass, field, replace
from typing import List, Optional, Tuple

import numpy as np

MSUN_S = 4.925491025543576e-6  # G M_sun / c^3 in seconds


@dataclass(frozen=True)
class Template:
    """Non-spinning inspiral template, detector-frame component masses in M_sun."""
    m1: float
    m2: float
    tc: float = 0.0     # coalescence time in seconds (0: merger at sample 0)
    phic: float = 0.0   # coalescence phase in radians

    @property
    def mtotal(self) -> float:
        return self.m1 + self.m2

    @property
    def eta(self) -> float:
        return self.m1 * self.m2 / (self.m1 + self.m2) ** 2

    @property
    def mchirp(self) -> float:
        return self.mtotal * self.eta ** 0.6


@dataclass(frozen=True)
class Injection:
    template_index: int   # index into the group's neighbour list (-1: the reference)
    group: int            # reference group the injected template belongs to
    sample: int           # arrival (coalescence) sample index
    snr: float            # optimal SNR in zero noise


@dataclass(frozen=True)
class Config:
    index: int
    name: str
    n: int
    fs: float
    f_low: float
    f_high: float
    pn_order: int                  # 2 (1PN) or 7 (3.5PN)
    dtype: str                     # "f64" or "f32" (data and complex outputs)
    threshold: float = 1e-3        # relative truncation threshold
    df_high: float = 53.0
    df_low_max: float = 5.0
    window_s: float = 1.0          # peak-window length in seconds
    groups: Tuple[Tuple[Template, Tuple[Template, ...]], ...] = field(default=(), repr=False)
    injections: Tuple[Injection, ...] = field(default=(), repr=False)
    noise_f_min: float = 0.0       # noise is generated for f >= noise_f_min only

    @property
    def dt(self) -> float:
        return 1.0 / self.fs

    @property
    def duration(self) -> float:
        return self.n / self.fs

    @property
    def df(self) -> float:
        return self.fs / self.n

    @property
    def window(self) -> int:
        return int(round(self.window_s * self.fs))

    @property
    def n_templates(self) -> int:
        return sum(1 + len(nb) for _, nb in self.groups)


def seed(config_index: int, stream: int) -> int:
    return 1000 * config_index + stream


# --------------------------------------------------------------------------
# Noise PSD (input; the paper uses a tabulated design curve, which is not here)
# --------------------------------------------------------------------------

def psd(f: np.ndarray) -> np.ndarray:
    """Analytic aLIGO-like one-sided PSD fit, x = f / 215 Hz, unit overall scale.

    S(x) = x^-4.14 - 5 x^-2 + 111 (1 - x^2 + x^4 / 2) / (1 + x^2 / 2).
    The overall scale cancels in the normalised SNR, so it is 1.  S(0) = inf.
    """
    f = np.asarray(f, dtype=np.float64)
    with np.errstate(divide="ignore", invalid="ignore"):
        x = f / 215.0
        s = x ** -4.14 - 5.0 / x ** 2 + 111.0 * (1.0 - x ** 2 + 0.5 * x ** 4) / (1.0 + 0.5 * x ** 2)
    return np.where(f > 0, s, np.inf)


def inv_psd(cfg: Config) -> np.ndarray:
    """1 / S_n(f_k) at the n/2+1 one-sided bins f_k = k df (0 at DC).

    The band limitation of Sec. II.A is NOT applied here; both implementations
    apply it themselves from (f_low, f_high).
    """
    f = np.arange(cfg.n // 2 + 1, dtype=np.float64) * cfg.df
    s = psd(f)
    out = np.zeros_like(f)
    ok = np.isfinite(s)
    out[ok] = 1.0 / s[ok]
    return out


def noise_normals(cfg: Config, realisation: int = 0) -> Tuple[np.ndarray, np.ndarray]:
    """Two independent standard-normal arrays (a, b) of length n/2+1."""
    rng = np.random.default_rng([seed(cfg.index, 0), realisation])
    a = rng.standard_normal(cfg.n // 2 + 1)
    b = rng.standard_normal(cfg.n // 2 + 1)
    return a, b


def noise_spectrum(cfg: Config, realisation: int = 0) -> np.ndarray:
    """One-sided coloured-noise spectrum (continuous-FT normalisation).

    x~[k] = sqrt(T S_k / 4) (a + i b) for 0 < k < n/2, so E|x~|^2 = T S_k / 2
    (one-sided PSD convention); the Nyquist bin is real with the same variance.
    Bins with f_k < noise_f_min (and DC) are zero: the synthetic strain is
    high-passed, as a search pipeline's conditioned data are, so that an FP32
    time series keeps its in-band precision.
    """
    a, b = noise_normals(cfg, realisation)
    n = cfg.n
    f = np.arange(n // 2 + 1) * cfg.df
    s = psd(f)
    amp = np.zeros(n // 2 + 1)
    keep = (f >= max(cfg.noise_f_min, cfg.df)) & np.isfinite(s)
    amp[keep] = np.sqrt(cfg.duration * s[keep] / 4.0)
    xf = amp * (a + 1j * b)
    xf[-1] = np.sqrt(2.0) * amp[-1] * a[-1]
    xf[0] = 0.0
    return xf


# --------------------------------------------------------------------------
# Template banks (A15 reading: a seeded lattice in duration offset x mass ratio)
# --------------------------------------------------------------------------

def newtonian_duration(t: Template, f: float) -> float:
    """Leading-order time to coalescence from frequency f (bank layout only)."""
    mc = t.mchirp * MSUN_S
    return 5.0 / 256.0 * (np.pi * f) ** (-8.0 / 3.0) * mc ** (-5.0 / 3.0)


def _masses_from_mchirp_eta(mc: float, eta: float) -> Tuple[float, float]:
    m = mc / eta ** 0.6
    d = np.sqrt(max(0.0, 1.0 - 4.0 * eta))
    return 0.5 * m * (1.0 + d), 0.5 * m * (1.0 - d)


def duration_lattice(ref: Template, f_low: float, k: int, dtau_min: float, dtau_max: float,
                     rng: np.random.Generator, eta_range=(0.20, 0.25), mrange=(1.0, 3.0),
                     n_eta: int = 8) -> Tuple[Template, ...]:
    """k neighbours around ``ref`` on a lattice of (duration offset, eta).

    |duration offset| is log-spaced in [dtau_min, dtau_max] seconds with both
    signs, eta is spaced over ``eta_range``; each node gets a small seeded
    jitter.  Nodes whose component masses leave ``mrange`` are replaced by a
    fresh jittered draw.  The kernel length of each neighbour follows its
    duration offset (Sec. II.B), so this sets the kernel-length mix.
    """
    tau_ref = newtonian_duration(ref, f_low)
    n_off = max(1, k // n_eta)
    mags = np.geomspace(dtau_min, dtau_max, max(1, n_off // 2 + n_off % 2))
    offsets = np.concatenate([mags, -mags])[:n_off]
    out: List[Template] = []
    etas = np.linspace(eta_range[0], eta_range[1], n_eta)
    node = 0
    tries = 0
    while len(out) < k:
        tries += 1
        if tries > 200 * k:
            raise RuntimeError("bank lattice: could not place neighbours in the mass range")
        off = offsets[node % len(offsets)] * np.exp(rng.uniform(-0.15, 0.15))
        eta = float(np.clip(etas[(node // len(offsets)) % n_eta] + rng.uniform(-0.004, 0.004), 0.05, 0.25))
        node += 1
        tau = tau_ref + off
        if tau <= 0:
            continue
        mc = ref.mchirp * (tau_ref / tau) ** 0.6
        m1, m2 = _masses_from_mchirp_eta(mc, eta)
        if m2 < mrange[0]:
            # too unequal for this chirp mass: fall back to the equal-mass node
            m1, m2 = _masses_from_mchirp_eta(mc, 0.25)
        if not (mrange[0] <= m2 <= m1 <= mrange[1]):
            continue
        out.append(Template(m1, m2))
    return tuple(out)


def _cfg1_bank(rng: np.random.Generator, k: int = 16) -> Tuple[Template, Tuple[Template, ...]]:
    ref = Template(2.8, 2.8)
    out = []
    while len(out) < k:
        mc = ref.mchirp * (1.0 + rng.uniform(-0.003, 0.003))
        eta = rng.uniform(0.24, 0.25)
        m1, m2 = _masses_from_mchirp_eta(mc, eta)
        out.append(Template(m1, m2))
    return ref, tuple(out)


def _injections(cfg_index: int, groups, count: int, snr_range, n: int, rng: np.random.Generator,
                margin: int) -> Tuple[Injection, ...]:
    inj = []
    for _ in range(count):
        g = int(rng.integers(0, len(groups)))
        j = int(rng.integers(0, len(groups[g][1])))
        s = int(rng.integers(margin, n - margin))
        inj.append(Injection(j, g, s, float(rng.uniform(*snr_range))))
    return tuple(inj)


def config(i: int, n_override: Optional[int] = None, k_override: Optional[int] = None) -> Config:
    """The five workloads (1-based), optionally shrunk (n, neighbours per group)
    for fast parity cases; the shrunk variants keep the band and bank recipe."""
    rb = np.random.default_rng(seed(i, 1))
    ri = np.random.default_rng(seed(i, 2))
    if i in (1, 3):
        n = n_override or 65536
        fs = 1024.0
        ref, nb = _cfg1_bank(rb, k_override or 16)
        groups = ((ref, nb),)
        cfg = Config(i, "fp64-small" if i == 1 else "precision-form", n, fs, 40.0, fs / 2 - 53.0, 2,
                     "f64", groups=groups, noise_f_min=20.0)
        inj = (Injection(int(ri.integers(0, len(nb))), 0, int(ri.integers(n // 8, n - n // 8)), 12.0),)
        return replace(cfg, injections=inj)
    if i == 2:
        n = n_override or (1 << 20)
        fs = 2048.0
        ref = Template(1.67, 1.67)
        nb = duration_lattice(ref, 20.0, k_override or 256, 0.05, 15.0, rb)
        groups = ((ref, nb),)
        cfg = Config(2, "paper-shaped-fp32", n, fs, 20.0, fs / 2 - 53.0, 7, "f32", groups=groups,
                     noise_f_min=10.0)
        return replace(cfg, injections=_injections(2, groups, 4, (8.0, 20.0), n, ri, n // 64))
    if i == 4:
        n = n_override or (1 << 20)
        fs = 2048.0
        n_ref = 64 if k_override is None else max(2, k_override // 8)
        # references spread log-uniformly in chirp mass over 1-3 M_sun components
        mcs = np.exp(rb.uniform(np.log(Template(1.1, 1.1).mchirp), np.log(Template(2.8, 2.8).mchirp), n_ref))
        groups = []
        for g in range(n_ref):
            m1, m2 = _masses_from_mchirp_eta(mcs[g], rb.uniform(0.235, 0.25))
            if m2 < 1.0:  # keep both components in 1-3 M_sun
                m1, m2 = _masses_from_mchirp_eta(mcs[g], 0.25)
            ref = Template(m1, m2)
            k = int(rb.integers(32, 513)) if k_override is None else max(2, k_override)
            nb = duration_lattice(ref, 20.0, k, 0.02, 30.0, rb, eta_range=(0.18, 0.25))
            groups.append((ref, nb))
        groups = tuple(groups)
        cfg = Config(4, "batched", n, fs, 20.0, fs / 2 - 53.0, 7, "f32", groups=groups, noise_f_min=10.0)
        return replace(cfg, injections=_injections(4, groups, 16, (8.0, 20.0), n, ri, n // 64))
    if i == 5:
        n = n_override or (1 << 23)
        fs = 2048.0
        n_ref = 128 if k_override is None else max(2, k_override // 8)
        groups = []
        for g in range(n_ref):
            m1 = rb.uniform(2.0, 3.0)
            m2 = rb.uniform(2.0, m1)
            ref = Template(m1, m2)
            k = 128 if k_override is None else max(2, k_override)
            nb = duration_lattice(ref, 5.0, k, 0.05, 120.0, rb, eta_range=(0.23, 0.25), mrange=(2.0, 3.0))
            groups.append((ref, nb))
        groups = tuple(groups)
        cfg = Config(5, "long-duration", n, fs, 5.0, fs / 2 - 53.0, 7, "f32", groups=groups,
                     noise_f_min=3.0)
        return replace(cfg, injections=_injections(5, groups, 16, (8.0, 30.0), n, ri, n // 64))
    raise ValueError(f"unknown config {i}")


def synthetic_bank(count: int, mrange=(1.0, 3.0), seed: int = 0) -> Tuple[Template, ...]:
    """A seeded non-spinning bank standing in for the paper's stochastic 1-3 M_sun bank
    (Sec. III.A, about 5.1e4 templates): log-uniform chirp mass over the range the component
    masses allow and uniform eta in [0.2, 0.25], keeping draws whose masses fall in mrange."""
    rng = np.random.default_rng(seed)
    lo, hi = mrange
    mc_lo = (lo * lo) ** 0.6 / (2 * lo) ** 0.2
    mc_hi = (hi * hi) ** 0.6 / (2 * hi) ** 0.2
    out: List[Template] = []
    while len(out) < count:
        mc = float(np.exp(rng.uniform(np.log(mc_lo), np.log(mc_hi))))
        eta = float(rng.uniform(0.2, 0.25))
        m = mc / eta ** 0.6
        d = float(np.sqrt(max(0.0, 1.0 - 4.0 * eta)))
        m1, m2 = 0.5 * m * (1.0 + d), 0.5 * m * (1.0 - d)
        if lo <= m2 and m1 <= hi:
            out.append(Template(m1, m2))
    return tuple(out)


def with_groups(cfg: Config, groups, name: str, seed_index: int = 6) -> Config:
    """``cfg`` with other reference groups (for instance the sets of a structured bank) and
    injections regenerated for them (16 at SNR 8-20, seeded)."""
    ri = np.random.default_rng(seed(seed_index, 2))
    groups = tuple(groups)
    cfg = replace(cfg, name=name, groups=groups)
    # injections go to groups with dependents (a one-template set has none)
    live = [g for g, (_, nb) in enumerate(groups) if len(nb)]
    if not live:
        return replace(cfg, injections=())
    inj = _injections(cfg.index, tuple(groups[g] for g in live), 16, (8.0, 20.0), cfg.n, ri, cfg.n // 64)
    return replace(cfg, injections=tuple(replace(i, group=live[i.group]) for i in inj))
