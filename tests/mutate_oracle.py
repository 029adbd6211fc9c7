"""Mutation check of the oracle's pins (run by hand: python tests/mutate_oracle.py).

The oracle is trusted only because its pins (tests/test_oracle_*.py) fail on a plausible
mistake.  This script plants such mistakes one at a time in a scratch copy of the oracle: a
dropped factor, a wrong sign or index, a transposed operand, an off-by-one, a changed tie rule.
It runs the pins against each one and reports which mistakes no pin catches.  EQUIVALENT lists
the mistakes that change no observable of the method (a constant template phase) and so cannot
fail a pin.  The exit status is non-zero if any other mistake survives.  Takes a few minutes.
"""
import os
import shutil
import subprocess
import sys
import tempfile
import time

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))

# (oracle file, text, planted replacement, what the mistake is)
M = [
 ("mf.py", "return (f >= f_low) & (f <= f_high)", "return (f > f_low) & (f <= f_high)", "band low edge exclusive"),
 ("mf.py", "return (f >= f_low) & (f <= f_high)", "return (f >= f_low) & (f < f_high)", "band high edge exclusive"),
 ("mf.py", "np.sqrt(4.0 * df * np.sum(", "np.sqrt(2.0 * df * np.sum(", "N factor 2 instead of 4"),
 ("mf.py", "* xf * np.conj(h) * inv_psd_band", "* np.conj(xf) * h * inv_psd_band", "conjugate on the data"),
 ("mf.py", "(_fft.fft(x) / fs)", "(_fft.fft(x) * fs)", "data spectrum dt -> fs"),
 ("mf.py", "np.cos(ph) + 1j * np.sin(ph)", "np.cos(ph) - 1j * np.sin(ph)", "snr_at wrong sign"),
 ("mf.py", "spec[: n // 2 + 1] = (4.0 * df / N)", "spec[: n // 2 + 1] = (2.0 * df / N)", "z factor 2 instead of 4"),
 ("mf.py", "return float(np.sqrt(4.0 * df * np.sum(np.abs(h) ** 2 * inv_psd_band)))", "return float(4.0 * df * np.sum(np.abs(h) ** 2 * inv_psd_band))", "N without sqrt"),
 ("taylorf2.py", "return f ** (-7.0 / 6.0)", "return f ** (-7.0 / 3.0)", "amplitude exponent"),
 ("taylorf2.py", "out[pos] = amplitude(f[pos]) * np.exp(-1j * psi)", "out[pos] = amplitude(f[pos]) * np.exp(1j * psi)", "template phase sign"),
 ("taylorf2.py", "return 2.0 * math.pi * f * tc - phic - math.pi / 4.0", "return 2.0 * math.pi * f * tc + phic - math.pi / 4.0", "phic sign"),
 ("taylorf2.py", "return 2.0 * math.pi * f * tc - phic - math.pi / 4.0", "return -2.0 * math.pi * f * tc - phic - math.pi / 4.0", "tc sign"),
 ("taylorf2.py", "MSUN_S = 4.925491025543576e-6", "MSUN_S = 4.93e-6", "solar mass in seconds"),
 ("taylorf2.py", "V_LSO = 1.0 / math.sqrt(6.0)", "V_LSO = 1.0 / 6.0", "v_lso"),
 ("taylorf2.py", "return mt * MSUN_S, m1 * m2 / mt ** 2", "return mt * MSUN_S, m1 * m2 / mt", "eta definition"),
 ("taylorf2.py", "a[3] = -16.0 * pi", "a[3] = 16.0 * pi", "alpha3 sign"),
 ("ratio.py", "K[sup] = norm * R * w[sup] * np.exp(1j * dpsi)", "K[sup] = norm * R * w[sup] * np.exp(-1j * dpsi)", "ratio phase conjugated"),
 ("ratio.py", "return _fft.ifft_unnormalised(spec) / n", "return _fft.ifft_unnormalised(spec) / (n // 2)", "kernel 1/n factor"),
 ("ratio.py", "w[lo] = 0.5 * (1.0 + np.cos(np.pi * (f[lo] - f_low) / df_low))", "w[lo] = 0.5 * (1.0 - np.cos(np.pi * (f[lo] - f_low) / df_low))", "low taper flipped"),
 ("ratio.py", "w[hi] = 0.5 * (1.0 - np.cos(np.pi * (f[hi] - (f_high + df_high)) / df_high))", "w[hi] = 0.5 * (1.0 - np.cos(np.pi * (f[hi] - f_high) / df_high))", "high taper origin"),
 ("ratio.py", "hi = (f > f_high) & (f < f_high + df_high)", "hi = (f > f_high) & (f < f_high + 0.5 * df_high)", "high taper width"),
 ("ratio.py", "cut2 = thr * thr * (amax2 if relative else 1.0)", "cut2 = thr * (amax2 if relative else 1.0)", "threshold on |rho|^2"),
 ("ratio.py", "m0 = min(cands, key=lambda m: signed_lag(m, n))", "m0 = max(cands, key=lambda m: signed_lag(m, n))", "arc tie rule"),
 ("ratio.py", "return m0, int(n - gmax)", "return m0, int(n - gmax + 1)", "arc length off by one"),
 ("ratio.py", "taps = rho[(m0 + np.arange(L)) % n]", "taps = rho[(m0 - np.arange(L)) % n]", "taps read backwards"),
 ("ratio.py", "dtp = abs(d2) / (2.0 * math.pi)", "dtp = abs(d2)", "df_low rule missing 2 pi"),
 ("ratio.py", "return min(df_low_max, 0.5 * f_low, rule)", "return min(df_low_max, rule)", "df_low without f_low/2 guard"),
 ("ratio.py", "rho = (2.0 * rho.real).astype(np.complex128)", "rho = (rho.real).astype(np.complex128)", "real form without factor 2"),
 ("ratio.py", "amp = thr * (1.0 if real else 2.0) * fs * peak", "amp = thr * fs * peak", "analytic relative amplitude factor"),
 ("ratio.py", "while nb < 4.0 * extent and nb < n:", "while nb < 1.0 * extent and nb < n:", "build grid too small"),
 ("reconstruct.py", "out += c * np.roll(z_ref, m0 + l)", "out += c * np.roll(z_ref, m0 - l)", "direct sum index sign"),
 ("reconstruct.py", "out[q] = np.sum(taps * z_ref[(i - m0 - l) % n])", "out[q] = np.sum(taps * z_ref[(i + m0 + l) % n])", "reconstruct_at index"),
 ("reconstruct.py", "a = int(np.argmax(seg))", "a = int(len(seg) - 1 - np.argmax(seg[::-1]))", "argmax last of equals"),
 ("reconstruct.py", "nw = (n + W - 1) // W", "nw = n // W", "ragged last window dropped"),
 ("data.py", "a = inj.snr / sigma(h, ipb, fs / n)", "a = inj.snr * sigma(h, ipb, fs / n)", "injection scale inverted"),
 ("data.py", "full[n // 2 + 1:] = np.conj(xf[1: n // 2][::-1])", "full[n // 2 + 1:] = xf[1: n // 2][::-1]", "negative half not conjugated"),
 ("data.py", "return (_fft.ifft_unnormalised(full).real * fs / n)", "return (_fft.ifft_unnormalised(full).real / n)", "strain missing fs"),
 ("bounds.py", "d_e = np.cbrt(R_e / (4.0 * math.pi * dfe * dfe * amp))", "d_e = np.cbrt(R_e / (2.0 * math.pi * dfe * dfe * amp))", "analytic span 2 pi"),
 ("bounds.py", "return dt_s / (4.0 * math.pi * df_low ** 2 * np.abs(d0 + np.asarray(lags_s)) ** 3)", "return dt_s / (4.0 * math.pi * df_low ** 2 * np.abs(d0 + np.asarray(lags_s)) ** 2)", "low tail power"),
 ("bank.py", "h = len(idx) // 2", "h = (len(idx) + 1) // 2", "bisection puts the extra in the first half"),
 ("bank.py", "if best < 0 or s < best_sum - 1e-9 * best_sum:", "if best < 0 or s > best_sum + 1e-9 * best_sum:", "reference maximises"),
 ("bank.py", "elif abs(s - best_sum) <= 1e-9 * best_sum and i < best:", "elif abs(s - best_sum) <= 1e-9 * best_sum and i > best:", "reference tie to highest index"),
 ("bank.py", "order = sorted(range(n), key=lambda i: (mc[i], i))", "order = sorted(range(n), key=lambda i: (eta[i], i))", "first bisection by eta"),
 ("fft.py", "rev |= ((idx >> b) & 1) << (bits - 1 - b)", "rev |= ((idx >> b) & 1) << b", "no bit reversal"),
 ("fft.py", "w = np.exp(sign * 2j * np.pi * m / size)", "w = np.exp(sign * 2j * np.pi * m / n)", "twiddles of the whole length"),
 ("fft.py", "a[..., half:] = top - bot", "a[..., half:] = bot - top", "butterfly difference reversed"),
 ("fft.py", "return _transform(x, -1.0)", "return _transform(x, +1.0)", "forward transform sign"),
 ("taylorf2.py", "return (math.pi * M / (128.0 * eta)) * (g2 / v ** 2 - 2.0 * g1 / v ** 3) * dv_df",
  "return (math.pi * M / (128.0 * eta)) * (g2 / v ** 2 - g1 / v ** 3) * dv_df", "Psi'' product rule"),
 ("taylorf2.py", "g1 += a6log * (np.log(4.0 * v) + 1.0)", "g1 += a6log * np.log(4.0 * v)", "log-term derivative"),
 ("ratio.py", "return m if m <= n // 2 else m - n", "return m if m < n // 2 else m - n", "signed lag at n/2"),
 ("bounds.py", "out[ok] = dt_s / np.sqrt(np.abs(delta_t_prime(fstar[ok], ref, tgt, pn_order)))",
  "out[ok] = 2.0 * dt_s / np.sqrt(np.abs(delta_t_prime(fstar[ok], ref, tgt, pn_order)))", "stationary envelope factor"),
 ("bounds.py", "fe = np.array([f_low - df_low, f_low, f_high, f_high + df_high])",
  "fe = np.array([f_low, f_low, f_high, f_high])", "span from the band edges only"),
 ("bounds.py", "return dt_s / (4.0 * math.pi * df_high ** 2 * np.abs(np.asarray(lags_s) + d1) ** 3)",
  "return dt_s / (4.0 * math.pi * df_high ** 2 * np.abs(np.asarray(lags_s) - d1) ** 3)", "high tail centre sign"),
 ("bounds.py", "m_hi = math.ceil(hi * fs)", "m_hi = math.floor(hi * fs)", "span end rounded inwards"),
 ("bank.py", "return (m1 * m2) ** 0.6 / (m1 + m2) ** 0.2", "return (m1 * m2) ** 0.6 / (m1 + m2) ** 0.4", "chirp mass exponent"),
 ("bank.py", "return m1 * m2 / ((m1 + m2) * (m1 + m2))", "return m1 * m2 / (m1 + m2)", "eta in the second bisection"),
 ("reconstruct.py", "mag2 = (z.real.astype(np.float64) ** 2 + z.imag.astype(np.float64) ** 2)",
  "mag2 = np.abs(z.real.astype(np.float64)) + np.abs(z.imag.astype(np.float64))", "peak of |Re| + |Im|"),
 ("data.py", "h = template(n, fs, t.m1, t.m2, cfg.pn_order, tc=inj.sample / fs)",
  "h = template(n, fs, t.m1, t.m2, cfg.pn_order, tc=(inj.sample + 1) / fs)", "injection one sample late"),
 ("bank.py", "lambda s: float(tau[s].max() - tau[s].min()) <= max_spread", "lambda s: float(tau[s].max() - tau[s].min()) < max_spread", "spread limit strict"),
 ("bank.py", "lambda x: len(x) <= max_size", "lambda x: len(x) < max_size", "size limit strict"),
 ("bank.py", "key=lambda i: (mc[i], i)", "key=lambda i: (mc[i], -i)", "chirp-mass ties in reverse bank order"),
 ("ratio.py", "amp = thr * (1.0 if real else 2.0) * fs * peak", "amp = thr * 2.0 * fs * peak", "real-form analytic amplitude factor"),
 ("ratio.py", "extent = float(np.abs(d).max()) * fs + 4.0 * fs / df_low", "extent = float(np.abs(d).max()) * fs", "build grid without the taper spread"),
 ("taylorf2.py", "g2 += ak * p * (p - 1) * v ** (p - 2)", "g2 += ak * p * p * v ** (p - 2)", "second derivative of a power"),
 ("ratio.py", "cut2 = thr * thr * (amax2 if relative else 1.0)", "cut2 = thr * thr * (1.0 if relative else amax2)", "relative and absolute swapped"),
]

# constant phase offsets of every template: |z|, t(f) and the ratio identity are unchanged
EQUIVALENT = {"v_lso"}


def main() -> int:
    scratch = tempfile.mkdtemp(prefix="oracle_mutants_")
    try:
        for d in ("oracle", "workload", "tests"):
            shutil.copytree(os.path.join(ROOT, d), os.path.join(scratch, d),
                            ignore=shutil.ignore_patterns("__pycache__"))
        tests = sorted(os.path.join("tests", f) for f in os.listdir(os.path.join(scratch, "tests"))
                       if f.startswith("test_oracle_"))
        env = dict(os.environ, PYTHONDONTWRITEBYTECODE="1")
        bad = []
        for fname, old, new, name in M:
            path = os.path.join(scratch, "oracle", fname)
            src = open(path).read()
            if old not in src:
                print(f"{'absent':9s} {fname:15s} {name}")
                bad.append(name)
                continue
            open(path, "w").write(src.replace(old, new, 1))
            t0 = time.time()
            r = subprocess.run([sys.executable, "-m", "pytest", "-x", "-q", "-p", "no:cacheprovider", *tests],
                               cwd=scratch, capture_output=True, text=True, timeout=900, env=env)
            open(path, "w").write(src)
            caught = r.returncode != 0
            by = next((ln.split(" - ")[0] for ln in r.stdout.splitlines() if ln.startswith(("FAILED", "ERROR"))), "")
            status = "caught" if caught else ("equivalent" if name in EQUIVALENT else "SURVIVED")
            if not caught and name not in EQUIVALENT:
                bad.append(name)
            print(f"{status:10s} {fname:15s} {name:44s} {time.time() - t0:5.1f}s {by}", flush=True)
        print(f"{len(M)} planted mistakes, {len(bad)} not caught by a pin (besides {len(EQUIVALENT)} equivalent)")
        return 1 if bad else 0
    finally:
        shutil.rmtree(scratch, ignore_errors=True)


if __name__ == "__main__":
    sys.exit(main())
