"""Plain FP64 CPU oracle for the ratio-filter hot path.

TEST INFRASTRUCTURE ONLY.  This package is what the CUDA library is checked
against; only the tests, the smoke check and the CPU-baseline leg of the
benchmark may import it.  It shares no code with the CUDA path: its FFT is its
own radix-2 transform, every template phase, normalisation, window, ratio
kernel, truncation, convolution and window maximum is written out here from
the paper's definitions, in float64 / complex128, with no blocking, fusion or
reordering beyond what the definitions state.

Modules (paper passages they follow):

* ``fft``         -- discrete Fourier transform by the textbook radix-2
                     Cooley-Tukey recursion; sign convention of Eq. (1).
* ``taylorf2``    -- stationary-phase template h(f) = B(f) exp(-i Psi(f))
                     (App. A, Eq. A1), Psi' = 2 pi t(f) (Eq. A2).
* ``mf``          -- data spectrum, normalisation N (Eq. 3) and complex SNR
                     z(t) (Eqs. 2, 4, 6).
* ``ratio``       -- window W(f) (Eq. 9), Delta f_low rule (Eq. 10), ratio
                     kernel (Eqs. 5, 7) and its threshold truncation (Sec. II.D).
* ``reconstruct`` -- target SNR by direct circular convolution (Eq. 8) and the
                     per-window peak (Sec. IV).
* ``data``        -- strain with injections (Sec. III.B) from the seeded draws
                     of the ``workload`` module.
* ``bounds``      -- App. A envelope and tail bounds (Eqs. A9-A11) and the
                     analytic kernel spans they give.
* ``bank``        -- structuring of a bank into reference sets: chirp-mass and
                     symmetric-mass-ratio bisection, duration-medoid reference
                     (Sec. III.A).

Every function states which passage it follows.  Parity of the paper's printed
example SNRs (Sec. IV, 5.769 and 8.903) is unpinned: the noise realisation and
PSD file behind them are not published.
"""
from . import fft, taylorf2, mf, ratio, reconstruct, data, bounds, bank  # noqa: F401
