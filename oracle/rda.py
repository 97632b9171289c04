"""Range-Doppler focusing operator M and approximated observation G = M^H with a
truncated-sinc RCMC (FP64) — the paper's own concrete example (Section III-C).

TEST INFRASTRUCTURE ONLY (see ``oracle/__init__``).

Eq. (14) writes the RDA focusing procedure as range compression (range FFT, range
matched filter P_tau, range IFFT), azimuth FFT, range cell migration correction C,
azimuth matched filter P_eta and azimuth IFFT; Eq. (16) defines C as a truncated-sinc
interpolation along range in the range-Doppler domain, and the approximated
observation (Eq. (18)) applies every sub-operation inverted in reverse order with the
conjugate phases and the interpolation D = C^T (Eq. (22)), so that G = M^H exactly
(Theorem 1).  Written out here:

  M(Y) = F_a^{-1}[ P_eta . C( F_a F_r^{-1}[ P_tau . F_r Y ] ) ]
  G(X) = F_r^{-1}[ P_tau^* . F_r F_a^{-1}[ D( P_eta^* . F_a X ) ] ],   D = C^T

  P_tau(f_tau)      = exp{ j pi f_tau^2 / K_r }                 (up-chirp matched filter)
  P_eta(f_eta, tau) = exp{ j 4 pi R0(tau) f0 D(f_eta) / c }    (exact azimuth matched filter)
  (C V)(f_eta, tau) = sum_t V(f_eta, b + t) sinc(b + t - (tau + dr(f_eta, tau))),
                      b = floor(tau + dr) - 3, t = 0..7 (indices mod N_r)
  dr(f_eta, tau)    = 2 R0(tau) (1/D(f_eta) - 1) fs / c   (migration in range samples)

with D(f_eta) the migration factor of ``csa.migration_factor``, sinc(x) =
sin(pi x)/(pi x), and the grids, FFT conventions and the circular N_a x N_r grid of
``csa``.  The readings (the range filter's sign, the exact instead of the parabolic
azimuth filter, 8 taps, circular indices) are listed in the design notes.
"""
from __future__ import annotations

import numpy as np

from . import csa

N_TAPS = 8          # truncated sinc: taps floor(pos) - 3 .. floor(pos) + 4
TAP_LO = N_TAPS // 2 - 1


def range_filter(g) -> np.ndarray:
    """P_tau(f_tau) = exp(j pi f_tau^2 / K_r), one value per range-frequency bin.  For a
    recorded (non-chirp) transmitted pulse (Section III-D, second generalisation: P_tau^*
    is replaced by the transmitted pulse), ``g.pulse`` holds the pulse's range spectrum S
    (``pulse_spectrum``), G multiplies by S and M by P_tau = conj(S)."""
    s = getattr(g, "pulse", None)
    if s is not None:
        return np.conj(np.asarray(s, dtype=np.complex128))
    ft = csa.f_tau_grid(g)
    return np.exp(1j * np.pi * ft ** 2 / csa.k_r(g))


def pulse_spectrum(g, pulse) -> np.ndarray:
    """Range spectrum S of a baseband pulse p(t) (a callable, t in seconds from the
    pulse's time origin, zero outside its support) on the circular range grid:
    S[j] = sum_n p(t_n) exp(-j 2 pi j n / N_r), t_n = n / fs for the signed sample index
    n (FFT order), so that the compressed peak of an echo p(tau - 2R/c) lies at 2R/c."""
    n = np.fft.fftfreq(g.n_rg, d=1.0 / g.n_rg)
    return np.fft.fft(pulse(n / g.fs))


def azimuth_filter(g) -> np.ndarray:
    """P_eta(f_eta, tau) = exp(j 4 pi R0(tau) f0 D(f_eta) / c), shape [N_a, N_r]."""
    d = csa.migration_factor(g)[:, None]
    r0 = csa.r0_grid(g)[None, :]
    return np.exp(4j * np.pi * r0 * csa.f0(g) * d / csa._c(g))


def migration(g) -> np.ndarray:
    """dr(f_eta, tau) = 2 R0(tau) (1/D(f_eta) - 1) fs / c in range samples, [N_a, N_r]."""
    d = csa.migration_factor(g)[:, None]
    r0 = csa.r0_grid(g)[None, :]
    return 2.0 * r0 * (1.0 / d - 1.0) * g.fs / csa._c(g)


def _taps(dr: np.ndarray):
    """For every output bin tau: the first tap index b = floor(tau + dr) - 3 and the
    weights sinc(b + t - (tau + dr)), t = 0..7."""
    n = dr.shape[1]
    pos = np.arange(n)[None, :] + dr
    base = np.floor(pos).astype(np.int64) - TAP_LO
    w = np.stack([np.sinc(base + t - pos) for t in range(N_TAPS)])
    return base, w


def rcmc_C(v: np.ndarray, dr: np.ndarray) -> np.ndarray:
    """U = C(V): U(f, tau) = sum_t V(f, b + t) w_t (Eq. (16), truncated to 8 taps)."""
    base, w = _taps(dr)
    n = v.shape[1]
    rows = np.arange(v.shape[0])[:, None]
    u = np.zeros_like(v, dtype=np.complex128)
    for t in range(N_TAPS):
        u += v[rows, (base + t) % n] * w[t]
    return u


def rcmc_D(u: np.ndarray, dr: np.ndarray) -> np.ndarray:
    """V = D(U) = C^T U: every U(f, tau) is spread back onto the taps it was read from
    with the same weights (Eq. (17), the transpose of C, Eq. (22))."""
    base, w = _taps(dr)
    n = u.shape[1]
    rows = np.broadcast_to(np.arange(u.shape[0])[:, None], u.shape)
    v = np.zeros_like(u, dtype=np.complex128)
    for t in range(N_TAPS):
        np.add.at(v, (rows, (base + t) % n), u * w[t])
    return v


def focus_M(g, y: np.ndarray) -> np.ndarray:
    """RDA focusing M(Y) (Eq. (14))."""
    a = csa.fft_rg(np.asarray(y, dtype=np.complex128))
    a *= range_filter(g)[None, :]
    a = csa.ifft_rg(a)
    a = csa.fft_az(a)
    a = rcmc_C(a, migration(g))
    a *= azimuth_filter(g)
    return csa.ifft_az(a)


def observe_G(g, x: np.ndarray) -> np.ndarray:
    """RDA approximated observation G(X) = M^H (Eq. (18)): azimuth FFT, P_eta^*, D,
    azimuth IFFT, range FFT, P_tau^*, range IFFT."""
    a = csa.fft_az(np.asarray(x, dtype=np.complex128))
    a *= np.conj(azimuth_filter(g))
    a = rcmc_D(a, migration(g))
    a = csa.ifft_az(a)
    a = csa.fft_rg(a)
    a *= np.conj(range_filter(g))[None, :]
    return csa.ifft_rg(a)
