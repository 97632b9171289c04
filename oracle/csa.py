"""Chirp-scaling focusing operator M and approximated observation G = M^{-1} (FP64).

TEST INFRASTRUCTURE ONLY (see ``oracle/__init__``).

Section III-C builds the approximated observation from the inverse of a focusing
procedure (Eqs. (14)-(18): frequency-domain matched filters, RCMC and FFTs along
azimuth and range); Section III-D states that the same construction applies to
the Chirp-Scaling Algorithm, whose phase functions the paper takes from its
reference [Cumming2004] (Cumming & Wong, ch. 7) without printing them.  They are
written out here from that textbook with zero squint and the reference Doppler
f_eta_ref = 0 (so D_ref = 1):

  D(f_eta)   = sqrt(1 - (c f_eta / (2 V f0))^2)
  K_m(f_eta) = K_r / (1 - K_r c R_ref f_eta^2 / (2 V^2 f0^3 D^3))
  H1(f_eta, tau)   = exp{ j pi K_m (1/D - 1) (tau - 2 R_ref / (c D))^2 }          chirp scaling
  H2(f_eta, f_tau) = exp{ j pi (D / K_m) f_tau^2 } exp{ j 4 pi f_tau R_ref (1/D - 1) / c }
                                                           range compression + SRC + bulk RCMC
  H3(f_eta, tau)   = exp{ j 4 pi R0(tau) f0 D / c }
                     * exp{ -j 4 pi (K_m / c^2) (1 - D) ((R0(tau) - R_ref) / D)^2 }
                                                    azimuth matched filter + residual phase

  M(Y) = F_a^{-1}[ H3 . F_r^{-1}[ H2 . F_r[ H1 . F_a Y ] ] ]
  G(X) = F_a^{-1}[ H1* . F_r^{-1}[ H2* . F_r[ H3* . F_a X ] ] ]

F is the unnormalised DFT (exp(-j 2 pi k n / N)), F^{-1} carries 1/N.  The grid is
circular with no padding or throwaway, so M is exactly unitary and G = M^{-1} = M^H
(Theorem 1 holds exactly, not approximately, for this operator pair).

Conventions: arrays are row-major [N_a][N_r]; axis 0 = azimuth (pulses, eta),
axis 1 = range (fast time, tau).  The scene-centre range bin is N_r/2 and is at
R_ref = r0; the azimuth time origin is pulse N_a/2.
"""
from __future__ import annotations

import os

import numpy as np
import scipy.fft as sfft

_WORKERS = os.cpu_count() or 1


def _c(g) -> float:
    return float(g.c) if getattr(g, "c", 0.0) else 299792458.0


# ----------------------------------------------------------------------------- grids

def eta_grid(g) -> np.ndarray:
    """Azimuth (slow) time of each pulse: eta_i = (i - N_a/2) / PRF."""
    return (np.arange(g.n_az) - g.n_az // 2) / g.prf


def tau_grid(g) -> np.ndarray:
    """Range (fast) time of each bin: tau_j = 2 R_ref / c + (j - N_r/2) / fs."""
    return 2.0 * g.r0 / _c(g) + (np.arange(g.n_rg) - g.n_rg // 2) / g.fs


def r0_grid(g) -> np.ndarray:
    """Slant range of each range bin, R0(tau) = c tau / 2."""
    return _c(g) * tau_grid(g) / 2.0


def f_eta_grid(g) -> np.ndarray:
    """Doppler frequency of each azimuth FFT bin (signed, unshifted)."""
    return np.fft.fftfreq(g.n_az, d=1.0 / g.prf)


def f_tau_grid(g) -> np.ndarray:
    """Range frequency of each range FFT bin (signed, unshifted)."""
    return np.fft.fftfreq(g.n_rg, d=1.0 / g.fs)


def f0(g) -> float:
    """Carrier frequency f0 = c / lambda."""
    return _c(g) / g.wavelength


def k_r(g) -> float:
    """Range FM rate of the up-chirp, K_r = B / T_p."""
    return g.bandwidth / g.pulse_len


# ----------------------------------------------------------------------------- CSA functions

def migration_factor(g) -> np.ndarray:
    """D(f_eta) = sqrt(1 - (c f_eta / (2 V f0))^2), one value per Doppler bin."""
    fe = f_eta_grid(g)
    return np.sqrt(1.0 - (_c(g) * fe / (2.0 * g.velocity * f0(g))) ** 2)


def modified_fm_rate(g) -> np.ndarray:
    """K_m(f_eta) = K_r / (1 - K_r c R_ref f_eta^2 / (2 V^2 f0^3 D^3))."""
    fe = f_eta_grid(g)
    d = migration_factor(g)
    c = _c(g)
    kr = k_r(g)
    return kr / (1.0 - kr * c * g.r0 * fe ** 2 / (2.0 * g.velocity ** 2 * f0(g) ** 3 * d ** 3))


def h1(g) -> np.ndarray:
    """Chirp-scaling phase H1(f_eta, tau), shape [N_a, N_r]."""
    d = migration_factor(g)[:, None]
    km = modified_fm_rate(g)[:, None]
    tau = tau_grid(g)[None, :]
    arg = np.pi * km * (1.0 / d - 1.0) * (tau - 2.0 * g.r0 / (_c(g) * d)) ** 2
    return np.exp(1j * arg)


def h2(g) -> np.ndarray:
    """Range compression, secondary range compression and bulk RCMC,
    H2(f_eta, f_tau), shape [N_a, N_r]."""
    d = migration_factor(g)[:, None]
    km = modified_fm_rate(g)[:, None]
    ft = f_tau_grid(g)[None, :]
    arg = np.pi * (d / km) * ft ** 2 + 4.0 * np.pi * ft * g.r0 * (1.0 / d - 1.0) / _c(g)
    return np.exp(1j * arg)


def h3(g) -> np.ndarray:
    """Azimuth matched filter and residual phase correction H3(f_eta, tau),
    shape [N_a, N_r]."""
    c = _c(g)
    d = migration_factor(g)[:, None]
    km = modified_fm_rate(g)[:, None]
    r0 = r0_grid(g)[None, :]
    arg = (4.0 * np.pi * r0 * f0(g) * d / c
           - 4.0 * np.pi * (km / c ** 2) * (1.0 - d) * ((r0 - g.r0) / d) ** 2)
    return np.exp(1j * arg)


# ----------------------------------------------------------------------------- operators

def fft_az(a):
    return sfft.fft(a, axis=0, workers=_WORKERS)


def ifft_az(a):
    return sfft.ifft(a, axis=0, workers=_WORKERS)


def fft_rg(a):
    return sfft.fft(a, axis=1, workers=_WORKERS)


def ifft_rg(a):
    return sfft.ifft(a, axis=1, workers=_WORKERS)


def focus_M(g, y: np.ndarray) -> np.ndarray:
    """CSA focusing M(Y): azimuth FFT, chirp scaling H1, range FFT, H2, range IFFT,
    H3, azimuth IFFT (Section III-C/D; Eq. (14) with CSA sub-operations)."""
    y = np.asarray(y, dtype=np.complex128)
    a = fft_az(y)
    a *= h1(g)
    a = fft_rg(a)
    a *= h2(g)
    a = ifft_rg(a)
    a *= h3(g)
    return ifft_az(a)


def observe_G(g, x: np.ndarray) -> np.ndarray:
    """Approximated observation G(X) = M^{-1}(X): every sub-operation of M inverted
    and applied in reverse order, phases conjugated (Section III-C items i-ii,
    Eq. (18))."""
    x = np.asarray(x, dtype=np.complex128)
    a = fft_az(x)
    a *= np.conj(h3(g))
    a = fft_rg(a)
    a *= np.conj(h2(g))
    a = ifft_rg(a)
    a *= np.conj(h1(g))
    return ifft_az(a)
