"""Exact point-target echo simulator (FP64, time domain).

TEST INFRASTRUCTURE ONLY (see ``oracle/__init__``).

Section II-A models the stripmap echo as the scene convolved with an azimuth
modulation and the transmitted pulse (Eqs. (1)-(2)); Section V generates raw data
"in time-domain by exact slant range".  For a point target at (eta_t, R_t) with
complex amplitude a, each echo sample is

  s(eta, tau) += a rect((tau - 2R/c)/T_p) rect((eta - eta_t)/T_a)
                 exp(-j 4 pi f0 R / c) exp(j pi K_r (tau - 2R/c)^2),
  R = sqrt(R_t^2 + V^2 (eta - eta_t)^2),   T_a = 0.886 lambda R_t / (La V),

i.e. an up-chirp of rate K_r = B/T_p delayed by the exact two-way range, within the
synthetic-aperture time of a uniformly illuminated antenna of length La.  This uses
no chirp-scaling formula and no FFT, so it pins the operator's phase conventions
independently.
"""
from __future__ import annotations

import numpy as np

from . import csa


def point_echo(g, rows, cols, amps, pulse=None) -> np.ndarray:
    """Raw echo [N_a, N_r] of point targets placed on image pixels (row, col):
    eta_t = eta_grid[row], R_t = R0(tau_grid[col]).  ``pulse``: a baseband transmitted
    pulse p(t) (callable, t from the pulse's time origin, zero outside its support) in
    place of the up-chirp rect(t/T_p) exp(j pi K_r t^2) (Section III-D, non-chirp
    pulses)."""
    c = csa._c(g)
    eta = csa.eta_grid(g)[:, None]
    tau = csa.tau_grid(g)[None, :]
    fc = csa.f0(g)
    kr = csa.k_r(g)
    out = np.zeros((g.n_az, g.n_rg), dtype=np.complex128)
    for row, col, a in zip(np.atleast_1d(rows), np.atleast_1d(cols), np.atleast_1d(amps)):
        eta_t = csa.eta_grid(g)[row]
        r_t = csa.r0_grid(g)[col]
        t_a = 0.886 * g.wavelength * r_t / (g.antenna_len * g.velocity)
        r = np.sqrt(r_t ** 2 + (g.velocity * (eta - eta_t)) ** 2)
        delay = tau - 2.0 * r / c
        in_beam = np.abs(eta - eta_t) <= t_a / 2
        if pulse is None:
            env = (np.abs(delay) <= g.pulse_len / 2) & in_beam
            ph = -4.0 * np.pi * fc * r / c + np.pi * kr * delay ** 2
            out += np.where(env, a * np.exp(1j * ph), 0.0)
        else:
            out += np.where(in_beam, a * np.exp(-4j * np.pi * fc * r / c) * pulse(delay), 0.0)
    return out


def add_noise(rng_noise: np.ndarray, s: np.ndarray, snr_db: float) -> np.ndarray:
    """s + n with n = unit-variance circular Gaussian field ``rng_noise`` scaled so
    that mean|s|^2 over the full grid / sigma_n^2 = 10^(snr_db/10)."""
    p = float(np.mean(np.abs(s) ** 2))
    sigma_n = np.sqrt(p / 10.0 ** (snr_db / 10.0))
    return s + sigma_n * rng_noise
