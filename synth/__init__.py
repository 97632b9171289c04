"""Seeded synthetic inputs shared by the CUDA path's tests/bench and the FP64 oracle.

This module holds data only: system geometries, random scene layouts, sampling
masks and unit-variance noise fields.  It contains none of the imaging method's
arithmetic (no focusing phases, no FFT operators, no thresholding), so that the
oracle and the CUDA path share nothing but their inputs.

Every generator takes a ``numpy.random.Generator`` (``default_rng(seed)``) and
returns NumPy arrays; callers move them to the device themselves.
"""
from __future__ import annotations

import dataclasses

import numpy as np

C_LIGHT = 299792458.0


@dataclasses.dataclass(frozen=True)
class Geometry:
    """Stripmap system parameters (the paper's Table 2 rows: R_c, V, f_0, PRF,
    K_r, T_r, F_r; the antenna length La only sets the simulated aperture)."""

    n_az: int            # N_a: pulses (rows, slow axis)
    n_rg: int            # N_r: range bins (columns, fast axis)
    wavelength: float    # lambda [m]
    velocity: float      # effective radar velocity V [m/s]
    r0: float            # slant range of the scene centre (range bin n_rg/2) [m]
    prf: float           # pulse repetition frequency [Hz]
    bandwidth: float     # chirp bandwidth B [Hz]
    pulse_len: float     # pulse duration T_p [s]
    fs: float            # range sampling rate [Hz]
    antenna_len: float   # La [m]
    c: float = C_LIGHT

    def with_shape(self, n_az: int, n_rg: int) -> "Geometry":
        return dataclasses.replace(self, n_az=int(n_az), n_rg=int(n_rg))


def airborne(n_az: int = 256, n_rg: int = 256) -> Geometry:
    """Airborne X-band geometry of the 256^2 / 2048^2 / batched / autofocus workloads."""
    return Geometry(n_az, n_rg, wavelength=0.03, velocity=150.0, r0=10e3, prf=200.0,
                    bandwidth=60e6, pulse_len=1e-6, fs=72e6, antenna_len=2.0)


def spaceborne(n_az: int = 8192, n_rg: int = 8192) -> Geometry:
    """Spaceborne C-band geometry of the 8192^2 workload."""
    return Geometry(n_az, n_rg, wavelength=0.0556, velocity=7100.0, r0=850e3, prf=1700.0,
                    bandwidth=30e6, pulse_len=40e-6, fs=36e6, antenna_len=10.0)


def paper_table2_simulation(n_az: int = 256, n_rg: int = 256, antenna_len: float = 4.0) -> Geometry:
    """The 'Simulation' column of the paper's Table 2 (Section V): R_c = 20 km,
    V = 350 m/s, f_0 = 5000 MHz, PRF = 175 Hz, K_r = 37.5 MHz/us, T_r = 2 us,
    F_r = 75 MHz, squint 0.  The table gives no antenna length; ``antenna_len``
    only shapes the simulated azimuth aperture."""
    kr = 37.5e6 / 1e-6
    tp = 2e-6
    return Geometry(n_az, n_rg, wavelength=C_LIGHT / 5000e6, velocity=350.0, r0=20e3,
                    prf=175.0, bandwidth=kr * tp, pulse_len=tp, fs=75e6,
                    antenna_len=antenna_len)


def wide_beam_lband(n_az: int = 4096, n_rg: int = 512) -> Geometry:
    """A short-range, wide-beam L-band geometry (lambda 0.24 m, La 1 m, R0 4 km) whose
    range cell migration (~10 bins) and secondary range compression are large
    enough that errors in those terms visibly defocus a point target."""
    return Geometry(n_az, n_rg, wavelength=0.24, velocity=250.0, r0=4000.0, prf=600.0,
                    bandwidth=100e6, pulse_len=2e-6, fs=120e6, antenna_len=1.0)


# ----------------------------------------------------------------------------- scenes

def point_targets(rng: np.random.Generator, n_az: int, n_rg: int, count: int,
                  az_halfwidth: int = 30) -> tuple[np.ndarray, np.ndarray, np.ndarray]:
    """Positions and complex amplitudes of isolated point targets.

    Azimuth bins are drawn from [n_az/2 - az_halfwidth, n_az/2 + az_halfwidth) and
    range bins from [n_rg/4, 3 n_rg/4), distinct pixels; unit amplitude and uniform
    phase.  Returns (rows, cols, amplitudes)."""
    seen: set[tuple[int, int]] = set()
    rows, cols = [], []
    while len(rows) < count:
        r = int(rng.integers(n_az // 2 - az_halfwidth, n_az // 2 + az_halfwidth))
        c = int(rng.integers(n_rg // 4, 3 * n_rg // 4))
        if (r, c) in seen:
            continue
        seen.add((r, c))
        rows.append(r)
        cols.append(c)
    phase = rng.uniform(0.0, 2.0 * np.pi, size=count)
    return np.array(rows), np.array(cols), np.exp(1j * phase)


def sparse_rayleigh(rng: np.random.Generator, n_az: int, n_rg: int, frac: float) -> np.ndarray:
    """Dense complex128 scene with round(frac*n) nonzeros at uniformly chosen pixels
    (without replacement); real and imaginary parts ~ N(0, 1)."""
    n = n_az * n_rg
    k = int(round(frac * n))
    x = np.zeros(n, dtype=np.complex128)
    idx = rng.choice(n, size=k, replace=False)
    x[idx] = rng.standard_normal(k) + 1j * rng.standard_normal(k)
    return x.reshape(n_az, n_rg)


def targets_over_clutter(rng: np.random.Generator, n_az: int, n_rg: int, n_targets: int = 2000,
                         ln_mu: float = 2.0, ln_sigma: float = 0.5,
                         clutter_db: float = -25.0) -> np.ndarray:
    """3x3-pixel bright targets (one complex value per target: lognormal(ln_mu, ln_sigma)
    amplitude, uniform phase) over circular-Gaussian clutter whose power is
    ``clutter_db`` below E[A^2] = exp(2 mu + 2 sigma^2) of the target amplitudes."""
    ea2 = np.exp(2 * ln_mu + 2 * ln_sigma ** 2)
    p_clutter = ea2 * 10.0 ** (clutter_db / 10.0)
    x = cn_noise(rng, (n_az, n_rg)) * np.sqrt(p_clutter)
    r = rng.integers(1, n_az - 1, size=n_targets)
    c = rng.integers(1, n_rg - 1, size=n_targets)
    amp = rng.lognormal(ln_mu, ln_sigma, size=n_targets) * np.exp(
        1j * rng.uniform(0, 2 * np.pi, size=n_targets))
    for dr in (-1, 0, 1):
        for dc in (-1, 0, 1):
            x[r + dr, c + dc] = amp
    return x


def theta_sinusoids(rng: np.random.Generator, n_az: int, count: int = 3,
                    max_cycles: float = 5.0, peak: float = 2 * np.pi) -> np.ndarray:
    """Per-pulse azimuth phase error: a sum of ``count`` sinusoids with frequencies
    uniform in (0, max_cycles] cycles per n_az-pulse record and uniform phases,
    scaled so that max |theta| = peak (radians)."""
    i = np.arange(n_az)
    f = rng.uniform(0.0, max_cycles, size=count)
    f = np.where(f == 0.0, max_cycles, f)
    ph = rng.uniform(0, 2 * np.pi, size=count)
    th = np.sum(np.sin(2 * np.pi * f[:, None] * i[None, :] / n_az + ph[:, None]), axis=0)
    return th * (peak / np.max(np.abs(th)))


# ----------------------------------------------------------------------------- sampling

def bernoulli_mask(rng: np.random.Generator, n_az: int, n_rg: int, rate: float) -> np.ndarray:
    """Boolean sampling mask S with i.i.d. Bernoulli(rate) entries."""
    return rng.random((n_az, n_rg)) < rate


def row_then_range_mask(rng: np.random.Generator, n_az: int, n_rg: int, s_az: float,
                        s_rg: float) -> np.ndarray:
    """The paper's simulation sampling (Section V): random rows (pulses) kept with
    rate s_az, then on every kept pulse random range samples kept with rate s_rg."""
    rows = rng.random(n_az) < s_az
    return (rng.random((n_az, n_rg)) < s_rg) & rows[:, None]


def pack_mask(mask: np.ndarray) -> np.ndarray:
    """Bit-pack a boolean mask, row-major: bit j of 32-bit word w is element 32 w + j.
    The element count must be a multiple of 32."""
    flat = np.ascontiguousarray(mask, dtype=bool).reshape(-1)
    if flat.size % 32:
        raise ValueError("mask size must be a multiple of 32")
    return np.packbits(flat, bitorder="little").view("<u4").copy()


def cn_noise(rng: np.random.Generator, shape) -> np.ndarray:
    """Circular complex Gaussian field with unit variance E|n|^2 = 1."""
    return (rng.standard_normal(shape) + 1j * rng.standard_normal(shape)) * np.sqrt(0.5)


def batch_shapes(rng: np.random.Generator, count: int = 64,
                 sizes=(512, 1024, 2048, 4096)) -> list[tuple[int, int]]:
    """Uneven patch shapes: each axis drawn uniformly from ``sizes``."""
    a = rng.choice(sizes, size=count)
    r = rng.choice(sizes, size=count)
    return [(int(x), int(y)) for x, y in zip(a, r)]


# ----------------------------------------------------------------------------- pulses

BARKER13 = np.array([1, 1, 1, 1, 1, -1, -1, 1, 1, -1, 1, -1, 1], dtype=np.float64)


def coded_pulse(code, chip: float):
    """Baseband phase-coded pulse p(t): chip k (duration ``chip`` seconds) carries
    code[k]; the chips span [-len(code) chip / 2, len(code) chip / 2) around the pulse's
    time origin; zero outside.  Returns a callable of t (seconds, array)."""
    code = np.asarray(code)
    n = len(code)

    def p(t):
        k = np.floor(np.asarray(t) / chip + n / 2.0).astype(np.int64)
        inside = (k >= 0) & (k < n)
        return np.where(inside, code[np.clip(k, 0, n - 1)], 0).astype(np.complex128)
    return p
