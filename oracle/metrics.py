"""Error and point-response metrics (FP64).

TEST INFRASTRUCTURE ONLY (see ``oracle/__init__``).

Section V-A measures reconstruction quality by the peak sidelobe ratio (PSLR: the
most prominent sidelobe relative to the main-lobe peak) and the impulse response
width (IRW: main-lobe width 3 dB below the peak), on a cut upsampled by 16 around
the peak.
"""
from __future__ import annotations

import numpy as np


def rel_l2(a: np.ndarray, ref: np.ndarray) -> float:
    """||a - ref||_2 / ||ref||_2."""
    ref = np.asarray(ref)
    den = np.linalg.norm(ref.reshape(-1))
    return float(np.linalg.norm((np.asarray(a) - ref).reshape(-1)) / (den if den else 1.0))


def upsample_cut(cut: np.ndarray, factor: int = 16) -> np.ndarray:
    """Band-limited (FFT zero-padding) upsampling of a 1-D complex cut."""
    n = cut.size
    spec = np.fft.fft(cut)
    pad = np.zeros(n * factor, dtype=np.complex128)
    h = n // 2
    pad[:h] = spec[:h]
    pad[-(n - h):] = spec[h:]
    return np.fft.ifft(pad) * factor


def pslr_irw(cut: np.ndarray, factor: int = 16) -> tuple[float, float]:
    """(PSLR in dB, IRW in ORIGINAL samples) of a 1-D complex cut whose peak is near
    its centre.  IRW counts the upsampled samples at or above -3 dB contiguous with
    the peak and divides by ``factor``; sidelobes are everything outside the first
    nulls (local minima) around the peak."""
    u = np.abs(upsample_cut(np.asarray(cut, dtype=np.complex128), factor))
    p = int(np.argmax(u))
    pk = u[p]
    lo = p
    while lo > 0 and u[lo - 1] < u[lo]:
        lo -= 1
    hi = p
    while hi < u.size - 1 and u[hi + 1] < u[hi]:
        hi += 1
    side = np.concatenate([u[:lo], u[hi + 1:]])
    pslr = 20.0 * np.log10(np.max(side) / pk) if side.size else -np.inf
    half = pk / np.sqrt(2.0)
    a = p
    while a > 0 and u[a - 1] >= half:
        a -= 1
    b = p
    while b < u.size - 1 and u[b + 1] >= half:
        b += 1
    return float(pslr), float((b - a + 1) / factor)
