"""Host check of the indexing argument behind the range-Doppler transpose's scatter
without atomics (no GPU): with the first tap b(tau) of every bin computed as the range
pass computes it (fp32 (hi, lo) coefficients, the double-float fraction, the rounding
of a fraction up to 1 onto the next tap), bins 9 or more apart in one half row start
8-tap spans at least 8 apart, and no two spans of a half row wrap onto each other.
Checked on every Doppler row of the test and benchmark geometries, and on rows at the
largest migration slope a plan accepts (1/2)."""
import numpy as np
import pytest

import synth

C_LIGHT = 299792458.0


def _split(v):
    hi = np.float32(v)
    return hi, np.float32(v - np.float64(hi))


def _first_taps(alpha, a0, nr):
    """b(tau) for tau = 0..nr-1, fp32 arithmetic in the order of the range pass (the
    exact error of the hi product is formed in FP64, where it is exact)."""
    al_hi, al_lo = _split(alpha)
    a0_hi, a0_lo = _split(a0)
    tau = np.arange(nr)
    fj = (tau - nr // 2).astype(np.float32)
    p = (al_hi * fj).astype(np.float32)
    e = (np.float64(al_hi) * fj.astype(np.float64) - p.astype(np.float64)).astype(np.float32)
    n1 = np.rint(a0_hi).astype(np.float32)
    n2 = np.rint(p).astype(np.float32)
    small = (np.float32(a0_lo) + e).astype(np.float32) + (al_lo * fj).astype(np.float32)
    fr = ((a0_hi - n1).astype(np.float32) + (p - n2).astype(np.float32)).astype(np.float32)
    fr = (fr + small.astype(np.float32)).astype(np.float32)
    fl = np.floor(fr)
    fc = (fr - fl).astype(np.float32)
    up = fc >= np.float32(1.0)
    return tau + n1.astype(np.int64) + n2.astype(np.int64) + fl.astype(np.int64) - 3 + up


def _check_row(b, nr):
    half = nr // 2
    for j in range(2):
        h = b[j * half:(j + 1) * half]
        # suffix minimum: the smallest first tap of any bin at least 9 further on
        suf = np.minimum.accumulate(h[::-1])[::-1]
        assert np.all(suf[9:] - h[:-9] >= 8)
        assert h.max() - h.min() <= nr - 8


def _rows(g):
    f0 = C_LIGHT / g.wavelength
    c0 = 2.0 * g.r0 * g.fs / C_LIGHT
    ks = np.arange(g.n_az)
    fe = np.where(ks < g.n_az // 2, ks, ks - g.n_az) * g.prf / g.n_az
    x = C_LIGHT * fe / (2.0 * g.velocity * f0)
    alpha = 1.0 / np.sqrt(1.0 - x * x) - 1.0
    return alpha, alpha * c0


@pytest.mark.parametrize("kind,na,nr", [("air", 256, 1024), ("space", 8192, 8192), ("lband", 4096, 512),
                                       ("table2", 256, 2048), ("lband", 1024, 8192)])
def test_scatter_rounds_are_disjoint(kind, na, nr):
    g = {"air": synth.airborne, "space": synth.spaceborne, "lband": synth.wide_beam_lband,
         "table2": synth.paper_table2_simulation}[kind](na, nr)
    alpha, a0 = _rows(g)
    step = 1 if na <= 1024 else 7    # a spread of rows of the large grids
    for k in range(0, na, step):
        _check_row(_first_taps(alpha[k], a0[k], nr), nr)


@pytest.mark.parametrize("nr", [64, 1024, 8192])
def test_scatter_rounds_at_the_largest_slope(nr):
    rng = np.random.default_rng(nr)
    for a0 in np.concatenate([rng.uniform(0, 5e5, 20), [0.0, 1.0 - 1e-9, 0.5]]):
        _check_row(_first_taps(0.5, a0 * 0.5, nr), nr)
