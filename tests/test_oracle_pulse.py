"""Pins of the oracle's non-chirp pulse (Section III-D, second generalisation: the
approximated observation applies to any transmitted pulse once P_tau^* is replaced by the
recorded pulse; range-Doppler pair).  No GPU."""
import dataclasses
import types

import numpy as np
import pytest

import synth
from oracle import csa, echo, rda

BARKER_PSLR_DB = 20.0 * np.log10(1.0 / 13.0)   # peak 13 chips, sidelobes 1 chip


def with_pulse(g, spectrum):
    """The geometry with a recorded pulse spectrum attached (what the oracle reads)."""
    return types.SimpleNamespace(**dataclasses.asdict(g), pulse=spectrum)


def _rand(rng, shape):
    return rng.standard_normal(shape) + 1j * rng.standard_normal(shape)


def test_pulse_spectrum_of_delayed_impulses():
    """A unit impulse at the pulse's time origin has a flat spectrum; delayed by d
    samples it is exp(-j 2 pi j d / N_r) at bin j (closed form: sign and origin)."""
    g = synth.airborne(16, 64)
    for d in (0, 1, 5, -3):
        p = lambda t, d=d: (np.abs(t * g.fs - d) < 0.5).astype(np.complex128)
        s = rda.pulse_spectrum(g, p)
        j = np.arange(g.n_rg)
        assert np.allclose(s, np.exp(-2j * np.pi * j * d / g.n_rg), atol=1e-12)


def test_chirp_spectrum_reduces_to_the_chirp_filter():
    """With S = exp(-j pi f^2 / K_r), the conjugate of the chirp matched filter, the
    recorded-pulse operators are the chirp ones: G multiplies by S, M by conj(S)."""
    g = synth.airborne(32, 128)
    gp = with_pulse(g, np.exp(-1j * np.pi * csa.f_tau_grid(g) ** 2 / csa.k_r(g)))
    rng = np.random.default_rng(1)
    x = _rand(rng, (32, 128))
    assert np.allclose(rda.observe_G(gp, x), rda.observe_G(g, x), atol=1e-12)
    assert np.allclose(rda.focus_M(gp, x), rda.focus_M(g, x), atol=1e-12)


@pytest.mark.parametrize("geom", ["air", "lband"])
def test_adjoint_identity_with_recorded_pulse(geom):
    """Theorem 1 (G^H = M) holds for any recorded spectrum, unit modulus or not."""
    g = synth.airborne(64, 128) if geom == "air" else synth.wide_beam_lband(128, 64)
    rng = np.random.default_rng(2)
    gp = with_pulse(g, _rand(rng, g.n_rg))
    x = _rand(rng, (g.n_az, g.n_rg))
    y = _rand(rng, (g.n_az, g.n_rg))
    lhs = np.vdot(y, rda.observe_G(gp, x))
    rhs = np.vdot(rda.focus_M(gp, y), x)
    assert abs(lhs - rhs) / abs(lhs) < 1e-12


def test_barker_coded_point_targets_focus():
    """Point targets illuminated by a 13-chip Barker phase code (3 range samples per
    chip), echoes from the exact slant range: the recorded-pulse M focuses each on its
    own pixel; the range cut is the code's autocorrelation (sidelobes 1/13 of the peak,
    -22.28 dB; one sample off the peak 2/3) and the azimuth response keeps its -13.26 dB
    sinc sidelobes."""
    g = synth.airborne(256, 256)
    p = synth.coded_pulse(synth.BARKER13, 3.0 / g.fs)
    gp = with_pulse(g, rda.pulse_spectrum(g, p))
    for r, c in [(128, 128), (140, 90), (110, 170)]:
        x = rda.focus_M(gp, echo.point_echo(g, [r], [c], [1.0], pulse=p))
        pr, pc = np.unravel_index(np.argmax(np.abs(x)), x.shape)
        assert (pr, pc) == (r, c)
        cut = np.abs(x[pr, pc - 60:pc + 61])
        side = np.concatenate([cut[:60 - 2], cut[60 + 3:]]).max()
        assert abs(20 * np.log10(side / cut[60]) - BARKER_PSLR_DB) < 0.2
        assert abs(cut[59] / cut[60] - 2 / 3) < 0.03 and abs(cut[61] / cut[60] - 2 / 3) < 0.03
        from oracle import metrics
        az_pslr, _ = metrics.pslr_irw(x[pr - 32:pr + 32, pc])
        assert abs(az_pslr - (-13.26)) < 0.1


@pytest.mark.parametrize("mode", ["niht", "fixed"])
def test_cs_rda_with_coded_pulse_recovers_targets(mode):
    """Algorithm 1 over the recorded-pulse range-Doppler pair (CS-RDA) on 5 Barker-coded
    point targets (30 dB noise, 50% sampling, K = 5): the support is the true pixels.
    The pulse's spectrum has energy 39 per bin, so ||S G|| > 1: the adaptive (NIHT) step
    takes it as recorded, the fixed step mu = 1 the spectrum scaled to peak magnitude 1
    (which keeps ||S G|| <= 1, Eq. (26))."""
    from oracle import ita
    g = synth.airborne(256, 256)
    p = synth.coded_pulse(synth.BARKER13, 3.0 / g.fs)
    spec = rda.pulse_spectrum(g, p)
    if mode == "fixed":
        spec = spec / np.abs(spec).max()
    gp = with_pulse(g, spec)
    rng = np.random.default_rng(0)
    rows, cols, amps = synth.point_targets(rng, 256, 256, 5)
    s = echo.point_echo(g, rows, cols, amps, pulse=p)
    s = echo.add_noise(synth.cn_noise(rng, s.shape), s, 30.0)
    mask = synth.bernoulli_mask(rng, 256, 256, 0.5)
    x, st = ita.ita(gp, mask * s, mask, 5, 30, ops="rda", mu_mode=mode)
    assert set(zip(*np.nonzero(x))) == set(zip(rows.tolist(), cols.tolist()))
    assert st[-1].resid_sq < st[0].resid_sq
