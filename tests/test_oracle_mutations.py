"""Planted-mistake check of the oracle's pins: each plausible slip in the oracle's
arithmetic (a flipped sign, a dropped term, a transposed axis, an un-conjugated
phase, an off-by-one rank) is planted in the oracle on the CPU, and at least one pin
must fail.  Nothing here touches the CUDA path."""
import numpy as np
import pytest

import synth
import test_oracle_ita as ita_pins
import test_oracle_operators as op_pins
from oracle import csa, echo, ita

C = 299792458.0

OP_PINS = [
    lambda: op_pins.test_dense_kronecker_form((16, 16)),
    lambda: op_pins.test_unitarity_and_adjoint("air"),
    op_pins.test_point_targets_focus_airborne,
    op_pins.test_point_target_matches_paper_table2_simulation,
    op_pins.test_residual_phase_sign_far_range,
    op_pins.test_src_and_bulk_rcmc_wide_beam,
]


def _h2_terms(g, mf_sign=1.0, bulk_sign=1.0):
    d = csa.migration_factor(g)[:, None]
    km = csa.modified_fm_rate(g)[:, None]
    ft = csa.f_tau_grid(g)[None, :]
    return np.exp(1j * (mf_sign * np.pi * (d / km) * ft ** 2
                        + bulk_sign * 4 * np.pi * ft * g.r0 * (1 / d - 1) / C))


def _h3_terms(g, az_sign=1.0, res_sign=-1.0):
    d = csa.migration_factor(g)[:, None]
    km = csa.modified_fm_rate(g)[:, None]
    r0 = csa.r0_grid(g)[None, :]
    return np.exp(1j * (az_sign * 4 * np.pi * r0 * csa.f0(g) * d / C
                        + res_sign * 4 * np.pi * (km / C ** 2) * (1 - d) * ((r0 - g.r0) / d) ** 2))


_H1, _H2, _H3, _D = csa.h1, csa.h2, csa.h3, csa.migration_factor


def _km_flipped(g):
    fe = csa.f_eta_grid(g)
    d = _D(g)
    kr = csa.k_r(g)
    return kr / (1 + kr * C * g.r0 * fe ** 2 / (2 * g.velocity ** 2 * csa.f0(g) ** 3 * d ** 3))


def _g_same_order(g, x):
    a = csa.fft_az(np.asarray(x, complex)) * np.conj(_H1(g))
    a = csa.ifft_rg(csa.fft_rg(a) * np.conj(_H2(g))) * np.conj(_H3(g))
    return csa.ifft_az(a)


def _g_h2_unconjugated(g, x):
    a = csa.fft_az(np.asarray(x, complex)) * np.conj(_H3(g))
    a = csa.ifft_rg(csa.fft_rg(a) * _H2(g)) * np.conj(_H1(g))
    return csa.ifft_az(a)


def _m_axes_swapped(g, y):
    a = csa.fft_rg(np.asarray(y, complex)) * _H1(g)
    a = csa.ifft_az(csa.fft_az(a) * _H2(g)) * _H3(g)
    return csa.ifft_rg(a)


OP_MUTATIONS = {
    "range matched filter sign": ("h2", lambda g: _h2_terms(g, mf_sign=-1.0)),
    "bulk RCMC sign": ("h2", lambda g: _h2_terms(g, bulk_sign=-1.0)),
    "bulk RCMC dropped": ("h2", lambda g: _h2_terms(g, bulk_sign=0.0)),
    "chirp scaling dropped": ("h1", lambda g: np.ones((g.n_az, g.n_rg), complex)),
    "chirp scaling sign": ("h1", lambda g: np.conj(_H1(g))),
    "azimuth matched filter sign": ("h3", lambda g: _h3_terms(g, az_sign=-1.0)),
    "residual phase sign": ("h3", lambda g: _h3_terms(g, res_sign=1.0)),
    "residual phase dropped": ("h3", lambda g: _h3_terms(g, res_sign=0.0)),
    "migration factor without square": (
        "migration_factor",
        lambda g: np.sqrt(1 - np.abs(C * csa.f_eta_grid(g) / (2 * g.velocity * csa.f0(g))))),
    "SRC term sign": ("modified_fm_rate", _km_flipped),
    "K_m replaced by K_r": ("modified_fm_rate", lambda g: np.full(g.n_az, csa.k_r(g))),
    "G phases not reversed": ("observe_G", _g_same_order),
    "G range phase not conjugated": ("observe_G", _g_h2_unconjugated),
    "M axes transposed": ("focus_M", _m_axes_swapped),
}


def _some_pin_fails(pins):
    for pin in pins:
        try:
            pin()
        except (AssertionError, ValueError, IndexError):
            return True
    return False


@pytest.mark.parametrize("name", sorted(OP_MUTATIONS))
def test_operator_mutation_is_caught(name, monkeypatch):
    attr, fn = OP_MUTATIONS[name]
    monkeypatch.setattr(csa, attr, fn)
    assert _some_pin_fails(OP_PINS), name


ITA_PINS = [
    ita_pins.test_soft_threshold_is_prox_by_brute_force,
    ita_pins.test_half_threshold_is_global_minimiser_by_brute_force,
    ita_pins.test_hard_threshold_is_l0_prox_by_brute_force,
    lambda: ita_pins.test_kth_largest_against_counting(7),
    lambda: ita_pins.test_full_sampling_closed_form("soft"),
    ita_pins.test_first_iterate_is_threshold_of_masked_mf,
    ita_pins.test_niht_step_properties,
    lambda: ita_pins.test_top_k_support_against_sorting_and_counting(5),
]

_soft, _half, _kth, _niht = ita.soft_threshold, ita.half_threshold, ita.kth_largest_magnitude, ita.niht_step
_hard = ita.hard_threshold
_top_k = ita.top_k_support


def _ita_iteration_unmasked(g, y, mask, x, k, mu_mode="fixed", mu=1.0, kind="soft", ops="csa"):
    r = y - csa.observe_G(g, x)
    b = x + mu * csa.focus_M(g, r)
    s = _kth(b, k)
    return ita.threshold(b, s, kind), ita.IterStats(0.0, mu, s, 0)


ITA_MUTATIONS = {
    "soft threshold halves sigma": ("soft_threshold", lambda b, s: _soft(b, s / 2)),
    "soft threshold drops phase": ("soft_threshold",
                                   lambda b, s: np.where(np.abs(b) > s, np.abs(b) - s, 0).astype(complex)),
    "half threshold wrong angle": ("half_lambda_mu", lambda s: np.sqrt(96.0) / 9.0 * s),
    "hard threshold keeps |b| >= sigma / 2": ("hard_threshold", lambda b, s: _hard(b, s / 2)),
    "K-th instead of (K+1)-th": ("kth_largest_magnitude", lambda b, k: _kth(b, max(k - 1, 0))),
    "NIHT ratio inverted": ("niht_step", lambda g, m, dx, sup, ops="csa": 1.0 / _niht(g, m, dx, sup, ops)),
    "mask dropped from residue": ("ita_iteration", _ita_iteration_unmasked),
    "top-K support picks the smallest": (
        "top_k_support", lambda v, k: _top_k(-1.0 / (np.abs(v) + 1e-300), k)),
    "top-K support keeps one too many": ("top_k_support", lambda v, k: _top_k(v, k + 1)),
}


@pytest.mark.parametrize("name", sorted(ITA_MUTATIONS))
def test_ita_mutation_is_caught(name, monkeypatch):
    attr, fn = ITA_MUTATIONS[name]
    monkeypatch.setattr(ita, attr, fn)
    assert _some_pin_fails(ITA_PINS), name


ECHO_PINS = [ita_pins.test_add_noise_sets_requested_snr]
_add_noise = echo.add_noise


def _noise_power_as_amplitude(rng_noise, s, snr_db):
    p = float(np.mean(np.abs(s) ** 2))
    return s + (p / 10.0 ** (snr_db / 10.0)) * rng_noise


def _noise_db_as_amplitude_ratio(rng_noise, s, snr_db):
    p = float(np.mean(np.abs(s) ** 2))
    return s + np.sqrt(p) / 10.0 ** (snr_db / 10.0) * rng_noise


ECHO_MUTATIONS = {
    "noise sigma from the power, not its square root": ("add_noise", _noise_power_as_amplitude),
    "noise SNR in dB taken as an amplitude ratio": ("add_noise", _noise_db_as_amplitude_ratio),
    "noise power from the peak, not the mean": (
        "add_noise", lambda n, s, snr: _add_noise(n * np.sqrt(np.max(np.abs(s) ** 2) /
                                                              np.mean(np.abs(s) ** 2)), s, snr)),
}


@pytest.mark.parametrize("name", sorted(ECHO_MUTATIONS))
def test_echo_mutation_is_caught(name, monkeypatch):
    attr, fn = ECHO_MUTATIONS[name]
    monkeypatch.setattr(echo, attr, fn)
    assert _some_pin_fails(ECHO_PINS), name


import test_oracle_pulse as pulse_pins  # noqa: E402
from oracle import rda  # noqa: E402

PULSE_PINS = [pulse_pins.test_pulse_spectrum_of_delayed_impulses,
              pulse_pins.test_chirp_spectrum_reduces_to_the_chirp_filter,
              pulse_pins.test_barker_coded_point_targets_focus]
_range_filter, _pulse_spectrum = rda.range_filter, rda.pulse_spectrum


def _rf_unconjugated(g):
    s = getattr(g, "pulse", None)
    return np.asarray(s, complex) if s is not None else _range_filter(g)


PULSE_MUTATIONS = {
    "recorded pulse not conjugated in M": ("range_filter", _rf_unconjugated),
    "pulse spectrum time-reversed": ("pulse_spectrum", lambda g, p: _pulse_spectrum(g, lambda t: p(-t))),
    "pulse spectrum by inverse DFT": (
        "pulse_spectrum", lambda g, p: g.n_rg * np.fft.ifft(p(np.fft.fftfreq(g.n_rg, 1.0 / g.n_rg) / g.fs))),
}


@pytest.mark.parametrize("name", sorted(PULSE_MUTATIONS))
def test_pulse_mutation_is_caught(name, monkeypatch):
    attr, fn = PULSE_MUTATIONS[name]
    monkeypatch.setattr(rda, attr, fn)
    assert _some_pin_fails(PULSE_PINS), name
