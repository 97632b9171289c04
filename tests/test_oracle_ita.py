"""Pins of the FP64 oracle's thresholds, K-th magnitude rule and ITA (no GPU)."""
import numpy as np
import pytest

import synth
from oracle import csa, echo, ita, metrics


def _rand(rng, shape):
    return rng.standard_normal(shape) + 1j * rng.standard_normal(shape)


# ----------------------------------------------------------------------------- thresholds

def test_soft_threshold_is_prox_by_brute_force():
    """soft(b, s) minimises |x - b|^2 + 2 s |x| over a fine complex grid."""
    rng = np.random.default_rng(4)
    g = np.linspace(-3, 3, 1201)
    xr, xi = np.meshgrid(g, g, indexing="ij")
    xc = xr + 1j * xi
    for _ in range(6):
        b = complex(rng.uniform(-2.5, 2.5), rng.uniform(-2.5, 2.5))
        s = rng.uniform(0.1, 1.5)
        obj = np.abs(xc - b) ** 2 + 2 * s * np.abs(xc)
        best = xc.reshape(-1)[np.argmin(obj)]
        assert abs(ita.soft_threshold(np.array([b]), s)[0] - best) < 1e-2


def test_half_threshold_is_global_minimiser_by_brute_force():
    """half(b, s) is the global minimiser of (x - z)^2 + lam |x|^(1/2), lam from s;
    jump point at |b| = s; complex inputs keep their phase."""
    xs = np.linspace(-6, 6, 240001)
    for s in (0.3, 1.0, 2.0):
        lam = ita.half_lambda_mu(s)
        for z in np.linspace(-5, 5, 41):
            obj = (xs - z) ** 2 + lam * np.sqrt(np.abs(xs))
            best = xs[np.argmin(obj)]
            got = ita.half_threshold(np.array([z + 0j]), s)[0]
            assert abs(got.real - best) < 2e-4 and got.imag == 0
        below = ita.half_threshold(np.array([s * (1 - 1e-9)]), s)[0]
        above = ita.half_threshold(np.array([s * (1 + 1e-9)]), s)[0]
        assert below == 0 and abs(above - 2 * s / 3) < 1e-6
    b = np.array([1.7 * np.exp(0.9j)])
    assert abs(np.angle(ita.half_threshold(b, 1.0)[0]) - 0.9) < 1e-12
    # worked value: z = 1, lam = 1 -> x* = 0.70152 (the jump point for lam = 1 is 0.94494)
    s1 = (54 ** (1 / 3) / 4)
    assert abs(ita.half_lambda_mu(s1) - 1.0) < 1e-12
    assert abs(ita.half_threshold(np.array([1.0 + 0j]), s1)[0].real - 0.70152) < 1e-5


def test_hard_threshold_is_l0_prox_by_brute_force():
    """hard(b, s) minimises |x - b|^2 + s^2 [x != 0] over a fine complex grid that
    contains b itself (the minimiser is b or 0)."""
    rng = np.random.default_rng(5)
    g = np.linspace(-3, 3, 601)
    xr, xi = np.meshgrid(g, g, indexing="ij")
    for _ in range(8):
        b = complex(rng.uniform(-2.5, 2.5), rng.uniform(-2.5, 2.5))
        s = rng.uniform(0.1, 3.0)
        xc = np.append((xr + 1j * xi).reshape(-1), b)
        obj = np.abs(xc - b) ** 2 + s ** 2 * (xc != 0)
        best = xc[np.argmin(obj)]
        assert abs(ita.hard_threshold(np.array([b]), s)[0] - best) < 1e-12


def test_half_threshold_zero_sigma_is_identity():
    rng = np.random.default_rng(5)
    b = _rand(rng, 50)
    assert np.allclose(ita.half_threshold(b, 0.0), b, atol=1e-12)
    assert np.allclose(ita.soft_threshold(b, 0.0), b, atol=0)


@pytest.mark.parametrize("k", [0, 1, 7, 99, 100, 150])
def test_kth_largest_against_counting(k):
    rng = np.random.default_rng(6)
    b = _rand(rng, 100)
    s = ita.kth_largest_magnitude(b, k)
    mag = np.abs(b)
    if k >= b.size:
        assert s == 0.0
    else:
        assert np.sum(mag > s) <= k and np.sum(mag >= s) >= k + 1
        assert np.count_nonzero(ita.soft_threshold(b, s)) <= k


@pytest.mark.parametrize("k", [0, 1, 5, 37, 64, 100])
def test_top_k_support_against_sorting_and_counting(k):
    """top_k_support picks exactly min(k, n) entries: those first in the order of
    decreasing magnitude with ties broken by the lower flat index (brute force over
    the sorted index list), and each picked entry has fewer than k strictly larger
    magnitudes (counting).  Exact ties are planted (|conj z| = |-z| = |z| exactly)."""
    rng = np.random.default_rng(13)
    v = _rand(rng, (8, 8))
    v.flat[10] = np.conj(v.flat[20])
    v.flat[30] = -v.flat[20]
    v.flat[40] = v.flat[41]
    sel = ita.top_k_support(v, k)
    assert sel.shape == v.shape and sel.dtype == bool
    assert int(sel.sum()) == min(k, v.size)
    mag = np.abs(v).reshape(-1)
    order = sorted(range(v.size), key=lambda i: (-mag[i], i))
    assert set(np.flatnonzero(sel).tolist()) == set(order[:k])
    for i in np.flatnonzero(sel):
        assert np.sum(mag > mag[i]) < k
    if 0 < k < v.size:
        assert mag[sel.reshape(-1)].min() >= mag[~sel.reshape(-1)].max()


def test_add_noise_sets_requested_snr():
    """add_noise: the SNR measured on its output (mean |s|^2 over the full grid over the
    mean power of what it added) is within 0.1 dB of the request, on a 256^2 point-target
    echo whose mean power is far from 1 (so an amplitude-for-power slip shows), at
    10, 20 and 30 dB; the noise covers every element of the grid."""
    g = synth.airborne(256, 256)
    rng = np.random.default_rng(12)
    rows, cols, amps = synth.point_targets(rng, 256, 256, 5)
    s = echo.point_echo(g, rows, cols, 3.0 * amps)
    p = float(np.mean(np.abs(s) ** 2))
    assert abs(np.log10(p)) > 0.3
    for snr in (10.0, 20.0, 30.0):
        out = echo.add_noise(synth.cn_noise(rng, s.shape), s, snr)
        n = out - s
        meas = 10.0 * np.log10(p / float(np.mean(np.abs(n) ** 2)))
        assert abs(meas - snr) < 0.1, (snr, meas)
        assert np.count_nonzero(n) == n.size


# ----------------------------------------------------------------------------- ITA

@pytest.mark.parametrize("kind", ["soft", "half", "hard"])
def test_full_sampling_closed_form(kind):
    """With S = 1 and mu = 1, M G = I gives B = X + M(Y - G X) = M(Y) at every
    iteration, so every iterate equals T_sigma(M(Y)) with sigma = |M Y|_(K+1)."""
    g = synth.airborne(64, 128)
    rng = np.random.default_rng(7)
    y = _rand(rng, (64, 128))
    mask = np.ones((64, 128), dtype=bool)
    k = 40
    my = csa.focus_M(g, y)
    ref = ita.threshold(my, ita.kth_largest_magnitude(my, k), kind)
    for iters in (1, 3):
        x, st = ita.ita(g, y, mask, k, iters, kind=kind)
        assert metrics.rel_l2(x, ref) < 1e-12
        assert st[-1].nnz <= k


def test_first_iterate_is_threshold_of_masked_mf():
    """X^(1) = T(mu M(S . Y)) for X^(0) = 0 at any mask and step."""
    g = synth.airborne(64, 64)
    rng = np.random.default_rng(8)
    y = _rand(rng, (64, 64))
    mask = synth.bernoulli_mask(rng, 64, 64, 0.4)
    b = 0.7 * csa.focus_M(g, mask * y)
    ref = ita.soft_threshold(b, ita.kth_largest_magnitude(b, 10))
    x, _ = ita.ita(g, y, mask, 10, 1, mu=0.7)
    assert metrics.rel_l2(x, ref) < 1e-12


def test_niht_step_properties():
    """||S G v|| <= ||v|| makes mu_i >= 1; at full sampling ||G v|| = ||v|| gives mu = 1."""
    g = synth.airborne(64, 64)
    rng = np.random.default_rng(9)
    dx = _rand(rng, (64, 64))
    sup = ita.top_k_support(dx, 30)
    assert abs(ita.niht_step(g, np.ones((64, 64)), dx, sup) - 1.0) < 1e-12
    mask = synth.bernoulli_mask(rng, 64, 64, 0.5)
    assert ita.niht_step(g, mask, dx, sup) > 1.0


def _config1_problem(seed):
    g = synth.airborne(256, 256)
    rng = np.random.default_rng(seed)
    rows, cols, amps = synth.point_targets(rng, 256, 256, 5)
    s = echo.point_echo(g, rows, cols, amps)
    s = echo.add_noise(synth.cn_noise(rng, s.shape), s, 30.0)
    mask = synth.bernoulli_mask(rng, 256, 256, 0.5)
    return g, rows, cols, s * mask, mask


@pytest.mark.parametrize("mode", ["fixed", "niht"])
def test_config1_recovers_point_support(mode):
    """256^2 airborne, 5 unit point targets, 30 dB noise, 50% Bernoulli sampling,
    K = 5, 100 iterations: the support of X^(100) is the 5 true pixels."""
    g, rows, cols, y, mask = _config1_problem(0)
    x, st = ita.ita(g, y, mask, 5, 100, mu_mode=mode)
    got = set(zip(*np.nonzero(x)))
    assert got == set(zip(rows.tolist(), cols.tolist()))
    assert st[-1].resid_sq < st[0].resid_sq
    if mode == "niht":
        assert all(s.mu >= 1.0 for s in st)
