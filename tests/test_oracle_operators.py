"""Pins of the FP64 oracle's operators M and G against what the paper and the
mathematics fix (no GPU)."""
import json
import os

import numpy as np
import pytest

import synth
from oracle import csa, echo, metrics

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")


def _rand(rng, shape):
    return rng.standard_normal(shape) + 1j * rng.standard_normal(shape)


# ----------------------------------------------------------------------------- FFT axes

def test_fft_axes_match_direct_dft():
    """F_a acts down columns (azimuth, axis 0), F_r along rows (range, axis 1),
    unnormalised forward / 1/N inverse: compare with the DFT sum written out."""
    rng = np.random.default_rng(1)
    x = _rand(rng, (8, 16))
    na, nr = x.shape
    fa = np.exp(-2j * np.pi * np.outer(np.arange(na), np.arange(na)) / na)
    fr = np.exp(-2j * np.pi * np.outer(np.arange(nr), np.arange(nr)) / nr)
    assert np.allclose(csa.fft_az(x), fa @ x, atol=1e-12)
    assert np.allclose(csa.fft_rg(x), x @ fr.T, atol=1e-12)
    assert np.allclose(csa.ifft_az(fa @ x), x, atol=1e-12)
    assert np.allclose(csa.ifft_rg(x @ fr.T), x, atol=1e-12)


# ----------------------------------------------------------------------------- Theorem 1, dense

def _dense_operators(g):
    """Matrices of M and G on vec(X) (column-major vec, as in Eqs. (19)-(22)):
    F_eta_hat = I (x) F_eta, F_tau_hat = F_tau^T (x) I, P_hat = diag(vec P)."""
    na, nr = g.n_az, g.n_rg
    f_eta = np.exp(-2j * np.pi * np.outer(np.arange(na), np.arange(na)) / na)
    f_tau = np.exp(-2j * np.pi * np.outer(np.arange(nr), np.arange(nr)) / nr)
    fe = np.kron(np.eye(nr), f_eta)
    fr = np.kron(f_tau.T, np.eye(na))
    fe_inv = np.kron(np.eye(nr), np.conj(f_eta) / na)
    fr_inv = np.kron(np.conj(f_tau).T / nr, np.eye(na))
    p1 = np.diag(csa.h1(g).reshape(-1, order="F"))
    p2 = np.diag(csa.h2(g).reshape(-1, order="F"))
    p3 = np.diag(csa.h3(g).reshape(-1, order="F"))
    m = fe_inv @ p3 @ fr_inv @ p2 @ fr @ p1 @ fe
    gm = fe_inv @ p1.conj() @ fr_inv @ p2.conj() @ fr @ p3.conj() @ fe
    return m, gm


@pytest.mark.parametrize("shape", [(16, 16), (8, 32), (32, 8)])
def test_dense_kronecker_form(shape):
    """The FFT-based M and G equal their Kronecker-product matrices, and the
    matrices satisfy G^H = M (Theorem 1) and M G = I (G = M^{-1})."""
    g = synth.airborne(*shape)
    m, gm = _dense_operators(g)
    rng = np.random.default_rng(2)
    for _ in range(3):
        x = _rand(rng, shape)
        v = x.reshape(-1, order="F")
        assert np.allclose(csa.focus_M(g, x).reshape(-1, order="F"), m @ v, atol=1e-11)
        assert np.allclose(csa.observe_G(g, x).reshape(-1, order="F"), gm @ v, atol=1e-11)
    assert np.allclose(gm.conj().T, m, atol=1e-12)
    assert np.allclose(m @ gm, np.eye(m.shape[0]), atol=1e-11)


# ----------------------------------------------------------------------------- invariants

@pytest.mark.parametrize("geom", ["air", "space"])
def test_unitarity_and_adjoint(geom):
    """M(G(Y)) = Y, G(M(X)) = X, ||G x|| = ||x|| and <G x, y> = <x, M y> to roundoff."""
    g = synth.airborne(256, 256) if geom == "air" else synth.spaceborne(128, 512)
    rng = np.random.default_rng(3)
    x = _rand(rng, (g.n_az, g.n_rg))
    y = _rand(rng, (g.n_az, g.n_rg))
    assert metrics.rel_l2(csa.focus_M(g, csa.observe_G(g, y)), y) < 1e-13
    assert metrics.rel_l2(csa.observe_G(g, csa.focus_M(g, x)), x) < 1e-13
    gx = csa.observe_G(g, x)
    assert abs(np.linalg.norm(gx) / np.linalg.norm(x) - 1) < 1e-13
    lhs = np.vdot(y, gx)
    rhs = np.vdot(csa.focus_M(g, y), x)
    assert abs(lhs - rhs) / abs(lhs) < 1e-12


def test_phase_tables_are_unit_modulus():
    g = synth.spaceborne(64, 256)
    for h in (csa.h1(g), csa.h2(g), csa.h3(g)):
        assert np.allclose(np.abs(h), 1.0, atol=1e-14)


# ----------------------------------------------------------------------------- point targets

def _focus_and_measure(g, rows, cols, win=16):
    """Focus each target's echo on its own; return (peak pixel, az, rg metrics)."""
    out = []
    for r, c in zip(rows, cols):
        x = csa.focus_M(g, echo.point_echo(g, [r], [c], [1.0]))
        pr, pc = np.unravel_index(np.argmax(np.abs(x)), x.shape)
        az = x[pr - win:pr + win, pc]
        # the focused range cut carries the per-bin carrier exp(+j 4 pi R0 / lambda);
        # remove it before band-limited upsampling
        rg = x[pr, pc - win:pc + win] * np.exp(
            -4j * np.pi * csa.r0_grid(g)[pc - win:pc + win] / g.wavelength)
        out.append(((pr, pc), metrics.pslr_irw(az), metrics.pslr_irw(rg)))
    return out


def test_point_targets_focus_airborne():
    """Exact time-domain echoes of point targets focus on their own pixels, with
    azimuth resolution La/2 and range resolution 0.886 c/(2B) (3 dB widths of a
    uniformly weighted aperture / chirp) and ~-13.3 dB sidelobes."""
    g = synth.airborne(256, 256)
    rng = np.random.default_rng(0)
    rows, cols, _ = synth.point_targets(rng, 256, 256, 5)
    res = _focus_and_measure(g, rows, cols)
    # all five together: each is a local maximum on its own pixel
    x = np.abs(csa.focus_M(g, echo.point_echo(g, rows, cols, np.ones(5))))
    for r, c in zip(rows, cols):
        assert x[r, c] == x[r - 2:r + 3, c - 2:c + 3].max()
    az_spacing = g.velocity / g.prf
    rg_spacing = g.c / (2 * g.fs)
    for (pk, (az_pslr, az_irw), (rg_pslr, rg_irw)), r, c in zip(res, rows, cols):
        assert pk == (r, c)
        assert abs(az_pslr - (-13.26)) < 0.1
        assert -13.7 < rg_pslr < -13.1
        assert abs(az_irw * az_spacing / (g.antenna_len / 2) - 1) < 0.03
        assert abs(rg_irw * rg_spacing / (0.886 * g.c / (2 * g.bandwidth)) - 1) < 0.03


def test_point_target_matches_paper_table2_simulation():
    """With the paper's own simulation parameters (Table 2), the fully sampled matched
    filter reproduces the range point response printed in Section V-A: IRW of 15
    samples after x16 upsampling and a PSLR of about -13.32 dB."""
    with open(os.path.join(GOLDEN, "paper_point_response.json")) as f:
        ref = json.load(f)
    g = synth.paper_table2_simulation(256, 256)
    assert abs(g.bandwidth / g.pulse_len - ref["table2_simulation"]["range_fm_rate_mhz_per_us"] * 1e12) < 1
    (pk, _, (rg_pslr, rg_irw)), = _focus_and_measure(g, [128], [128])
    assert pk == (128, 128)
    assert round(rg_irw * ref["upsample_factor"]) == ref["irw_range_upsampled_samples"]
    assert abs(rg_pslr - ref["pslr_range_db"]) < 0.2


def test_residual_phase_sign_far_range():
    """Targets far from the reference range (256 x 2048 airborne grid) stay focused in
    azimuth only if the residual phase of H3 carries the right sign: a flipped or
    dropped residual term leaves a quadratic Doppler phase (PSLR -10.3 / -12.2 dB)."""
    g = synth.airborne(256, 2048)
    res = _focus_and_measure(g, [128, 128], [200, 1900])
    for (pk, (az_pslr, _), _), c in zip(res, [200, 1900]):
        assert pk == (128, c)
        assert az_pslr < -12.9


def test_src_and_bulk_rcmc_wide_beam():
    """In a wide-beam L-band geometry (range migration ~10 bins, K_m differs from K_r by
    ~1%) point targets focus on their pixels with near-textbook sidelobes only if the
    bulk RCMC term and the modified FM rate K_m (secondary range compression) are
    right: K_m = K_r gives range PSLR -12.5 dB, a flipped SRC term -11.1 dB."""
    g = synth.wide_beam_lband(4096, 512)
    res = _focus_and_measure(g, [2048, 2048], [256, 102])
    for (pk, (az_pslr, _), (rg_pslr, _)), c in zip(res, [256, 102]):
        assert pk == (2048, c)
        assert rg_pslr < -13.1
        assert az_pslr < -12.5
