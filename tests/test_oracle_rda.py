"""Pins of the FP64 oracle's RDA operator pair (Section III-C: Eqs. (14)-(18), (22);
truncated-sinc RCMC) against the matrix form of Theorem 1, exact shifts and point
targets (no GPU)."""
import json
import os

import numpy as np
import pytest

import synth
from oracle import csa, echo, metrics, rda

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")


def _rand(rng, shape):
    return rng.standard_normal(shape) + 1j * rng.standard_normal(shape)


def _dense_rda(g):
    """Matrices of M and G on vec(X) (column-major vec, Eqs. (19)-(22)) with the RCMC
    matrix C built entry by entry from its definition: for azimuth-frequency bin k and
    output range bin i, taps j = floor(i + dr) - 3 + t (mod N_r), weight sinc(j - i - dr)."""
    na, nr = g.n_az, g.n_rg
    f_eta = np.exp(-2j * np.pi * np.outer(np.arange(na), np.arange(na)) / na)
    f_tau = np.exp(-2j * np.pi * np.outer(np.arange(nr), np.arange(nr)) / nr)
    fe = np.kron(np.eye(nr), f_eta)
    fr = np.kron(f_tau.T, np.eye(na))
    fe_inv = np.kron(np.eye(nr), np.conj(f_eta) / na)
    fr_inv = np.kron(np.conj(f_tau).T / nr, np.eye(na))
    pt = np.diag(np.tile(rda.range_filter(g)[None, :], (na, 1)).reshape(-1, order="F"))
    pe = np.diag(rda.azimuth_filter(g).reshape(-1, order="F"))
    dr = rda.migration(g)
    cm = np.zeros((na * nr, na * nr))
    for k in range(na):
        for i in range(nr):
            pos = i + dr[k, i]
            b = int(np.floor(pos)) - 3
            for t in range(8):
                j = (b + t) % nr
                cm[i * na + k, j * na + k] += np.sinc(b + t - pos)
    m = fe_inv @ pe @ cm @ fe @ fr_inv @ pt @ fr
    gm = fr_inv @ pt.conj() @ fr @ fe_inv @ cm.T @ pe.conj() @ fe
    return m, gm


@pytest.mark.parametrize("shape,geom", [((16, 16), "lband"), ((8, 32), "lband"), ((16, 16), "air")])
def test_rda_dense_matrix_form_and_theorem1(shape, geom):
    """The FFT/interpolation operators equal their matrices, and G^H = M exactly
    (Theorem 1: D = C^T)."""
    g = synth.wide_beam_lband(*shape) if geom == "lband" else synth.airborne(*shape)
    m, gm = _dense_rda(g)
    rng = np.random.default_rng(4)
    for _ in range(2):
        x = _rand(rng, shape)
        v = x.reshape(-1, order="F")
        assert np.allclose(rda.focus_M(g, x).reshape(-1, order="F"), m @ v, atol=1e-11)
        assert np.allclose(rda.observe_G(g, x).reshape(-1, order="F"), gm @ v, atol=1e-11)
    assert np.allclose(gm.conj().T, m, atol=1e-12)


@pytest.mark.parametrize("geom", ["air", "space", "lband"])
def test_rda_adjoint_identity(geom):
    """<G x, y> = <x, M y> to roundoff at sizes beyond the dense test."""
    g = {"air": synth.airborne(128, 256), "space": synth.spaceborne(64, 512),
         "lband": synth.wide_beam_lband(256, 128)}[geom]
    rng = np.random.default_rng(5)
    x = _rand(rng, (g.n_az, g.n_rg))
    y = _rand(rng, (g.n_az, g.n_rg))
    lhs = np.vdot(y, rda.observe_G(g, x))
    rhs = np.vdot(rda.focus_M(g, y), x)
    assert abs(lhs - rhs) / abs(lhs) < 1e-12


def test_rcmc_integer_migration_is_a_shift():
    """With an integer migration the truncated sinc is a Kronecker delta: C is the
    circular shift by dr, and D = C^T the opposite shift."""
    rng = np.random.default_rng(6)
    v = _rand(rng, (4, 32))
    dr = np.zeros((4, 32)) + np.array([0, 1, 3, 7])[:, None]
    u = rda.rcmc_C(v, dr)
    for k, s in enumerate([0, 1, 3, 7]):
        assert np.allclose(u[k], np.roll(v[k], -s), atol=1e-14)
        assert np.allclose(rda.rcmc_D(u, dr)[k], v[k], atol=1e-14)


def _focus_and_measure(g, rows, cols, win=16):
    out = []
    for r, c in zip(rows, cols):
        x = rda.focus_M(g, echo.point_echo(g, [r], [c], [1.0]))
        pr, pc = np.unravel_index(np.argmax(np.abs(x)), x.shape)
        az = x[pr - win:pr + win, pc]
        rg = x[pr, pc - win:pc + win] * np.exp(
            -4j * np.pi * csa.r0_grid(g)[pc - win:pc + win] / g.wavelength)
        out.append(((pr, pc), metrics.pslr_irw(az), metrics.pslr_irw(rg)))
    return out


def test_rda_point_targets_airborne():
    """Exact time-domain echoes focus on their own pixels with azimuth resolution La/2,
    range resolution 0.886 c/(2B) and ~-13.3 dB sidelobes."""
    g = synth.airborne(256, 256)
    rng = np.random.default_rng(0)
    rows, cols, _ = synth.point_targets(rng, 256, 256, 5)
    az_spacing = g.velocity / g.prf
    rg_spacing = g.c / (2 * g.fs)
    for (pk, (az_pslr, az_irw), (rg_pslr, rg_irw)), r, c in zip(_focus_and_measure(g, rows, cols), rows, cols):
        assert pk == (r, c)
        assert abs(az_pslr - (-13.26)) < 0.1 and -13.7 < rg_pslr < -13.1
        assert abs(az_irw * az_spacing / (g.antenna_len / 2) - 1) < 0.03
        assert abs(rg_irw * rg_spacing / (0.886 * g.c / (2 * g.bandwidth)) - 1) < 0.03


def test_rda_matches_paper_table2_point_response():
    """The paper's RDA point response (Section V-A, Table 2 simulation column, 100%
    samples): range IRW of 15 samples after x16 upsampling, PSLR about -13.32 dB."""
    with open(os.path.join(GOLDEN, "paper_point_response.json")) as f:
        ref = json.load(f)
    g = synth.paper_table2_simulation(256, 256)
    (pk, (az_pslr, _), (rg_pslr, rg_irw)), = _focus_and_measure(g, [128], [128])
    assert pk == (128, 128)
    assert round(rg_irw * ref["upsample_factor"]) == ref["irw_range_upsampled_samples"]
    assert abs(rg_pslr - ref["pslr_range_db"]) < 0.35
    assert abs(az_pslr - ref["pslr_azimuth_db"]) < 0.35


def test_rcmc_needed_for_wide_beam():
    """With a wide beam (migration up to 36 range bins) the RCMC interpolation is what
    focuses the target in azimuth: without it (C = I) the azimuth response spreads."""
    g = synth.wide_beam_lband(4096, 512)
    (pk, (az_pslr, az_irw), _), = _focus_and_measure(g, [2048], [256])
    assert pk == (2048, 256) and az_pslr < -12.5
    s = echo.point_echo(g, [2048], [256], [1.0])
    a = csa.fft_az(csa.ifft_rg(csa.fft_rg(s) * rda.range_filter(g)[None, :]))
    x_no = np.abs(csa.ifft_az(a * rda.azimuth_filter(g)))
    x_ok = np.abs(rda.focus_M(g, s))
    assert x_no.max() < 0.7 * x_ok.max()


def test_cs_rda_recovers_point_targets():
    """Algorithm 1 over the range-Doppler pair (the paper's CS-RDA) on the 256^2
    airborne scene of 5 unit point targets (exact echo model, 30 dB noise, 50%
    sampling, K = 5): after 30 iterations the support is exactly the true pixels."""
    from oracle import ita
    g = synth.airborne(256, 256)
    rng = np.random.default_rng(0)
    rows, cols, amps = synth.point_targets(rng, 256, 256, 5)
    s = echo.point_echo(g, rows, cols, amps)
    s = echo.add_noise(synth.cn_noise(rng, s.shape), s, 30.0)
    mask = synth.bernoulli_mask(rng, 256, 256, 0.5)
    x, st = ita.ita(g, mask * s, mask, 5, 30, ops="rda")
    assert set(zip(*np.nonzero(x))) == set(zip(rows.tolist(), cols.tolist()))
    assert all(a.nnz <= 5 for a in st)
