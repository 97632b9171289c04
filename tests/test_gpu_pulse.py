"""GPU parity of the non-chirp pulse (Section III-D, second generalisation: P_tau^*
replaced by the recorded transmitted pulse) on the range-Doppler pair: G and M with a
recorded spectrum (a Barker-13 phase code, and an arbitrary complex table) against the
FP64 oracle, the chirp filter restored, CS-RDA solves on Barker-coded point targets, and
the host checks (a chirp-scaling plan rejects a pulse; non-finite entries are refused)."""
import numpy as np
import pytest

import synth
from gpu_helpers import crand, dev, dev_mask, host, lib
from oracle import echo, ita, metrics, rda
from test_oracle_pulse import with_pulse

pytestmark = pytest.mark.gpu


def _barker(g):
    return rda.pulse_spectrum(g, synth.coded_pulse(synth.BARKER13, 3.0 / g.fs))


@pytest.mark.parametrize("geom,shape,table", [("air", (256, 256), "barker"), ("air", (128, 512), "random"),
                                              ("space", (8192, 1024), "barker")])
def test_recorded_pulse_operators_match_oracle(geom, shape, table):
    csar = lib()
    g = (synth.airborne if geom == "air" else synth.spaceborne)(*shape)
    rng = np.random.default_rng(3)
    spec = _barker(g) if table == "barker" else crand(rng, g.n_rg)
    spec = spec.astype(np.complex64).astype(np.complex128)   # the table as the GPU holds it
    gp = with_pulse(g, spec)
    plan = csar.csar_plan_create(g, flags=csar.PLAN_RDA)
    csar.csar_plan_set_pulse(plan, spec)
    x = crand(rng, shape)
    assert metrics.rel_l2(host(csar.csar_G(plan, dev(x))), rda.observe_G(gp, x)) < 1e-5
    assert metrics.rel_l2(host(csar.csar_M(plan, dev(x))), rda.focus_M(gp, x)) < 1e-5
    # back to the chirp filter
    csar.csar_plan_set_pulse(plan, None)
    assert metrics.rel_l2(host(csar.csar_G(plan, dev(x))), rda.observe_G(g, x)) < 1e-5
    csar.csar_plan_check(plan)


@pytest.mark.parametrize("mode", ["niht", "fixed"])
def test_cs_rda_coded_pulse_solve_matches_oracle(mode):
    """5 Barker-coded point targets (exact echo, 30 dB noise, 50% sampling, K = 5), 30
    iterations: the GPU recovers the 5 pixels and matches the oracle's image (NIHT with
    the recorded spectrum; fixed step with it scaled to peak magnitude 1)."""
    csar = lib()
    g = synth.airborne(256, 256)
    p = synth.coded_pulse(synth.BARKER13, 3.0 / g.fs)
    spec = _barker(g)
    if mode == "fixed":
        spec = spec / np.abs(spec).max()
    spec = spec.astype(np.complex64).astype(np.complex128)
    gp = with_pulse(g, spec)
    rng = np.random.default_rng(0)
    rows, cols, amps = synth.point_targets(rng, 256, 256, 5)
    s = echo.point_echo(g, rows, cols, amps, pulse=p)
    s = echo.add_noise(synth.cn_noise(rng, s.shape), s, 30.0)
    mask = synth.bernoulli_mask(rng, 256, 256, 0.5)
    y = mask * s
    x_ref, st_ref = ita.ita(gp, y, mask, 5, 30, ops="rda", mu_mode=mode)
    plan = csar.csar_plan_create(g, flags=csar.PLAN_RDA)
    csar.csar_plan_set_pulse(plan, spec)
    X, st = csar.csar_solve(plan, dev(y), dev_mask(mask), 5, 30, mu_mode=mode, stats=True)
    xg = host(X)
    assert set(zip(*np.nonzero(xg))) == set(zip(rows.tolist(), cols.tolist()))
    assert metrics.rel_l2(xg, x_ref) < 1e-3
    sig_ref = np.array([a.sigma for a in st_ref])
    assert np.max(np.abs(st["sigma"] - sig_ref) / sig_ref) < 1e-3


def test_recorded_pulse_host_checks():
    csar = lib()
    g = synth.airborne(64, 64)
    plan = csar.csar_plan_create(g)
    with pytest.raises(csar.CsarError) as e:
        csar.csar_plan_set_pulse(plan, np.ones(64, complex))
    assert e.value.status == 2
    plan_r = csar.csar_plan_create(g, flags=csar.PLAN_RDA)
    bad = np.ones(64, complex)
    bad[7] = np.nan
    with pytest.raises(csar.CsarError) as e:
        csar.csar_plan_set_pulse(plan_r, bad)
    assert e.value.status == 1
