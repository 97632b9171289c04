"""Quality experiments of Section V-A on synthetic data, with both operator pairs
(CS-RDA and CS-CSA) and the matched filter (MF = M(S.Y), the conventional image):

* reconstruction ability (RA): 9 unit-amplitude targets with uniform random phases on a
  3 x 3 lattice of 6-sample spacing at the scene centre, exact time-domain echoes, 20 dB
  noise, the paper's row-then-range sampling with s_a : s_r = 1 : 5, K = 18, 100
  iterations with the adaptive (NIHT) step of Section IV-B, and with mu = 1 for
  comparison; sampling rates from 100% down to 0.45%.  A reconstruction succeeds when the
  pixels at or above half the largest magnitude are exactly the 9 targets.
* reconstruction quality (RQ): one point target at the centre, noise-free, 10% samples
  for CS (K = 600) and 100% for the MF; PSLR and IRW of x16-upsampled 16-sample cuts
  through the peak in range and azimuth, under two readings of the upsampling: band-
  limited (FFT zero padding, as in the matched-filter pins) and linear interpolation of
  the magnitude.

System parameters: the Table 2 simulation column on a 256 x 256 grid (the paper's
180 x 180 scene does not fit a power-of-two transform grid).  Run with ``-s`` to print
the tables."""
import numpy as np
import pytest

import synth
from gpu_helpers import dev, dev_mask, host, lib
from oracle import csa, echo, metrics

pytestmark = pytest.mark.gpu

N = 256
RATES = [1.0, 0.3, 0.1, 0.05, 0.03, 0.02, 0.013, 0.01, 0.0065, 0.0055, 0.0045]
SEEDS = [0, 1, 2]


def _rates(rate):
    """(s_a, s_r) with s_a s_r = rate and s_r = 5 s_a (s_r capped at 1)."""
    s_a = np.sqrt(rate / 5.0)
    s_r = 5.0 * s_a
    if s_r > 1.0:
        return rate, 1.0
    return s_a, s_r


def _lattice():
    c = N // 2
    return [(c + 6 * i, c + 6 * j) for i in (-1, 0, 1) for j in (-1, 0, 1)]


def _success(img, targets):
    mag = np.abs(img)
    top = mag.max()
    if top == 0:
        return False
    found = set(zip(*np.nonzero(mag >= 0.5 * top)))
    return found == set(targets)


def _ra_sweep(csar, rda_pair):
    g = synth.paper_table2_simulation(N, N)
    plan = csar.csar_plan_create(g, flags=csar.PLAN_RDA if rda_pair else 0)
    targets = _lattice()
    rows = [t[0] for t in targets]
    cols = [t[1] for t in targets]
    table = {}
    for rate in RATES:
        cs_ok = fx_ok = mf_ok = 0
        for seed in SEEDS:
            rng = np.random.default_rng(100 + seed)
            amps = np.exp(2j * np.pi * rng.random(9))
            s = echo.point_echo(g, rows, cols, amps)
            s = echo.add_noise(synth.cn_noise(rng, s.shape), s, 20.0)
            mask = synth.row_then_range_mask(rng, N, N, *_rates(rate))
            if not mask.any():
                continue
            y = dev(mask * s)
            m = dev_mask(mask)
            cs_ok += _success(host(csar.csar_solve(plan, y, m, 18, 100, mu_mode="niht")), targets)
            fx_ok += _success(host(csar.csar_solve(plan, y, m, 18, 100)), targets)
            mf_ok += _success(host(csar.csar_M(plan, y)), targets)
        table[rate] = (cs_ok, mf_ok, fx_ok)
    return table


def _lowest_all(table, col):
    ok = [r for r, v in table.items() if v[col] == len(SEEDS)]
    return min(ok) if ok else None


def _pslr_irw_linear(cut, factor=16):
    """PSLR (dB) and IRW (original samples) of |cut| linearly interpolated by
    ``factor``; lobes and the -3 dB width as in ``metrics.pslr_irw``."""
    m = np.abs(np.asarray(cut))
    u = np.interp(np.arange((m.size - 1) * factor + 1) / factor, np.arange(m.size), m)
    p = int(np.argmax(u))
    lo, hi = p, p
    while lo > 0 and u[lo - 1] < u[lo]:
        lo -= 1
    while hi < u.size - 1 and u[hi + 1] < u[hi]:
        hi += 1
    side = np.concatenate([u[:lo], u[hi + 1:]])
    pslr = 20.0 * np.log10(side.max() / u[p]) if side.size and side.max() > 0 else -np.inf
    a, b = p, p
    while a > 0 and u[a - 1] >= u[p] / np.sqrt(2.0):
        a -= 1
    while b < u.size - 1 and u[b + 1] >= u[p] / np.sqrt(2.0):
        b += 1
    return float(pslr), (b - a + 1) / factor


def _cuts(g, img, win=8):
    """Peak pixel and (PSLR, IRW) of the range and azimuth cuts, band-limited and
    linear readings."""
    pr, pc = np.unravel_index(np.argmax(np.abs(img)), img.shape)
    az = img[pr - win:pr + win, pc]
    rg = img[pr, pc - win:pc + win] * np.exp(
        -4j * np.pi * csa.r0_grid(g)[pc - win:pc + win] / g.wavelength)
    return ((int(pr), int(pc)), metrics.pslr_irw(rg), metrics.pslr_irw(az),
            _pslr_irw_linear(rg), _pslr_irw_linear(az))


def _rq(csar, rda_pair):
    g = synth.paper_table2_simulation(N, N)
    plan = csar.csar_plan_create(g, flags=csar.PLAN_RDA if rda_pair else 0)
    c = N // 2
    s = echo.point_echo(g, [c], [c], [1.0])
    mf = host(csar.csar_M(plan, dev(s)))
    rng = np.random.default_rng(7)
    mask = synth.row_then_range_mask(rng, N, N, *_rates(0.1))
    X = host(csar.csar_solve(plan, dev(mask * s), dev_mask(mask), 600, 100))
    return _cuts(g, mf), _cuts(g, X)


@pytest.mark.parametrize("pair", ["rda", "csa"])
def test_reconstruction_ability(pair):
    """Every method recovers the lattice from all samples; at 10% CS still recovers it
    on at least 2 of the 3 seeds where the matched-filter image no longer separates it
    from the artefacts of the random pulse selection.  (The paper reports CS-RDA success
    down to 0.65%; this setup's CS fails from 5% down: see the printed table.)"""
    csar = lib()
    table = _ra_sweep(csar, pair == "rda")
    print(f"\nRA, CS-{pair.upper()} vs MF: successes out of {len(SEEDS)} seeds")
    print("rate     CS(NIHT)  MF  CS(mu=1)")
    for rate, (cs_ok, mf_ok, fx_ok) in table.items():
        print(f"{rate * 100:6.2f}%  {cs_ok}         {mf_ok}   {fx_ok}")
    lo_cs, lo_mf = _lowest_all(table, 0), _lowest_all(table, 1)
    print(f"lowest rate with all seeds recovered: CS {lo_cs}, MF {lo_mf}")
    assert table[1.0][0] == len(SEEDS) and table[1.0][1] == len(SEEDS)
    assert table[0.1][0] >= 2 and table[0.1][0] >= table[0.1][1]


@pytest.mark.parametrize("pair", ["rda", "csa"])
def test_reconstruction_quality(pair):
    """Point response of the MF and of CS at 10% samples.  The paper reports
    -13.32 dB / 15 upsampled samples for the RDA image and -22.71 dB (range),
    -21.32 dB (azimuth) / 8 samples for CS-RDA; the printed table records what this
    setup gives under both upsampling readings.  Asserted: both peaks on the target's
    pixel, the MF's textbook sidelobe level, and the low range sidelobes of the sparse
    image under the linear reading (the band-limited upsampling of a near-single-pixel
    image is itself a sinc with -13 dB sidelobes)."""
    csar = lib()
    mf, cs = _rq(csar, pair == "rda")
    print(f"\nRQ, {pair.upper()} (IRW in x16 samples)")
    for name, (pk, rg, az, rg_l, az_l) in (("MF", mf), ("CS", cs)):
        print(f"{name} peak {pk}  band-limited: PSLR(R) {rg[0]:7.2f} PSLR(A) {az[0]:7.2f} "
              f"IRW(R) {rg[1] * 16:5.1f} IRW(A) {az[1] * 16:5.1f}  linear: PSLR(R) {rg_l[0]:7.2f} "
              f"PSLR(A) {az_l[0]:7.2f} IRW(R) {rg_l[1] * 16:5.1f} IRW(A) {az_l[1] * 16:5.1f}")
    c = N // 2
    assert mf[0] == (c, c) and cs[0] == (c, c)
    assert mf[1][0] < -12.0 and mf[2][0] < -12.0
    assert cs[3][0] < -18.0


def _ra_case(g, rate, seed, sampling):
    rng = np.random.default_rng(100 + seed)
    targets = _lattice()
    amps = np.exp(2j * np.pi * rng.random(9))
    s = echo.point_echo(g, [t[0] for t in targets], [t[1] for t in targets], amps)
    s = echo.add_noise(synth.cn_noise(rng, s.shape), s, 20.0)
    if sampling == "row_range":
        mask = synth.row_then_range_mask(rng, N, N, *_rates(rate))
    elif sampling == "row_range_5to1":
        s_r = np.sqrt(rate / 5.0)
        s_a = 5.0 * s_r
        mask = synth.row_then_range_mask(rng, N, N, *((s_a, s_r) if s_a <= 1.0 else (1.0, rate)))
    else:
        mask = synth.bernoulli_mask(rng, N, N, rate)
    return mask * s, mask


@pytest.mark.parametrize("sampling", ["row_range", "row_range_5to1", "bernoulli"])
def test_reconstruction_ability_gpu_matches_oracle(sampling):
    """The RA sweep (CS-RDA, NIHT step, K = 18, 100 iterations, 20 dB noise, seed 0) run
    by the FP64 oracle and by the GPU gives the same success at every rate, under three
    readings of the paper's sampling: row-then-range with s_a : s_r = 1 : 5 (few pulses,
    many range samples each), the same with the ratio the other way round (5 : 1), and
    i.i.d. 2-D sampling.  With the 5 : 1 reading or 2-D sampling CS-RDA succeeds at every
    rate down to 0.65%, the lowest rate the paper reports as recovered; with 1 : 5 it
    fails below 10% (9 of 256 pulses kept at 0.65%).  The printed table records all."""
    from oracle import ita
    csar = lib()
    g = synth.paper_table2_simulation(N, N)
    plan = csar.csar_plan_create(g, flags=csar.PLAN_RDA)
    targets = _lattice()
    rows = []
    for rate in RATES[:-2]:                      # down to 0.65%
        y, mask = _ra_case(g, rate, 0, sampling)
        x_ref, _ = ita.ita(g, y, mask, 18, 100, mu_mode="niht", ops="rda")
        xg = host(csar.csar_solve(plan, dev(y), dev_mask(mask), 18, 100, mu_mode="niht"))
        rows.append((rate, _success(x_ref, targets), _success(xg, targets)))
    print(f"\nRA ({sampling}), CS-RDA seed 0: rate oracle GPU")
    for rate, o, gg in rows:
        print(f"{rate * 100:6.2f}%  {int(o)}  {int(gg)}")
    assert all(o == gg for _, o, gg in rows)
    if sampling != "row_range":
        assert all(o for _, o, _ in rows)
    else:
        assert rows[0][1] and rows[2][1] and not rows[-1][1]
