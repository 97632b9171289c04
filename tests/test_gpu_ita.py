"""GPU parity of the ITA (Algorithm 1 / Eq. (25)) against the FP64 oracle: single
iterations with every step/threshold mode, full solves on the 256^2 point-target
workload and on distributed scenes, the degenerate cases, and the 8192^2 workload."""
import os

import numpy as np
import pytest

import synth
from gpu_helpers import crand, dev, dev_mask, host, lib
from oracle import csa, echo, ita, metrics

pytestmark = pytest.mark.gpu

GOLDEN = os.path.join(os.path.dirname(os.path.abspath(__file__)), "golden")


def assert_iterate_matches(x_gpu, x_ref, b_ref, sigma_ref, rel=1e-4, band=1e-4):
    """Identical support except entries with ||b| - sigma| <= band*sigma; values
    within rel (relative L2) of the oracle."""
    mag = np.abs(b_ref)
    clear = np.abs(mag - sigma_ref) > band * max(sigma_ref, 1e-30)
    sup_gpu = x_gpu != 0
    sup_ref = x_ref != 0
    assert np.array_equal(sup_gpu[clear], sup_ref[clear]), (
        int(np.sum(sup_gpu[clear] != sup_ref[clear])))
    if np.any(x_ref):
        assert metrics.rel_l2(x_gpu, x_ref) < rel
    else:
        assert np.abs(x_gpu).max() < 1e-6


def oracle_solve(g, y, mask, K, iters, **kw):
    """The oracle's Algorithm 1 for `iters` iterations, also returning b and sigma of the
    last iteration (for the support rule of the final image)."""
    x, st = ita.ita(g, y, mask, K, iters - 1, **kw)
    x, last, b = ita.ita_iteration(g, y, np.asarray(mask, dtype=np.float64), x, K, return_b=True,
                                   **{k: v for k, v in kw.items() if k != "x0"})
    return x, st + [last], b, last.sigma


def assert_final_matches_golden(xg, gold, rel=1e-3):
    """Final image against a stored oracle result: identical support outside the stored
    band (| |b| - sigma | <= 1e-4 sigma at the last iteration), values within rel."""
    flat = xg.reshape(-1)
    ref = np.zeros(flat.size, np.complex128)
    ref[gold["idx"]] = gold["val"]
    band = np.zeros(flat.size, dtype=bool)
    band[gold["band"]] = True
    diff = (flat != 0) != (ref != 0)
    assert not np.any(diff & ~band), int(np.sum(diff & ~band))
    assert metrics.rel_l2(flat, ref) < rel


def _problem(seed, na=256, nr=256, frac=0.01, rate=0.5, geom=synth.airborne, noise_db=None):
    g = geom(na, nr)
    rng = np.random.default_rng(seed)
    x = synth.sparse_rayleigh(rng, na, nr, frac)
    y = csa.observe_G(g, x)
    if noise_db is not None:
        y = echo.add_noise(synth.cn_noise(rng, y.shape), y, noise_db)
    mask = synth.bernoulli_mask(rng, na, nr, rate)
    return g, x, mask * y, mask


@pytest.mark.parametrize("mu_mode,mu,kind,x0", [
    ("fixed", 1.0, "soft", "sparse"), ("fixed", 0.7, "half", "sparse"),
    ("niht", 1.0, "soft", "sparse"), ("niht", 1.0, "half", "zero"), ("fixed", 1.3, "soft", "zero"),
    ("fixed", 1.0, "hard", "sparse"), ("niht", 1.0, "hard", "zero"),
])
@pytest.mark.parametrize("shape", [(256, 256), (64, 512), (1024, 128)])
def test_single_iteration(mu_mode, mu, kind, x0, shape):
    csar = lib()
    import torch
    na, nr = shape
    g, xt, y, mask = _problem(5, na, nr)
    rng = np.random.default_rng(9)
    x = (synth.sparse_rayleigh(rng, na, nr, 0.02) if x0 == "sparse"
         else np.zeros((na, nr), complex))
    K = int(0.01 * na * nr)
    x_ref, st, b_ref = ita.ita_iteration(g, y, mask, x, K, mu_mode, mu, kind, return_b=True)
    plan = csar.csar_plan_create(g)
    X = dev(x)
    sig = torch.zeros(1, dtype=torch.float32, device="cuda")
    csar.csar_ita_step(plan, dev(y), dev_mask(mask), X, K, mu_mode, mu, kind, sigma=sig)
    torch.cuda.synchronize()
    csar.csar_plan_check(plan)
    assert abs(sig.item() - st.sigma) <= 1e-5 * st.sigma
    xg = host(X)
    assert np.count_nonzero(xg) <= K
    assert_iterate_matches(xg, x_ref, b_ref, st.sigma)


def test_config1_point_targets_solve():
    """256^2 airborne, 5 unit point targets from the exact echo model + 30 dB noise,
    50% Bernoulli sampling, K = 5, 100 iterations: the GPU recovers the 5 pixels and
    matches the oracle image."""
    csar = lib()
    g = synth.airborne(256, 256)
    rng = np.random.default_rng(0)
    rows, cols, amps = synth.point_targets(rng, 256, 256, 5)
    s = echo.point_echo(g, rows, cols, amps)
    s = echo.add_noise(synth.cn_noise(rng, s.shape), s, 30.0)
    mask = synth.bernoulli_mask(rng, 256, 256, 0.5)
    y = mask * s
    x_ref, st_ref, b_ref, s_ref = oracle_solve(g, y, mask, 5, 100)
    plan = csar.csar_plan_create(g)
    X, st = csar.csar_solve(plan, dev(y), dev_mask(mask), 5, 100, stats=True)
    xg = host(X)
    assert set(zip(*np.nonzero(xg))) == set(zip(rows.tolist(), cols.tolist()))
    assert_iterate_matches(xg, x_ref, b_ref, s_ref, rel=1e-3)
    sig_ref = np.array([s_.sigma for s_ in st_ref])
    assert np.max(np.abs(st["sigma"] - sig_ref) / sig_ref) < 1e-3
    res_ref = np.array([s_.resid_sq for s_ in st_ref])
    assert np.max(np.abs(st["resid_sq"] - res_ref) / res_ref) < 1e-3


@pytest.mark.parametrize("mu_mode,kind", [("fixed", "soft"), ("niht", "soft"), ("fixed", "half"),
                                          ("niht", "hard")])
def test_distributed_scene_solve(mu_mode, kind):
    """512^2 airborne, 1% Rayleigh scene, G(X) echo + 20 dB noise, 50% sampling,
    K = 1% of n, 30 iterations."""
    csar = lib()
    g, xt, y, mask = _problem(21, 512, 512, noise_db=20.0)
    K = int(round(0.01 * 512 * 512))
    iters = 30
    x_ref, st_ref, b_ref, s_ref = oracle_solve(g, y, mask, K, iters, mu_mode=mu_mode, kind=kind)
    plan = csar.csar_plan_create(g)
    X, st = csar.csar_solve(plan, dev(y), dev_mask(mask), K, iters, mu_mode=mu_mode, thresh=kind,
                            stats=True)
    xg = host(X)
    assert_iterate_matches(xg, x_ref, b_ref, s_ref, rel=1e-3)
    assert np.all(st["nnz"] <= K)
    if mu_mode == "niht":
        # with hard thresholding the support-restricted gradient Delta X_Gamma vanishes
        # at a fixed point (in the oracle 6e-2 of |X| after one iteration, 4e-5 after
        # five, 7e-9 after eleven), so later NIHT steps are ratios of fp32 rounding
        n_mu = 5 if kind == "hard" else iters
        mu_ref = np.array([s_.mu for s_ in st_ref])[:n_mu]
        assert np.max(np.abs(st["mu"][:n_mu] - mu_ref) / mu_ref) < 1e-3


def test_degenerate_cases():
    csar = lib()
    import torch
    g, xt, y, mask = _problem(4, 128, 128)
    plan = csar.csar_plan_create(g)
    Y, M = dev(y), dev_mask(mask)
    # K = 0: sigma = max |b|, nothing survives
    assert not np.any(host(csar.csar_solve(plan, Y, M, 0, 3)))
    # K >= n: sigma = 0, soft threshold is the identity: X^(1) = mu M(S Y)
    x1 = host(csar.csar_solve(plan, Y, M, 128 * 128, 1))
    assert metrics.rel_l2(x1, csa.focus_M(g, y)) < 1e-5
    # all-zero echo and mask: the iterate stays 0
    z = torch.zeros_like(Y)
    assert not np.any(host(csar.csar_solve(plan, z, M, 100, 3)))
    m0 = dev_mask(np.zeros_like(mask))
    assert not np.any(host(csar.csar_solve(plan, Y, m0, 100, 3)))
    # full sampling, mu = 1: every iterate equals T(M(Y)) (closed form of M G = I)
    full = np.ones_like(mask)
    yf = crand(np.random.default_rng(2), (128, 128))
    xr = ita.soft_threshold(csa.focus_M(g, yf), ita.kth_largest_magnitude(csa.focus_M(g, yf), 300))
    for iters in (1, 4):
        xg = host(csar.csar_solve(plan, dev(yf), dev_mask(full), 300, iters))
        assert metrics.rel_l2(xg, xr) < 1e-4


def test_nonfinite_echo_is_reported():
    csar = lib()
    g, xt, y, mask = _problem(6, 64, 64)
    y = y.copy()
    idx = np.argwhere(mask)[0]
    y[tuple(idx)] = np.nan
    plan = csar.csar_plan_create(g)
    with pytest.raises(csar.CsarError) as e:
        csar.csar_solve(plan, dev(y), dev_mask(mask), 10, 2, stats=True)
    assert e.value.status == 6


def test_host_buffer_entry_point():
    csar = lib()
    import synth as sy
    g, xt, y, mask = _problem(8, 256, 256)
    plan = csar.csar_plan_create(g)
    K = 655
    xd = host(csar.csar_solve(plan, dev(y), dev_mask(mask), K, 10))
    xh = csar.csar_solve_host(plan, y.astype(np.complex64), sy.pack_mask(mask), K, 10)
    assert np.array_equal(xh.reshape(256, 256), xd.astype(np.complex64))


def test_full_size_spaceborne_iterations():
    """8192^2 spaceborne workload (2000 3x3 targets over -25 dB clutter, 40% sampling,
    K = 20000) in the launch configuration the benchmark times: 20 iterations against
    the stored FP64 oracle result (tests/golden/make_ita_goldens.py), final image with
    the support rule, sigma_i and ||r_i||^2 at every iteration."""
    csar = lib()
    gold = np.load(os.path.join(GOLDEN, "config3_it20.npz"))
    g = synth.spaceborne(8192, 8192)
    rng = np.random.default_rng(0)
    x = synth.targets_over_clutter(rng, 8192, 8192)
    mask = synth.bernoulli_mask(rng, 8192, 8192, 0.4)
    y = csa.observe_G(g, x)
    del x
    y *= mask
    K, iters = int(gold["K"]), int(gold["iters"])
    plan = csar.csar_plan_create(g)
    X, stg = csar.csar_solve(plan, dev(y), dev_mask(mask), K, iters, stats=True)
    del y
    xg = host(X)
    assert np.max(np.abs(stg["sigma"] - gold["sigma"]) / gold["sigma"]) <= 1e-4
    assert np.max(np.abs(stg["resid_sq"] - gold["resid_sq"]) / gold["resid_sq"]) <= 1e-4
    assert_final_matches_golden(xg, gold)


def test_dense_iterate_groups_are_deterministic():
    """Iterates with more entries per column group than the direct DFT takes use the
    clustered FFT path for G(X); repeated solves give bit-identical images."""
    csar = lib()
    g, xt, y, mask = _problem(12, 4096, 1024, frac=0.005)
    plan = csar.csar_plan_create(g)
    K = int(round(0.005 * 4096 * 1024))
    Y, M = dev(y), dev_mask(mask)
    a = host(csar.csar_solve(plan, Y, M, K, 8))
    b = host(csar.csar_solve(plan, Y, M, K, 8))
    assert np.array_equal(a, b)
    x_ref, _, b_ref, s_ref = oracle_solve(g, y, mask, K, 8)
    assert_iterate_matches(a, x_ref, b_ref, s_ref, rel=1e-3)


@pytest.mark.parametrize("na,nr,p,half", [
    (8192, 64, 1, 0), (8192, 64, 2, 0), (8192, 64, 4, 0), (8192, 64, 8, 0), (8192, 64, 16, 0),
    (8192, 64, 2, 1), (8192, 64, 4, 1), (8192, 64, 8, 1), (8192, 64, 16, 1),
    (4096, 128, 1, 0), (4096, 128, 4, 0), (4096, 128, 8, 0), (4096, 128, 1, 1), (4096, 128, 2, 1),
    (4096, 128, 4, 1), (4096, 128, 8, 1), (2048, 128, 2, 0), (2048, 128, 4, 0), (2048, 128, 1, 1), (2048, 128, 4, 1),
    (1024, 128, 1, 1), (8192, 64, 4, 2), (8192, 64, 8, 2)])
def test_every_column_configuration(na, nr, p, half):
    """The column passes under every configuration they are built for (cluster size,
    full, half (half = 1) or wide (half = 2) tiles: cross-CTA exchanges of the blocked and strided transforms, the
    residue pass, the selection and the sparse-input FFT path): 3 NIHT iterations on a
    2% scene against the oracle."""
    csar = lib()
    g, xt, y, mask = _problem(31, na, nr, frac=0.02)
    K = int(round(0.02 * na * nr))
    x_ref, st_ref, b_ref, s_ref = oracle_solve(g, y, mask, K, 3, mu_mode="niht")
    flags = csar.plan_col_cluster(p) | {0: 0, 1: csar.PLAN_COL_HALF_TILE, 2: csar.PLAN_COL_WIDE_TILE}[half]
    plan = csar.csar_plan_create(g, flags=flags)
    X, st = csar.csar_solve(plan, dev(y), dev_mask(mask), K, 3, mu_mode="niht", stats=True)
    csar.csar_plan_check(plan)
    assert_iterate_matches(host(X), x_ref, b_ref, s_ref, rel=1e-3)
    sig_ref = np.array([s_.sigma for s_ in st_ref])
    assert np.max(np.abs(st["sigma"] - sig_ref) / sig_ref) < 1e-4


@pytest.mark.parametrize("rate,iters", [(0.8, 4), (0.95, 3)])
def test_sharp_threshold_drops(rate, iters):
    """Noiseless bright sparse scene at high sampling: sigma falls by 4x (0.8) or 13x
    (0.95) per iteration, so the candidate cut predicted from the previous sigma is too
    high (exact re-pass) or the (K+1)-th key lies under the histogram floor (full
    re-pass, second check, candidate re-pass).  The GPU follows the oracle."""
    csar = lib()
    na = nr = 256
    g = synth.airborne(na, nr)
    rng = np.random.default_rng(3)
    k = 60 if rate > 0.9 else 30
    x = np.zeros((na, nr), complex)
    idx = rng.choice(na * nr, k, replace=False)
    x.flat[idx] = 10 * np.exp(2j * np.pi * rng.random(k))
    mask = synth.bernoulli_mask(rng, na, nr, rate)
    y = mask * csa.observe_G(g, x)
    x_ref, st_ref, b_ref, s_ref = oracle_solve(g, y, mask, k, iters)
    sig_ref = np.array([s_.sigma for s_ in st_ref])
    assert np.max(sig_ref[:-1] / sig_ref[1:]) > (6.0 if rate > 0.9 else 3.0)
    plan = csar.csar_plan_create(g)
    X, st = csar.csar_solve(plan, dev(y), dev_mask(mask), k, iters, stats=True)
    csar.csar_plan_check(plan)
    assert np.max(np.abs(st["sigma"] - sig_ref) / sig_ref) < 1e-2
    xg = host(X)
    assert set(np.flatnonzero(xg)) == set(np.flatnonzero(x_ref))
    assert_iterate_matches(xg, x_ref, b_ref, s_ref, rel=1e-3)


@pytest.mark.parametrize("rate", [0.3, 0.5])
def test_config2_precision_study(rate):
    """2048^2 airborne precision study: 1% Rayleigh scene (sigma = 1), echo G(X) + 20 dB
    noise, Bernoulli sampling at 30% and 50%, K = 41943.  Per-operator rel-L2 of the
    complex64 G and M against the FP64 oracle (<= 1e-5) and the ITA against the oracle
    over the configuration's 200 iterations (stored oracle result,
    tests/golden/make_ita_goldens.py): final image <= 1e-3 with the support rule,
    sigma_i and ||r_i||^2 <= 1e-4 at every iteration; the values are printed."""
    csar = lib()
    na = nr = 2048
    g = synth.airborne(na, nr)
    rng = np.random.default_rng(2)
    x = synth.sparse_rayleigh(rng, na, nr, 0.01)
    y_clean = csa.observe_G(g, x)
    y = echo.add_noise(synth.cn_noise(rng, y_clean.shape), y_clean, 20.0)
    mask = synth.bernoulli_mask(rng, na, nr, rate)
    ys = mask * y
    plan = csar.csar_plan_create(g)
    e_g = metrics.rel_l2(host(csar.csar_G(plan, dev(x))), y_clean)
    e_m = metrics.rel_l2(host(csar.csar_M(plan, dev(ys))), csa.focus_M(g, ys))
    gold = np.load(os.path.join(GOLDEN, f"config2_r{int(round(rate * 100))}.npz"))
    K, iters = int(gold["K"]), int(gold["iters"])
    X, st = csar.csar_solve(plan, dev(ys), dev_mask(mask), K, iters, stats=True)
    csar.csar_plan_check(plan)
    xg = host(X)
    ref = np.zeros(na * nr, complex)
    ref[gold["idx"]] = gold["val"]
    e_x = metrics.rel_l2(xg.reshape(-1), ref)
    e_s = float(np.max(np.abs(st["sigma"] - gold["sigma"]) / gold["sigma"]))
    e_r = float(np.max(np.abs(st["resid_sq"] - gold["resid_sq"]) / gold["resid_sq"]))
    print(f"\nconfig 2, {int(rate * 100)}% sampling: rel-L2 G {e_g:.2e}, M {e_m:.2e}, "
          f"X^({iters}) {e_x:.2e}; max sigma rel err {e_s:.2e}, max resid rel err {e_r:.2e}")
    assert e_g < 1e-5 and e_m < 1e-5
    assert e_s < 1e-4 and e_r < 1e-4
    assert_final_matches_golden(xg, gold)
    assert np.count_nonzero(xg) <= K
