"""GPU parity of the persistent, tensor-copy-fed column passes (CSAR_PLAN_COL_PERSIST):
the operators G and M and ITA solves against the FP64 oracle in every built persistent
configuration (clusters of 1, 2, 4, 8 and 16 CTAs, tiles of 4 or 8 columns) with more
tiles than resident clusters (several tiles per cluster, a ragged last round); the
spaceborne 8192^2 operators; and agreement with the per-tile column kernels of the same
configuration."""
import numpy as np
import pytest

import synth
from gpu_helpers import crand, dev, dev_mask, host, lib
from oracle import csa, ita, metrics

pytestmark = pytest.mark.gpu


def _flags(csar, p=0, half=False):
    f = csar.PLAN_COL_PERSIST
    if p:
        f |= csar.plan_col_cluster(p)
    if half:
        f |= csar.PLAN_COL_HALF_TILE
    return f


@pytest.mark.parametrize("na,nr,p", [
    (8192, 1024, 8), (8192, 1024, 16), (4096, 512, 4), (2048, 1024, 2), (1024, 2048, 1)])
def test_persistent_operators_match_oracle(na, nr, p):
    """G and M, in place and out of place, against the oracle (rel-L2 <= 1e-5)."""
    csar = lib()
    import torch
    g = synth.spaceborne(na, nr) if na == 8192 else synth.airborne(na, nr)
    rng = np.random.default_rng(na + nr)
    x = crand(rng, (na, nr))
    plan = csar.csar_plan_create(g, flags=_flags(csar, p, half=True))
    yg = host(csar.csar_G(plan, dev(x)))
    assert metrics.rel_l2(yg, csa.observe_G(g, x)) < 1e-5
    X = dev(x)
    csar.csar_M(plan, X, X)
    torch.cuda.synchronize()
    assert metrics.rel_l2(host(X), csa.focus_M(g, x)) < 1e-5
    csar.csar_plan_check(plan)


@pytest.mark.parametrize("na,nr,p", [(8192, 1024, 8), (8192, 1024, 16), (4096, 512, 4), (2048, 1024, 2),
                                     (1024, 2048, 1)])
@pytest.mark.parametrize("mu_mode", ["fixed", "niht"])
def test_persistent_ita_matches_oracle(na, nr, p, mu_mode):
    """3 ITA iterations on a 2% scene against the oracle (support rule on the final
    image), and within 1e-6 of the per-tile column kernels of the same configuration (the
    same arithmetic; the order in which candidates and iterate entries are appended may
    differ, which changes summation order only)."""
    csar = lib()
    g = synth.airborne(na, nr)
    rng = np.random.default_rng(31)
    xt = synth.sparse_rayleigh(rng, na, nr, 0.02)
    mask = synth.bernoulli_mask(rng, na, nr, 0.5)
    y = mask * csa.observe_G(g, xt)
    K = int(round(0.02 * na * nr))
    x_ref, st_ref = ita.ita(g, y, mask, K, 2, mu_mode=mu_mode)
    x_ref, last, b_ref = ita.ita_iteration(g, y, mask.astype(float), x_ref, K, mu_mode, return_b=True)
    Y, M = dev(y), dev_mask(mask)
    plan = csar.csar_plan_create(g, flags=_flags(csar, p, half=True))
    X, st = csar.csar_solve(plan, Y, M, K, 3, mu_mode=mu_mode, stats=True)
    csar.csar_plan_check(plan)
    xg = host(X)
    clear = np.abs(np.abs(b_ref) - last.sigma) > 1e-4 * last.sigma
    assert np.array_equal((xg != 0)[clear], (x_ref != 0)[clear])
    assert metrics.rel_l2(xg, x_ref) < 1e-3
    sig_ref = np.array([s.sigma for s in st_ref] + [last.sigma])
    assert np.max(np.abs(st["sigma"] - sig_ref) / sig_ref) < 1e-4
    plain = csar.csar_plan_create(g, flags=csar.plan_col_cluster(p) | csar.PLAN_COL_HALF_TILE |
                                  csar.PLAN_COL_NO_PERSIST)
    X2 = csar.csar_solve(plain, Y, M, K, 3, mu_mode=mu_mode)
    assert metrics.rel_l2(xg, host(X2)) < 1e-6


def test_persistent_spaceborne_8192_operators():
    """The spaceborne 8192^2 grid (2048 tiles of 4 columns over the resident clusters):
    G against the oracle, and M(G(x)) = x (Theorem 1 with M G = I)."""
    csar = lib()
    import torch
    n = 8192
    g = synth.spaceborne(n, n)
    rng = np.random.default_rng(8)
    x = np.zeros((n, n), np.complex128)
    idx = rng.choice(n * n, 50000, replace=False)
    x.flat[idx] = crand(rng, 50000)
    plan = csar.csar_plan_create(g, flags=csar.PLAN_COL_PERSIST)
    y = csar.csar_G(plan, dev(x))
    yg = host(y)
    assert metrics.rel_l2(yg, csa.observe_G(g, x)) < 1e-5
    del yg
    csar.csar_M(plan, y, y)
    torch.cuda.synchronize()
    assert metrics.rel_l2(host(y), x) < 1e-5
    csar.csar_plan_check(plan)
