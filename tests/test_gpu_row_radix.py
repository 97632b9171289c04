"""GPU parity of the range passes' second radix schedule (16 values per thread: a row of
8192 bins as 2 x 16 x 16 x 16 instead of 8 x 32 x 32; rows of 1024 to 8192 bins), which
the autotuner may choose per shape: the operators G and M against the FP64 oracle, ITA
solves within 1e-6 of the default schedule (the same arithmetic in another radix order),
and the autotuner's record of its choice."""
import numpy as np
import pytest

import synth
from gpu_helpers import crand, dev, dev_mask, host, lib
from oracle import csa, metrics

pytestmark = pytest.mark.gpu


@pytest.mark.parametrize("na,nr", [(512, 1024), (256, 2048), (256, 4096), (128, 8192)])
def test_radix16_operators_match_oracle(na, nr, monkeypatch):
    csar = lib()
    import torch
    g = synth.airborne(na, nr)
    rng = np.random.default_rng(nr)
    x = crand(rng, (na, nr))
    monkeypatch.setenv("CSAR_ROW_REGS", "16")
    plan = csar.csar_plan_create(g)
    assert metrics.rel_l2(host(csar.csar_G(plan, dev(x))), csa.observe_G(g, x)) < 1e-5
    X = dev(x)
    csar.csar_M(plan, X, X)
    torch.cuda.synchronize()
    assert metrics.rel_l2(host(X), csa.focus_M(g, x)) < 1e-5
    csar.csar_plan_check(plan)


@pytest.mark.parametrize("na,nr", [(1024, 2048), (512, 8192)])
def test_radix16_ita_matches_default(na, nr, monkeypatch):
    csar = lib()
    g = synth.airborne(na, nr)
    rng = np.random.default_rng(5)
    xt = synth.sparse_rayleigh(rng, na, nr, 0.01)
    mask = synth.bernoulli_mask(rng, na, nr, 0.5)
    y = mask * csa.observe_G(g, xt)
    K = int(round(0.01 * na * nr))
    Y, M = dev(y), dev_mask(mask)
    ref = host(csar.csar_solve(csar.csar_plan_create(g), Y, M, K, 5))
    monkeypatch.setenv("CSAR_ROW_REGS", "16")
    plan = csar.csar_plan_create(g)
    got = host(csar.csar_solve(plan, Y, M, K, 5))
    csar.csar_plan_check(plan)
    assert metrics.rel_l2(got, ref) < 1e-6


def test_autotune_records_range_schedule(tmp_path, monkeypatch):
    """The tune file holds one line per shape: main and residue column configurations and
    the range passes' values per thread (16 or 32)."""
    csar = lib()
    f = tmp_path / "tune.txt"
    monkeypatch.setenv("CSAR_TUNE_FILE", str(f))
    g = synth.airborne(1024, 2048)
    assert csar.csar_autotune(g, iters=3) in (1, 2, 4, 8, 16)
    rows = [list(map(int, ln.split())) for ln in f.read_text().splitlines() if ln.strip()]
    mine = [r for r in rows if r[:2] == [1024, 2048]]
    assert len(mine) == 1 and len(mine[0]) == 7 and mine[0][6] in (16, 32)
    rng = np.random.default_rng(6)
    x = crand(rng, (1024, 2048))
    plan = csar.csar_plan_create(g)
    assert metrics.rel_l2(host(csar.csar_G(plan, dev(x))), csa.observe_G(g, x)) < 1e-5
