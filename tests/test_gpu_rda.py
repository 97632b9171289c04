"""GPU parity of the range-Doppler operator pair (Section III-C: range compression,
azimuth FFT, 8-tap truncated-sinc RCMC C with the azimuth matched filter, azimuth IFFT;
G = M^H with D = C^T) against the FP64 oracle, and Theorem 1 on the GPU."""
import numpy as np
import pytest

import synth
from gpu_helpers import crand, dev, host, lib
from oracle import metrics, rda

pytestmark = pytest.mark.gpu
TOL = 1e-5

SHAPES = [("air", 16, 16), ("air", 256, 256), ("air", 512, 1024), ("lband", 64, 512),
          ("lband", 4096, 512), ("space", 1024, 256), ("space", 8192, 1024)]


def _geom(kind, na, nr):
    return {"air": synth.airborne, "space": synth.spaceborne, "lband": synth.wide_beam_lband}[kind](na, nr)


@pytest.mark.parametrize("kind,na,nr", SHAPES)
def test_rda_G_and_M_match_oracle(kind, na, nr):
    csar = lib()
    g = _geom(kind, na, nr)
    plan = csar.csar_plan_create(g, flags=csar.PLAN_RDA)
    rng = np.random.default_rng(na + 3 * nr)
    x = crand(rng, (na, nr))
    y = crand(rng, (na, nr))
    assert metrics.rel_l2(host(csar.csar_G(plan, dev(x))), rda.observe_G(g, x)) < TOL
    assert metrics.rel_l2(host(csar.csar_M(plan, dev(y))), rda.focus_M(g, y)) < TOL


def test_rda_theorem1_and_in_place_on_gpu():
    """<G x, y> = <x, M y> computed by the CUDA path only; in-place G and M."""
    import torch
    csar = lib()
    g = synth.wide_beam_lband(1024, 2048)
    plan = csar.csar_plan_create(g, flags=csar.PLAN_RDA)
    rng = np.random.default_rng(12)
    x, y = dev(crand(rng, (1024, 2048))), dev(crand(rng, (1024, 2048)))
    gx = csar.csar_G(plan, x)
    my = csar.csar_M(plan, y)
    lhs = torch.vdot(y.reshape(-1).to(torch.complex128), gx.reshape(-1).to(torch.complex128))
    rhs = torch.vdot(my.reshape(-1).to(torch.complex128), x.reshape(-1).to(torch.complex128))
    assert abs((lhs - rhs) / lhs).item() < TOL
    d = x.clone()
    csar.csar_G(plan, d, d)
    assert (torch.linalg.vector_norm(d - gx) / torch.linalg.vector_norm(gx)).item() < 1e-6
    d = y.clone()
    csar.csar_M(plan, d, d)
    assert (torch.linalg.vector_norm(d - my) / torch.linalg.vector_norm(my)).item() < 1e-6


def test_rda_plan_rejects_the_ita():
    csar = lib()
    g = synth.airborne(64, 64)
    plan = csar.csar_plan_create(g, flags=csar.PLAN_RDA)
    y = dev(crand(np.random.default_rng(1), (64, 64)))
    from gpu_helpers import dev_mask
    with pytest.raises(csar.CsarError) as e:
        csar.csar_solve(plan, y, dev_mask(np.ones((64, 64), bool)), 10, 2)
    assert e.value.status == 2


def test_rda_plan_rejects_steep_migration():
    """The transpose's atomic-free scatter needs a migration slope alpha = 1/D - 1 of at
    most 1/2 (D >= 2/3); a PRF whose edge Doppler reaches 0.8 of 2V/lambda (D = 0.6,
    alpha = 2/3) is refused at plan creation."""
    import dataclasses
    csar = lib()
    g = dataclasses.replace(synth.airborne(64, 64), prf=0.8 * 4 * 150.0 / 0.03)
    with pytest.raises(csar.CsarError) as e:
        csar.csar_plan_create(g, flags=csar.PLAN_RDA)
    assert e.value.status == 2


def test_rda_G_is_deterministic():
    """The transpose D = C^T sums each accumulator in a fixed order: repeated G calls
    agree bit for bit (also on a row length with several rows per CTA)."""
    import torch
    csar = lib()
    for na, nr in ((512, 8192), (256, 512)):
        plan = csar.csar_plan_create(synth.wide_beam_lband(na, nr), flags=csar.PLAN_RDA)
        x = dev(crand(np.random.default_rng(na), (na, nr)))
        a = csar.csar_G(plan, x)
        b = csar.csar_G(plan, x)
        assert torch.equal(a, b)
