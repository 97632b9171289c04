"""GPU parity of the approximated observation G and the focusing operator M against
the FP64 oracle (relative L2 <= 1e-5 per operator application), and the operator
invariants (M G = I, adjoint identity, norm preservation) on the GPU."""
import numpy as np
import pytest

import synth
from gpu_helpers import crand, dev, host, lib
from oracle import csa, metrics

pytestmark = pytest.mark.gpu
TOL = 1e-5

SHAPES = [
    ("air", 16, 16), ("air", 16, 64), ("air", 64, 16), ("air", 32, 128), ("air", 256, 256),
    ("air", 512, 1024), ("air", 2048, 2048), ("space", 128, 512), ("space", 1024, 256),
    ("space", 4096, 512), ("lband", 4096, 512),
]


def _geom(kind, na, nr):
    if kind == "air":
        return synth.airborne(na, nr)
    if kind == "space":
        return synth.spaceborne(na, nr)
    return synth.wide_beam_lband(na, nr)


@pytest.mark.parametrize("kind,na,nr", SHAPES)
def test_G_and_M_match_oracle(kind, na, nr):
    csar = lib()
    g = _geom(kind, na, nr)
    plan = csar.csar_plan_create(g)
    rng = np.random.default_rng(na * 7 + nr)
    x = crand(rng, (na, nr))
    y = crand(rng, (na, nr))
    gx = host(csar.csar_G(plan, dev(x)))
    my = host(csar.csar_M(plan, dev(y)))
    assert metrics.rel_l2(gx, csa.observe_G(g, x)) < TOL
    assert metrics.rel_l2(my, csa.focus_M(g, y)) < TOL


@pytest.mark.parametrize("kind,na,nr", [("air", 256, 256), ("space", 1024, 2048), ("air", 64, 4096)])
def test_invariants_on_gpu(kind, na, nr):
    """M(G(y)) = y, the adjoint identity <G x, y> = <x, M y> (Theorem 1) and
    ||G x|| = ||x||, all computed by the CUDA path only."""
    import torch
    csar = lib()
    plan = csar.csar_plan_create(_geom(kind, na, nr))
    rng = np.random.default_rng(11)
    x, y = dev(crand(rng, (na, nr))), dev(crand(rng, (na, nr)))
    mgy = csar.csar_M(plan, csar.csar_G(plan, y))
    assert (torch.linalg.vector_norm(mgy - y) / torch.linalg.vector_norm(y)).item() < TOL
    gx = csar.csar_G(plan, x)
    my = csar.csar_M(plan, y)
    lhs = torch.vdot(y.reshape(-1).to(torch.complex128), gx.reshape(-1).to(torch.complex128))
    rhs = torch.vdot(my.reshape(-1).to(torch.complex128), x.reshape(-1).to(torch.complex128))
    assert abs((lhs - rhs) / lhs).item() < TOL
    ratio = (torch.linalg.vector_norm(gx) / torch.linalg.vector_norm(x)).item()
    assert abs(ratio - 1) < TOL


def test_in_place_and_point_target_focus():
    """In-place G/M; an exact time-domain point echo focuses on its pixel on the GPU."""
    from oracle import echo
    csar = lib()
    g = synth.airborne(256, 256)
    plan = csar.csar_plan_create(g)
    s = echo.point_echo(g, [128, 150], [128, 100], [1.0, 1.0])
    d = dev(s)
    csar.csar_M(plan, d, d)
    xg = host(d)
    assert metrics.rel_l2(xg, csa.focus_M(g, s)) < TOL
    a = np.abs(xg)
    assert a[128, 128] == a[120:137, 120:137].max() and a[150, 100] == a[142:159, 92:109].max()
    csar.csar_G(plan, d, d)
    assert metrics.rel_l2(host(d), s) < TOL


def test_full_size_spaceborne_8192():
    """The 8192 x 8192 spaceborne operators against the oracle at full size."""
    csar = lib()
    g = synth.spaceborne(8192, 8192)
    plan = csar.csar_plan_create(g)
    rng = np.random.default_rng(3)
    x = synth.targets_over_clutter(rng, 8192, 8192)
    gx_gpu = host(csar.csar_G(plan, dev(x)))
    gx = csa.observe_G(g, x)
    assert metrics.rel_l2(gx_gpu, gx) < TOL
    del gx_gpu
    mx_gpu = host(csar.csar_M(plan, dev(gx)))
    assert metrics.rel_l2(mx_gpu, x) < TOL
