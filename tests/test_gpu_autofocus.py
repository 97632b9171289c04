"""GPU parity of the differentiable autofocus path (spec differentiation row):
loss and direct gradients, the unrolled-ITA gradient with respect to theta against the
FP64 oracle, and finite differences of the GPU loss on the 4096^2 autofocus workload."""
import numpy as np
import pytest

import synth
from gpu_helpers import dev, dev_mask, host, lib
from oracle import autofocus as af
from oracle import csa, metrics

pytestmark = pytest.mark.gpu


def _problem(seed, na, nr, frac, rate=0.5, peak=2 * np.pi):
    g = synth.airborne(na, nr)
    rng = np.random.default_rng(seed)
    x = synth.sparse_rayleigh(rng, na, nr, frac)
    theta_true = synth.theta_sinusoids(rng, na, peak=peak)
    mask = synth.bernoulli_mask(rng, na, nr, rate)
    y = mask * (np.exp(1j * theta_true)[:, None] * csa.observe_G(g, x))
    theta = theta_true + 0.05 * synth.theta_sinusoids(rng, na, peak=1.0)
    return g, x, y, mask, theta


def _t(theta):
    import torch
    return torch.from_numpy(theta.astype(np.float32)).cuda()


@pytest.mark.parametrize("shape", [(64, 64), (256, 512)])
def test_loss_and_direct_gradients(shape):
    csar = lib()
    na, nr = shape
    g, x, y, mask, theta = _problem(1, na, nr, 0.02)
    xe = 0.9 * x
    loss, gx, gt = af.loss_and_grads(g, y, mask, theta.astype(np.float32).astype(np.float64), xe)
    plan = csar.csar_plan_create(g)
    l, gxd, gtd = csar.csar_af_loss(plan, dev(y), dev_mask(mask), _t(theta), dev(xe))
    assert abs(l.item() - loss) <= 1e-5 * loss
    assert metrics.rel_l2(host(gxd), gx) < 1e-4
    assert metrics.rel_l2(gtd.cpu().numpy().astype(np.float64), gt) < 1e-4


@pytest.mark.parametrize("shape,k,iters", [((64, 64), 40, 6), ((256, 256), 655, 10), ((2048, 128), 2621, 6)])
def test_unrolled_gradient_matches_oracle(shape, k, iters):
    """dL/dtheta through the unrolled ITA: torch.autograd over the C-ABI forward and
    backward against the oracle's hand-derived adjoint (itself pinned by finite
    differences)."""
    import torch
    csar = lib()
    na, nr = shape
    g, x, y, mask, theta = _problem(2, na, nr, 0.01)
    th64 = theta.astype(np.float32).astype(np.float64)
    loss_ref, grad_ref, x_ref, _ = af.unrolled_loss_grad(g, y, mask, th64, k, iters)
    plan = csar.csar_plan_create(g)
    th = _t(theta).requires_grad_(True)
    L = csar.autofocus_loss(plan, dev(y), dev_mask(mask), th, k, iters)
    L.backward()
    assert abs(L.item() - loss_ref) <= 1e-3 * loss_ref
    assert metrics.rel_l2(th.grad.cpu().numpy().astype(np.float64), grad_ref) < 1e-3


def test_finite_differences_full_autofocus_workload():
    """4096^2 airborne, 0.5% scene, 50% sampling, theta = 3 sinusoids (peak 2 pi),
    K = 83886, 50-iteration unroll: the autograd directional derivative of the GPU loss
    matches central differences of the GPU loss along random unit directions.  The
    unrolled loss is piecewise smooth (soft-threshold kinks at support changes) and its
    value carries fp32 rounding (~1e-4 relative at this residual level), so the step is
    3e-3 rad and the bar 1e-2 of the derivative's typical size along a random unit
    direction; the 1e-3 bar is checked against the FP64 oracle above."""
    import torch
    csar = lib()
    na = nr = 4096
    g = synth.airborne(na, nr)
    rng = np.random.default_rng(5)
    x = synth.sparse_rayleigh(rng, na, nr, 0.005).astype(np.complex64)
    theta_true = synth.theta_sinusoids(rng, na)
    mask = synth.bernoulli_mask(rng, na, nr, 0.5)
    plan = csar.csar_plan_create(g)
    yg = csar.csar_G(plan, dev(x))
    ph = torch.from_numpy(np.exp(1j * theta_true).astype(np.complex64)).cuda()[:, None]
    Y = (yg * ph).contiguous()
    md = dev_mask(mask)
    K, iters = 83886, 50
    theta = theta_true + 0.02 * synth.theta_sinusoids(rng, na, peak=1.0)
    th = _t(theta).requires_grad_(True)
    L = csar.autofocus_loss(plan, Y, md, th, K, iters)
    L.backward()
    grad = th.grad.double().cpu().numpy()
    eps = 3e-3
    # a random unit direction's derivative is typically |grad| / sqrt(n_az); one that is
    # nearly orthogonal to grad has a much smaller derivative whose central difference is
    # dominated by the loss's rounding, so the 1e-2 bar is relative to the larger of the
    # two values and that typical size
    typical = np.linalg.norm(grad) / np.sqrt(na)
    for _ in range(3):
        d = rng.standard_normal(na)
        d /= np.linalg.norm(d)
        with torch.no_grad():
            lp = csar.autofocus_loss(plan, Y, md, _t(theta + eps * d), K, iters).item()
            lm = csar.autofocus_loss(plan, Y, md, _t(theta - eps * d), K, iters).item()
        fd = (lp - lm) / (2 * eps)
        an = float(np.dot(grad, d))
        assert abs(fd - an) <= 1e-2 * max(abs(fd), abs(an), typical), (fd, an, typical)
