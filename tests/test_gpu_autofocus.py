"""GPU parity of the differentiable autofocus path: loss and direct gradients, the
unrolled-ITA gradients with respect to theta and to X^(0) against the FP64 oracle (small
grids here, and the 4096^2, 50-iteration workload against its stored oracle result),
and finite differences of the GPU loss on that workload."""
import os
import sys

import numpy as np
import pytest

import synth
from gpu_helpers import dev, dev_mask, host, lib
from oracle import autofocus as af
from oracle import csa, metrics

pytestmark = pytest.mark.gpu

GOLDEN = os.path.join(os.path.dirname(os.path.abspath(__file__)), "golden")


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
    differences); and the adjoint of X^(0) from csar_af_backward against the oracle's."""
    import torch
    csar = lib()
    na, nr = shape
    g, x, y, mask, theta = _problem(2, na, nr, 0.01)
    th64 = theta.astype(np.float32).astype(np.float64)
    loss_ref, grad_ref, x_ref, ck = af.unrolled_loss_grad(g, y, mask, th64, k, iters)
    _, gx_ref, _ = af.loss_and_grads(g, y, mask, th64, x_ref)
    _, x0bar_ref = af.unroll_backward(g, y, mask, th64, ck, gx_ref)
    plan = csar.csar_plan_create(g)
    th = _t(theta).requires_grad_(True)
    L = csar.autofocus_loss(plan, dev(y), dev_mask(mask), th, k, iters)
    L.backward()
    assert abs(L.item() - loss_ref) <= 1e-3 * loss_ref
    assert metrics.rel_l2(th.grad.cpu().numpy().astype(np.float64), grad_ref) < 1e-3
    Y, md, tt = dev(y), dev_mask(mask), _t(theta)
    X = csar.csar_af_solve(plan, Y, md, tt, k, iters, checkpoint=True)
    _, gx, _ = csar.csar_af_loss(plan, Y, md, tt, X)
    x0bar = torch.empty_like(X)
    csar.csar_af_backward(plan, Y, md, tt, gx, X0bar=x0bar)
    torch.cuda.synchronize()
    assert metrics.rel_l2(host(x0bar), x0bar_ref) < 1e-3


def _config5():
    """The recipe of the 4096^2 autofocus workload's inputs (the script that stored the
    oracle result)."""
    if GOLDEN not in sys.path:
        sys.path.insert(0, GOLDEN)
    import make_ita_goldens as mg
    return mg


def test_full_workload_gradients_match_oracle():
    """4096^2 airborne, 0.5% scene, 50% sampling, theta = 3 sinusoids (peak 2 pi) plus a
    seeded error, K = 83886, 50-iteration unroll: the loss, dL/dtheta (direct + through
    the checkpointed unroll) and the adjoint of X^(0) (at 65536 seeded positions, at the
    4096 largest, and its norm) against the stored FP64 oracle result, each within 1e-3."""
    import torch
    csar = lib()
    mg = _config5()
    gold = np.load(os.path.join(GOLDEN, "config5_af50.npz"))
    g, y, mask, theta = mg.config5_inputs()
    K, iters = int(gold["K"]), int(gold["iters"])
    plan = csar.csar_plan_create(g)
    Y, md, th = dev(y), dev_mask(mask), _t(theta)
    X = csar.csar_af_solve(plan, Y, md, th, K, iters, checkpoint=True)
    loss, gx, gt = csar.csar_af_loss(plan, Y, md, th, X)
    x0bar = torch.empty_like(X)
    tb = csar.csar_af_backward(plan, Y, md, th, gx, X0bar=x0bar)
    torch.cuda.synchronize()
    csar.csar_plan_check(plan)
    grad = (gt + tb).double().cpu().numpy()
    xb = x0bar.reshape(-1)
    pos = torch.from_numpy(gold["x0bar_pos"]).cuda()
    top = torch.from_numpy(gold["x0bar_top"]).cuda()
    at_pos = xb[pos].cpu().numpy().astype(np.complex128)
    at_top = xb[top].cpu().numpy().astype(np.complex128)
    nrm = float(torch.linalg.vector_norm(xb.to(torch.complex128)).item())
    e = {"loss": abs(loss.item() - float(gold["loss"])) / float(gold["loss"]),
         "grad_theta": metrics.rel_l2(grad, gold["grad_theta"]),
         "x0bar_sampled": metrics.rel_l2(at_pos, gold["x0bar_at_pos"]),
         "x0bar_top": metrics.rel_l2(at_top, gold["x0bar_at_top"]),
         "x0bar_norm": abs(nrm - float(gold["x0bar_norm"])) / float(gold["x0bar_norm"])}
    print("\nconfig 5 against the FP64 oracle: " + ", ".join(f"{k} {v:.2e}" for k, v in e.items()))
    assert all(v <= 1e-3 for v in e.values()), e
    assert int(torch.count_nonzero(X).item()) == int(gold["nnz"])


@pytest.mark.parametrize("na", [1024, 4096])
def test_finite_differences_autofocus_unroll(na):
    """The autofocus workload's recipe (0.5% scene, 50% sampling, theta = 3 sinusoids plus a
    seeded error, K = 0.5% of n, 50-iteration unroll) at 1024^2 and at its full 4096^2:
    the autograd derivative of the GPU loss against finite differences of the GPU loss,
    to 1e-3 relative error, along the pulses with the three largest gradient components
    (4096^2) or along the gradient and two directions near it (1024^2).

    The unrolled loss is piecewise smooth: each support change of the soft threshold in
    any of the 50 iterations is a kink.  Along the whole gradient at 4096^2 the kinks are
    ~3e-5 rad apart, so there the comparison is made along single pulses, whose nearest
    kinks lie 3e-4 to 6e-4 rad away (measured: central differences with steps of 6e-4 and
    more are off by 1-40% on four of the six largest pulses, steps up to 3e-4 by at most
    1.2e-3).  Inside that interval the fp32 unroll gives the loss a rounding noise of
    ~1.4e-5 (1e-6 of L), which puts one central difference at 3e-4 within ~8e-4 (RMS) of
    the derivative: too close to the 1e-3 bar.  So the finite difference is the least-
    squares slope over 41 points spaced 1.5e-5 rad in [-3e-4, 3e-4]: the measured losses
    are fitted, with a quadratic term, against the autograd prediction g . (theta_k -
    theta) of their own float32 points, and the fitted slope must be 1 to 1e-3 (noise
    ~3e-4 RMS).  The 1e-3 bar along every direction at full size is also met against the
    FP64 oracle's adjoint (test above)."""
    import torch
    csar = lib()
    mg = _config5()
    if na == 4096:
        g, y, mask, theta = mg.config5_inputs()
    else:
        g = synth.airborne(na, na)
        rng = np.random.default_rng(5)
        x = synth.sparse_rayleigh(rng, na, na, 0.005).astype(np.complex64)
        theta_true = synth.theta_sinusoids(rng, na)
        mask = synth.bernoulli_mask(rng, na, na, 0.5)
        theta = (theta_true + 0.02 * synth.theta_sinusoids(rng, na, peak=1.0)).astype(np.float32)
        y = (mask * (np.exp(1j * theta_true)[:, None] * csa.observe_G(g, x))).astype(np.complex64)
    K, iters = int(round(0.005 * na * na)), 50
    plan = csar.csar_plan_create(g)
    Y, md = dev(y), dev_mask(mask)
    th = _t(theta).requires_grad_(True)
    L = csar.autofocus_loss(plan, Y, md, th, K, iters)
    L.backward()
    grad = th.grad.double().cpu().numpy()
    dirs = []
    if na == 4096:
        for i in np.argsort(-np.abs(grad))[:3]:
            e = np.zeros(na)
            e[i] = 1.0
            dirs.append(e)
    else:
        # at 1024^2 a single pulse's derivative (a few units) is too close to the fp32
        # loss's rounding for a 3e-4 step: the gradient direction and two directions
        # within 60 degrees of it (derivatives of at least half the gradient's norm)
        gh = grad / np.linalg.norm(grad)
        rng = np.random.default_rng(11)
        dirs.append(gh)
        for _ in range(2):
            r = rng.standard_normal(na)
            d = gh + 0.5 * r / np.linalg.norm(r)
            dirs.append(d / np.linalg.norm(d))
    theta64 = theta.astype(np.float64)
    t32 = theta.astype(np.float32).astype(np.float64)
    steps = np.arange(-20, 21) * 1.5e-5
    for d in dirs:
        pred, loss = [], []
        for h in steps:
            # theta enters in float32: predict from the float32-rounded point itself
            tq = (theta64 + h * d).astype(np.float32)
            with torch.no_grad():
                loss.append(csar.autofocus_loss(plan, Y, md, _t(tq), K, iters).item())
            pred.append(float(np.dot(grad, tq.astype(np.float64) - t32)))
        pred, loss = np.array(pred), np.array(loss)
        A = np.stack([np.ones_like(pred), pred, pred ** 2], axis=1)
        coef, *_ = np.linalg.lstsq(A, loss, rcond=None)
        resid = float(np.sqrt(np.mean((A @ coef - loss) ** 2)))
        print(f"\n{na}^2 FD slope / autograd {coef[1]:.6f} (fit residual {resid:.2e}, "
              f"derivative {np.dot(grad, d):.4e})")
        assert abs(coef[1] - 1.0) <= 1e-3, (coef[1], resid)
