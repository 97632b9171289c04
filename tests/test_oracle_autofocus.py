"""Pins of the oracle's autofocus gradients by central finite differences (no GPU)."""
import numpy as np
import pytest

import synth
from oracle import autofocus as af
from oracle import csa, ita


def _problem(seed=0, na=32, nr=32, frac=0.02):
    g = synth.airborne(na, nr)
    rng = np.random.default_rng(seed)
    x = synth.sparse_rayleigh(rng, na, nr, frac)
    theta_true = synth.theta_sinusoids(rng, na, peak=0.5)
    mask = synth.bernoulli_mask(rng, na, nr, 0.5)
    y = mask * (np.exp(1j * theta_true)[:, None] * csa.observe_G(g, x))
    theta = synth.theta_sinusoids(rng, na, peak=0.3)
    return g, y, mask, theta, x


def test_rotation_identity():
    """A_theta^H A_theta = M S G does not depend on theta; the ITA on Y_theta equals the
    ITA with the theta-observation written out."""
    g, y, mask, theta, x = _problem(1)
    ph = np.exp(1j * theta)[:, None]
    lhs = csa.focus_M(g, np.conj(ph) * mask * (y - ph * csa.observe_G(g, x)))
    rhs = csa.focus_M(g, mask * (af.rotate(y, theta) - csa.observe_G(g, x)))
    assert np.allclose(lhs, rhs, atol=1e-12)


def test_loss_gradients_by_finite_differences():
    g, y, mask, theta, x = _problem(2)
    loss, gx, gth = af.loss_and_grads(g, y, mask, theta, x)
    eps = 1e-6
    rng = np.random.default_rng(3)
    for _ in range(3):
        d = rng.standard_normal(theta.shape)
        fd = (af.loss_and_grads(g, y, mask, theta + eps * d, x)[0]
              - af.loss_and_grads(g, y, mask, theta - eps * d, x)[0]) / (2 * eps)
        assert abs(fd - np.dot(gth, d)) <= 1e-6 * max(1.0, abs(fd))
        dz = rng.standard_normal(x.shape) + 1j * rng.standard_normal(x.shape)
        fd = (af.loss_and_grads(g, y, mask, theta, x + eps * dz)[0]
              - af.loss_and_grads(g, y, mask, theta, x - eps * dz)[0]) / (2 * eps)
        assert abs(fd - np.real(np.vdot(gx, dz))) <= 1e-6 * max(1.0, abs(fd))


@pytest.mark.parametrize("seed", [0, 4])
def test_unrolled_gradient_by_finite_differences(seed):
    """d/dtheta of ||S.(Y_theta - G X_I(theta))||^2 through I = 6 soft-threshold
    iterations, against central differences along random directions (the support
    does not change within +-eps for these seeds, checked)."""
    g, y, mask, theta, x = _problem(seed)
    k, iters = 20, 6
    loss, grad, xi, ck = af.unrolled_loss_grad(g, y, mask, theta, k, iters)
    rng = np.random.default_rng(10 + seed)
    eps = 1e-6
    for _ in range(4):
        d = rng.standard_normal(theta.shape)
        lp, _, xp, _ = af.unrolled_loss_grad(g, y, mask, theta + eps * d, k, iters)
        lm, _, xm, _ = af.unrolled_loss_grad(g, y, mask, theta - eps * d, k, iters)
        assert np.array_equal(xp != 0, xi != 0) and np.array_equal(xm != 0, xi != 0)
        fd = (lp - lm) / (2 * eps)
        assert abs(fd - np.dot(grad, d)) <= 1e-5 * max(1.0, abs(fd)), (fd, np.dot(grad, d))


def test_unroll_backward_wrt_start_by_finite_differences():
    """Xbar^(0) from the backward equals the derivative of the loss with respect to a
    non-zero starting iterate X^(0)."""
    g, y, mask, theta, x = _problem(5)
    k, iters = 20, 4
    x0 = 0.3 * x

    def f(z0):
        xi, ck = af.ita_unroll(g, y, mask, theta, k, iters, x0=z0)
        return af.loss_and_grads(g, y, mask, theta, xi), xi, ck

    (loss, gx, _), xi, ck = f(x0)
    _, x0bar = af.unroll_backward(g, y, mask, theta, ck, gx)
    rng = np.random.default_rng(6)
    eps = 1e-6
    for _ in range(3):
        dz = rng.standard_normal(x.shape) + 1j * rng.standard_normal(x.shape)
        fd = (f(x0 + eps * dz)[0][0] - f(x0 - eps * dz)[0][0]) / (2 * eps)
        assert abs(fd - np.real(np.vdot(x0bar, dz))) <= 1e-5 * max(1.0, abs(fd))


def test_threshold_vjp_matches_jacobian_of_soft_threshold():
    """The threshold VJP equals the transpose of the finite-difference Jacobian of
    b -> soft(b, |b|_(K+1)) (sigma moving with b)."""
    rng = np.random.default_rng(7)
    b = rng.standard_normal(12) + 1j * rng.standard_normal(12)
    k = 5

    def f(bb):
        s = ita.kth_largest_magnitude(bb, k)
        return ita.soft_threshold(bb, s)

    xn = f(b)
    mag = np.abs(b)
    j = int(np.argsort(-mag, kind="stable")[k])
    xbar = rng.standard_normal(12) + 1j * rng.standard_normal(12)
    bbar = af.threshold_vjp(xn, mag[j], j, b[j], xbar)
    eps = 1e-7
    for i in range(12):
        for dz in (1.0, 1j):
            e = np.zeros(12, complex)
            e[i] = eps * dz
            fd = np.real(np.vdot(xbar, (f(b + e) - f(b - e)) / (2 * eps)))
            assert abs(fd - np.real(np.conj(bbar[i]) * dz)) < 1e-6
