"""Differentiable autofocus through the unrolled ITA (FP64).

TEST INFRASTRUCTURE ONLY (see ``oracle/__init__``).

Observation with a per-pulse azimuth phase error theta (one value per echo row):
    A_theta X = S . (exp(j theta_eta) . G(X)),   A_theta^H r = M(exp(-j theta_eta) . S . r).
Because |exp(j theta)| = 1 and S is 0/1, the ITA of Eq. (25) for this observation is
the plain ITA on the de-rotated echo Y_theta = exp(-j theta_eta) . Y, and the loss
    L(X, theta) = ||Y - A_theta X||^2 = ||S . (Y_theta - G(X))||^2.

Gradients use the torch convention for complex arguments (dL/dRe + j dL/dIm, i.e.
dL = Re <grad, dz>).  With r = S . (Y_theta - G(X)):
    grad_X L      = -2 M(r)
    dL/dtheta_eta = 2 sum_tau Im(conj(r) Y_theta)          (row eta)

Backward through one soft-threshold iteration X' = T_sigma(B), B = X + mu M(S.(Y_theta - G X)),
sigma = |B|_(K+1) (the element j*):  for kept entries (|b| > sigma), u = b/|b|,
    bbar = (1 - sigma/|b|) xbar + (sigma/|b|) Re(conj(u) xbar) u,
    sigmabar = -sum_kept Re(conj(u) xbar),   bbar_{j*} += sigmabar u_{j*};
then  Xbar += bbar - mu M(S . G(bbar)),   Ybar_theta += mu S . G(bbar),
and every Ybar_theta contributes  thetabar_eta += sum_tau Im(conj(Ybar_theta) Y_theta).
These are derived here (the paper does not differentiate the method) and pinned by
central finite differences in tests/test_oracle_autofocus.py.
"""
from __future__ import annotations

import dataclasses

import numpy as np

from . import csa, ita


def rotate(y: np.ndarray, theta: np.ndarray) -> np.ndarray:
    """Y_theta = exp(-j theta_eta) . Y (row eta = pulse eta)."""
    return np.exp(-1j * np.asarray(theta, dtype=np.float64))[:, None] * y


def loss_and_grads(g, y, mask, theta, x):
    """L = ||S.(Y_theta - G X)||^2, grad_X L, dL/dtheta."""
    yt = rotate(y, theta)
    r = mask * (yt - csa.observe_G(g, x))
    loss = float(np.vdot(r, r).real)
    gx = -2.0 * csa.focus_M(g, r)
    gth = 2.0 * np.sum(mask * np.imag(np.conj(r) * yt), axis=1)
    return loss, gx, gth


@dataclasses.dataclass
class Checkpoint:
    x_next: np.ndarray    # X^(i+1)
    sigma: float          # sigma_i
    jstar: int            # flat index of the (K+1)-th largest |b|
    b_jstar: complex      # b at j*


def ita_unroll(g, y, mask, theta, k, iters, mu=1.0, x0=None):
    """Soft-threshold ITA with fixed step on Y_theta from X^(0) = x0 (default 0),
    keeping one checkpoint per iteration.  Returns (X^(iters), checkpoints)."""
    yt = rotate(y, theta)
    x = (np.zeros((g.n_az, g.n_rg), complex) if x0 is None else np.asarray(x0, complex).copy())
    ck = []
    for _ in range(iters):
        r = mask * (yt - csa.observe_G(g, x))
        b = x + mu * csa.focus_M(g, r)
        mag = np.abs(b).reshape(-1)
        order = np.argsort(-mag, kind="stable")
        jstar = int(order[k]) if k < mag.size else -1
        sigma = float(mag[jstar]) if jstar >= 0 else 0.0
        x = ita.soft_threshold(b, sigma)
        ck.append(Checkpoint(x.copy(), sigma, jstar, complex(b.reshape(-1)[jstar]) if jstar >= 0 else 0j))
    return x, ck


def threshold_vjp(x_next, sigma, jstar, b_jstar, xbar):
    """bbar of the soft threshold at sigma = |b_{j*}| for output X' = x_next."""
    bbar = np.zeros_like(xbar)
    kept = x_next != 0
    xk = x_next[kept]
    u = xk / np.abs(xk)
    bmag = np.abs(xk) + sigma
    xb = xbar[kept]
    proj = np.real(np.conj(u) * xb)
    bbar[kept] = (1.0 - sigma / bmag) * xb + (sigma / bmag) * proj * u
    if jstar >= 0 and sigma > 0:
        sbar = -float(np.sum(proj))
        flat = bbar.reshape(-1)
        flat[jstar] += sbar * b_jstar / abs(b_jstar)
    return bbar


def unroll_backward(g, y, mask, theta, ck, xbar_final, mu=1.0):
    """Adjoint of ita_unroll: returns (thetabar, Xbar^(0)) for the adjoint xbar_final
    of X^(iters)."""
    yt = rotate(y, theta)
    xbar = np.asarray(xbar_final, complex).copy()
    thbar = np.zeros(g.n_az)
    for c in reversed(ck):
        bbar = threshold_vjp(c.x_next, c.sigma, c.jstar, c.b_jstar, xbar)
        gb = mask * csa.observe_G(g, bbar)
        xbar = bbar - mu * csa.focus_M(g, gb)
        thbar += mu * np.sum(np.imag(np.conj(gb) * yt), axis=1)
    return thbar, xbar


def unrolled_loss_grad(g, y, mask, theta, k, iters, mu=1.0):
    """L(theta) = ||S.(Y_theta - G X_I(theta))||^2 with X_I the unrolled ITA, and
    dL/dtheta (direct + through the unroll)."""
    x, ck = ita_unroll(g, y, mask, theta, k, iters, mu)
    loss, gx, gth = loss_and_grads(g, y, mask, theta, x)
    thb, _ = unroll_backward(g, y, mask, theta, ck, gx, mu)
    return loss, gth + thb, x, ck
