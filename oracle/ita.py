"""Thresholding, the K-th magnitude rule and the iterative thresholding algorithm (FP64).

TEST INFRASTRUCTURE ONLY (see ``oracle/__init__``).

Algorithm 1 / Eq. (25): starting from X^(0) = 0, each iteration forms the residue
R = S . (Y - G(X)) (the sampling operators Theta_eta, Theta_tau of Eq. (24)
generalised to a 2-D mask S applied to a zero-filled echo), applies the matched
filter to it, Delta X = M(R), and thresholds X + mu Delta X.  Section IV-B sets the
threshold from the (K+1)-th largest magnitude of b = X + mu Delta X
(lambda_i mu_i = |b|_(K+1)) and the step either fixed or adaptively (NIHT).

The operator pair is a module with ``observe_G`` and ``focus_M``: the chirp-scaling
pair (``csa``, the default) or the range-Doppler pair of Section III-C (``rda``; with
it Algorithm 1 is the paper's CS-RDA).
"""
from __future__ import annotations

import dataclasses

import numpy as np

from . import csa, rda

_OPS = {"csa": csa, "rda": rda}


# ----------------------------------------------------------------------------- thresholds

def soft_threshold(b: np.ndarray, sigma: float) -> np.ndarray:
    """Complex soft thresholding e_{1,sigma} (Eq. (9)) with sgn(b) = b/|b|:
    b (1 - sigma/|b|) where |b| > sigma, else 0.  (Eq. (9) prints '>=';
    the value at |b| = sigma is 0 either way.)"""
    b = np.asarray(b, dtype=np.complex128)
    mag = np.abs(b)
    out = np.zeros_like(b)
    keep = mag > sigma
    out[keep] = b[keep] * (1.0 - sigma / mag[keep])
    return out


def half_lambda_mu(sigma: float) -> float:
    """lambda*mu for which the half-threshold jump point (54^(1/3)/4)(lambda mu)^(2/3)
    equals sigma: lambda mu = (sqrt(96)/9) sigma^(3/2)."""
    return np.sqrt(96.0) / 9.0 * float(sigma) ** 1.5


def half_threshold(b: np.ndarray, sigma: float) -> np.ndarray:
    """Complex half thresholding (q = 1/2, named as analytic in Section II-B; the
    closed form is that of the L_1/2 regulariser of the paper's reference [Xu2010]):
    the global minimiser of |x - b|^2 + lambda mu |x|^(1/2), taken along the phase of b.
    With t = (54^(1/3)/4)(lambda mu)^(2/3) = sigma:
      x = (b/|b|) (2/3)|b| (1 + cos(2 pi/3 - (2/3) phi)),
      phi = arccos((lambda mu / 8) (|b|/3)^(-3/2))      for |b| > t, else 0."""
    b = np.asarray(b, dtype=np.complex128)
    lm = half_lambda_mu(sigma)
    mag = np.abs(b)
    out = np.zeros_like(b)
    keep = mag > sigma
    m = mag[keep]
    arg = np.clip((lm / 8.0) * (m / 3.0) ** -1.5, -1.0, 1.0)
    phi = np.arccos(arg)
    shrunk = (2.0 / 3.0) * m * (1.0 + np.cos(2.0 * np.pi / 3.0 - (2.0 / 3.0) * phi))
    out[keep] = b[keep] / m * shrunk
    return out


def hard_threshold(b: np.ndarray, sigma: float) -> np.ndarray:
    """Hard thresholding (q = 0, Section II-B): the global minimiser of
    |x - b|^2 + lambda mu [x != 0] with lambda mu = sigma^2 keeps b where |b| > sigma
    and is 0 elsewhere (cost sigma^2 against |b|^2)."""
    b = np.asarray(b, dtype=np.complex128)
    return np.where(np.abs(b) > sigma, b, 0)


def threshold(b: np.ndarray, sigma: float, kind: str) -> np.ndarray:
    if kind == "soft":
        return soft_threshold(b, sigma)
    if kind == "half":
        return half_threshold(b, sigma)
    if kind == "hard":
        return hard_threshold(b, sigma)
    raise ValueError(kind)


def kth_largest_magnitude(b: np.ndarray, k: int) -> float:
    """|b|_(k+1): the (k+1)-th largest magnitude (Section IV-B, lambda_i rule);
    0 when k >= number of elements."""
    mag = np.abs(np.asarray(b)).reshape(-1)
    if k >= mag.size:
        return 0.0
    return float(np.sort(mag)[::-1][k])


def top_k_support(v: np.ndarray, k: int) -> np.ndarray:
    """Boolean mask of the k largest magnitudes of v (ties broken by index)."""
    flat = np.abs(np.asarray(v)).reshape(-1)
    k = min(int(k), flat.size)
    order = np.argsort(-flat, kind="stable")[:k]
    sel = np.zeros(flat.size, dtype=bool)
    sel[order] = True
    return sel.reshape(np.shape(v))


# ----------------------------------------------------------------------------- ITA

@dataclasses.dataclass
class IterStats:
    resid_sq: float      # ||S . (Y - G(X^(i)))||^2
    mu: float            # step mu_i
    sigma: float         # lambda_i mu_i = |b|_(K+1)
    nnz: int             # nonzeros of X^(i+1)


def niht_step(g, mask: np.ndarray, dx: np.ndarray, support: np.ndarray, ops: str = "csa") -> float:
    """Adaptive step of Section IV-B (the NIHT rule of [Blumensath2010]):
    mu_i = ||Delta X_Gamma||^2 / ||S . G(Delta X_Gamma)||^2, where Delta X_Gamma is
    Delta X restricted to Gamma.  Eq. (27) prints the reciprocal ratio; this is the
    reading under which mu_i^{-1} <= ||S G||^2 as Eq. (26) requires."""
    dg = np.where(support, dx, 0)
    num = float(np.vdot(dg, dg).real)
    if num == 0.0:
        return 1.0
    den_v = mask * _OPS[ops].observe_G(g, dg)
    den = float(np.vdot(den_v, den_v).real)
    return num / den if den > 0.0 else 1.0


def ita_iteration(g, y: np.ndarray, mask: np.ndarray, x: np.ndarray, k: int,
                  mu_mode: str = "fixed", mu: float = 1.0, kind: str = "soft",
                  return_b: bool = False, ops: str = "csa"):
    """One iteration of Algorithm 1 in the paper's order.  Returns (X^(i+1), stats),
    plus b = X + mu Delta X when return_b."""
    op = _OPS[ops]
    r = mask * (y - op.observe_G(g, x))                       # residue
    dx = op.focus_M(g, r)                                     # MF on residue
    if mu_mode == "niht":
        support = x != 0
        if not support.any():
            support = top_k_support(dx, k)
        mu_i = niht_step(g, mask, dx, support, ops)
    else:
        mu_i = float(mu)
    b = x + mu_i * dx                                         # gradient step
    sigma = kth_largest_magnitude(b, k)                       # lambda_i mu_i
    x_new = threshold(b, sigma, kind)                         # thresholding
    st = IterStats(float(np.vdot(r, r).real), mu_i, sigma, int(np.count_nonzero(x_new)))
    return (x_new, st, b) if return_b else (x_new, st)


def ita(g, y: np.ndarray, mask: np.ndarray, k: int, iters: int, mu_mode: str = "fixed",
        mu: float = 1.0, kind: str = "soft", x0: np.ndarray | None = None, ops: str = "csa"):
    """Algorithm 1: exactly ``iters`` iterations from X^(0) = 0 (or x0).
    Returns (X^(iters), [IterStats])."""
    x = (np.zeros((g.n_az, g.n_rg), dtype=np.complex128) if x0 is None
         else np.asarray(x0, dtype=np.complex128).copy())
    mask = np.asarray(mask, dtype=np.float64)
    y = np.asarray(y, dtype=np.complex128)
    stats = []
    for _ in range(iters):
        x, st = ita_iteration(g, y, mask, x, k, mu_mode, mu, kind, ops=ops)
        stats.append(st)
    return x, stats
