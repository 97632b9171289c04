"""Writes the stored oracle results of the long ITA runs (FP64, CPU).

Runs the FP64 oracle (``oracle/``) on seeded inputs from ``synth`` only; nothing here
touches the CUDA path.  Each output ``.npz`` holds, for the final iterate X^(I) of
Algorithm 1 (Eq. (25)):

  idx, val        flat indices and values (complex64) of the nonzeros of X^(I)
  band            flat indices with | |b| - sigma | <= 1e-4 sigma at the last iteration
                  (b = X^(I-1) + mu Delta X), where the support may differ
  sigma, resid_sq per-iteration sigma_i = |b|_(K+1) and ||S.(Y - G X^(i))||^2
  shape, K, iters the workload

Workloads (inputs re-created by the tests from the same seeds):
  config2_r30, config2_r50  2048^2 airborne, 1% Rayleigh scene, G(X) + 20 dB noise,
                            Bernoulli 30% / 50%, K = 41943, 200 iterations
  config3_it20              8192^2 spaceborne, 2000 3x3 targets over -25 dB clutter,
                            Bernoulli 40%, K = 20000, 20 iterations
  config5_af50              4096^2 airborne autofocus: 0.5% scene, 50% sampling, theta =
                            3 sinusoids (peak 2 pi) plus a seeded error, K = 83886,
                            50-iteration soft-threshold unroll.  Holds instead the loss,
                            dL/dtheta (direct + through the unroll), the adjoint of X^(0)
                            at 65536 seeded positions and at the 4096 largest, its norm,
                            and the final iterate's nonzero count.

Usage: python tests/golden/make_ita_goldens.py [config2_r30 config2_r50 config3_it20 config5_af50]
"""
from __future__ import annotations

import os
import sys
import time

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(os.path.dirname(HERE))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

import synth  # noqa: E402
from oracle import autofocus as af  # noqa: E402
from oracle import csa, echo, ita  # noqa: E402

BAND = 1e-4


def config2_inputs(rate: float):
    """2048^2 precision-study echo and mask (seed 2)."""
    na = nr = 2048
    g = synth.airborne(na, nr)
    rng = np.random.default_rng(2)
    x = synth.sparse_rayleigh(rng, na, nr, 0.01)
    y_clean = csa.observe_G(g, x)
    y = echo.add_noise(synth.cn_noise(rng, y_clean.shape), y_clean, 20.0)
    mask = synth.bernoulli_mask(rng, na, nr, rate)
    return g, mask * y, mask


def config3_inputs():
    """8192^2 spaceborne echo and mask (seed 0): Y = S . G(X), no added noise."""
    g = synth.spaceborne(8192, 8192)
    rng = np.random.default_rng(0)
    x = synth.targets_over_clutter(rng, 8192, 8192)
    mask = synth.bernoulli_mask(rng, 8192, 8192, 0.4)
    y = csa.observe_G(g, x)
    del x
    y *= mask
    return g, y, mask


def config5_inputs():
    """4096^2 autofocus workload (seed 5): the echo S . exp(j theta_true) G(X) as the
    GPU receives it (complex64), and the estimate theta (float32) the gradient is
    taken at."""
    na = nr = 4096
    g = synth.airborne(na, nr)
    rng = np.random.default_rng(5)
    x = synth.sparse_rayleigh(rng, na, nr, 0.005).astype(np.complex64)
    theta_true = synth.theta_sinusoids(rng, na)
    mask = synth.bernoulli_mask(rng, na, nr, 0.5)
    theta = theta_true + 0.02 * synth.theta_sinusoids(rng, na, peak=1.0)
    y = mask * (np.exp(1j * theta_true)[:, None] * csa.observe_G(g, x))
    return g, y.astype(np.complex64), mask, theta.astype(np.float32)


def x0bar_positions(n: int) -> np.ndarray:
    """Seeded positions at which the adjoint of X^(0) is stored."""
    return np.sort(np.random.default_rng(77).choice(n, 65536, replace=False)).astype(np.int64)


def run_autofocus(out: str) -> None:
    t0 = time.time()
    g, y, mask, theta = config5_inputs()
    K, iters = 83886, 50
    y64 = y.astype(np.complex128)
    th64 = theta.astype(np.float64)
    x, ck = af.ita_unroll(g, y64, mask, th64, K, iters)
    loss, gx, gth = af.loss_and_grads(g, y64, mask, th64, x)
    thb, x0bar = af.unroll_backward(g, y64, mask, th64, ck, gx)
    del ck
    flat = x0bar.reshape(-1)
    pos = x0bar_positions(flat.size)
    top = np.argsort(-np.abs(flat))[:4096].astype(np.int64)
    np.savez_compressed(
        out, loss=np.array(loss), grad_theta=gth + thb, grad_theta_direct=gth,
        x0bar_pos=pos, x0bar_at_pos=flat[pos], x0bar_top=top, x0bar_at_top=flat[top],
        x0bar_norm=np.array(np.linalg.norm(flat)), nnz=np.array(np.count_nonzero(x)),
        K=np.array(K), iters=np.array(iters))
    print(f"{os.path.basename(out)}: loss {loss:.6e}, {time.time() - t0:.0f} s")


def run(g, y, mask, K: int, iters: int, out: str) -> None:
    t0 = time.time()
    x, st = ita.ita(g, y, mask, K, iters - 1)
    x, last, b = ita.ita_iteration(g, y, np.asarray(mask, dtype=np.float64), x, K, return_b=True)
    st.append(last)
    flat = x.reshape(-1)
    idx = np.flatnonzero(flat).astype(np.int32)
    band = np.flatnonzero(np.abs(np.abs(b.reshape(-1)) - last.sigma) <= BAND * last.sigma)
    np.savez_compressed(
        out, idx=idx, val=flat[idx].astype(np.complex64), band=band.astype(np.int32),
        sigma=np.array([s.sigma for s in st]), resid_sq=np.array([s.resid_sq for s in st]),
        shape=np.array(x.shape), K=np.array(K), iters=np.array(iters))
    print(f"{os.path.basename(out)}: {len(idx)} nonzeros, {len(band)} in the band, "
          f"{time.time() - t0:.0f} s")


def main(names) -> None:
    for name in names:
        out = os.path.join(HERE, name + ".npz")
        if name == "config2_r30":
            run(*config2_inputs(0.3), 41943, 200, out)
        elif name == "config2_r50":
            run(*config2_inputs(0.5), 41943, 200, out)
        elif name == "config3_it20":
            run(*config3_inputs(), 20000, 20, out)
        elif name == "config5_af50":
            run_autofocus(out)
        else:
            raise SystemExit(f"unknown workload {name}")


if __name__ == "__main__":
    main(sys.argv[1:] or ["config2_r30", "config2_r50", "config3_it20", "config5_af50"])
