"""Parity cases run by tests/test_gpu_failure.py in a child process that has loaded the
checked build of the library (CSAR_LIB_PATH): small G, M, ITA and autofocus cases against
the FP64 oracle; every plan is checked for a latched device error afterwards."""
import os
import sys

import numpy as np

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
sys.path.insert(0, ROOT)
sys.path.insert(0, os.path.join(ROOT, "tests"))

import synth  # noqa: E402
from gpu_helpers import crand, dev, dev_mask, host  # noqa: E402
from oracle import autofocus as af  # noqa: E402
from oracle import csa, ita, metrics, rda  # noqa: E402
from paper_1302_3120_gb300 import csar  # noqa: E402


def main():
    assert csar.LIB_PATH.endswith("libcsar_checked.so"), csar.LIB_PATH
    rng = np.random.default_rng(7)
    for na, nr in [(256, 256), (1024, 512), (8192, 128)]:
        g = synth.airborne(na, nr)
        x = crand(rng, (na, nr))
        for flags, op in [(0, csa), (csar.PLAN_RDA, rda)]:
            plan = csar.csar_plan_create(g, flags=flags)
            assert metrics.rel_l2(host(csar.csar_G(plan, dev(x))), op.observe_G(g, x)) < 1e-5
            assert metrics.rel_l2(host(csar.csar_M(plan, dev(x))), op.focus_M(g, x)) < 1e-5
            xt = synth.sparse_rayleigh(rng, na, nr, 0.02)
            mask = synth.bernoulli_mask(rng, na, nr, 0.5)
            y = mask * op.observe_G(g, xt)
            K = int(0.02 * na * nr)
            for mode in ("fixed", "niht"):
                x_ref, _ = ita.ita(g, y, mask, K, 3, mu_mode=mode, ops="rda" if flags else "csa")
                X = csar.csar_solve(plan, dev(y), dev_mask(mask), K, 3, mu_mode=mode)
                assert metrics.rel_l2(host(X), x_ref) < 1e-3, (na, nr, flags, mode)
            csar.csar_plan_check(plan)
    # autofocus forward/backward
    import torch
    g = synth.airborne(256, 256)
    xs = synth.sparse_rayleigh(rng, 256, 256, 0.01)
    th_true = synth.theta_sinusoids(rng, 256)
    mask = synth.bernoulli_mask(rng, 256, 256, 0.5)
    y = mask * (np.exp(1j * th_true)[:, None] * csa.observe_G(g, xs))
    theta = (th_true + 0.05 * synth.theta_sinusoids(rng, 256, peak=1.0)).astype(np.float32)
    _, grad_ref, _, _ = af.unrolled_loss_grad(g, y, mask, theta.astype(np.float64), 655, 6)
    plan = csar.csar_plan_create(g)
    th = torch.from_numpy(theta).cuda().requires_grad_(True)
    L = csar.autofocus_loss(plan, dev(y), dev_mask(mask), th, 655, 6)
    L.backward()
    assert metrics.rel_l2(th.grad.double().cpu().numpy(), grad_ref) < 1e-3
    csar.csar_plan_check(plan)
    print("checked build: all cases match")


if __name__ == "__main__":
    main()
