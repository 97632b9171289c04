"""Batched ITA over patches of uneven size (spec batching row): one graph launch
per iteration, holding one launch per pass over a work table of every patch when all
sizes are served by the batched kernels (512 to 4096 per axis), else one branch per
patch, gives the same images as the per-patch loop, matches the oracle, and the
autotuner picks a working column configuration."""
import numpy as np
import pytest

import synth
from gpu_helpers import dev, dev_mask, host, lib
from oracle import csa, ita, metrics

pytestmark = pytest.mark.gpu


def _patches(seed, count, sizes):
    rng = np.random.default_rng(seed)
    shapes = synth.batch_shapes(rng, count, sizes)
    out = []
    for na, nr in shapes:
        g = synth.airborne(na, nr)
        x = synth.sparse_rayleigh(rng, na, nr, 0.01)
        mask = synth.bernoulli_mask(rng, na, nr, 0.5)
        out.append((g, x, mask))
    return out


def test_batched_equals_per_patch_loop_and_oracle():
    csar = lib()
    pts = _patches(3, 6, (256, 512, 1024))
    geoms = [p[0] for p in pts]
    Ys, Ms, Ks, ys = [], [], [], []
    for g, x, mask in pts:
        plan = csar.csar_plan_create(g)
        yd = csar.csar_G(plan, dev(x))
        y = host(yd) * mask
        ys.append(y)
        Ys.append(dev(y))
        Ms.append(dev_mask(mask))
        Ks.append(int(round(0.01 * g.n_az * g.n_rg)))
    iters = 12
    batch = csar.csar_batch_create(geoms)
    Xb = csar.csar_solve_batched(batch, Ys, Ms, Ks, iters)
    csar.csar_batch_check(batch)
    for i, (g, x, mask) in enumerate(pts):
        plan = csar.csar_plan_create(g)
        Xl = csar.csar_solve(plan, Ys[i], Ms[i], Ks[i], iters)
        assert np.array_equal(host(Xb[i]), host(Xl))
    g, x, mask = pts[0]
    x_ref, _ = ita.ita(g, ys[0], mask, Ks[0], iters)
    assert metrics.rel_l2(host(Xb[0]), x_ref) < 1e-3
    # a second solve on the same batch reuses the captured graphs
    Xb2 = csar.csar_solve_batched(batch, Ys, Ms, Ks, iters)
    assert all(np.array_equal(host(a), host(b)) for a, b in zip(Xb, Xb2))


def test_autotune_and_forced_cluster_sizes():
    csar = lib()
    g = synth.airborne(4096, 512)
    p = csar.csar_autotune(g, iters=3)
    assert p in (1, 2, 4, 8)
    rng = np.random.default_rng(4)
    x = synth.sparse_rayleigh(rng, 4096, 512, 0.01)
    ref = csa.observe_G(g, x)
    for q in (1, 2, 4, 8):
        plan = csar.csar_plan_create(g, flags=csar.plan_col_cluster(q))
        assert metrics.rel_l2(host(csar.csar_G(plan, dev(x))), ref) < 1e-5


def test_batched_real_patch_mix():
    """The batched workload's own mix: 64 patches with each axis drawn from {512, 1024,
    2048, 4096} (seeded), 1% Rayleigh scenes, 50% masks, K_p = 1% of each patch, 6
    iterations.  Every patch's image is bit-identical to the per-patch loop's, and the
    smallest patch of every azimuth size class is checked against the FP64 oracle (its
    echo formed by the oracle's G; the other patches' echoes by the library's G)."""
    import torch
    csar = lib()
    rng = np.random.default_rng(2024)
    shapes = synth.batch_shapes(rng, 64)
    assert len({a for a, _ in shapes}) == 4
    checked = {}
    for i, (a, r) in enumerate(shapes):
        if a not in checked or a * r < shapes[checked[a]][0] * shapes[checked[a]][1]:
            checked[a] = i
    geoms, Ys, Ms, Ks, host_y, masks = [], [], [], [], {}, {}
    for i, (a, r) in enumerate(shapes):
        g = synth.airborne(a, r)
        x = synth.sparse_rayleigh(rng, a, r, 0.01)
        mask = synth.bernoulli_mask(rng, a, r, 0.5)
        if i in checked.values():
            y = mask * csa.observe_G(g, x)
            host_y[i], masks[i] = y, mask
            Ys.append(dev(y))
        else:
            plan = csar.csar_plan_create(g)
            Ys.append(csar.csar_G(plan, dev(x)) * dev_mask_float(mask))
            plan.close()
        geoms.append(g)
        Ms.append(dev_mask(mask))
        Ks.append(int(round(0.01 * a * r)))
    iters = 6
    batch = csar.csar_batch_create(geoms)
    Xb = csar.csar_solve_batched(batch, Ys, Ms, Ks, iters)
    csar.csar_batch_check(batch)
    # every size is served by the batched kernels: one launch per pass, and each patch's
    # image equals that of a plan configured as a batch member
    for i, g in enumerate(geoms):
        plan = csar.csar_plan_create(g, flags=csar.PLAN_BATCH_MEMBER)
        Xl = csar.csar_solve(plan, Ys[i], Ms[i], Ks[i], iters)
        assert torch.equal(Xb[i], Xl), i
        plan.close()
    # a second solve on the same batch replays the captured graphs
    Xb2 = csar.csar_solve_batched(batch, Ys, Ms, Ks, iters)
    assert all(torch.equal(a, b) for a, b in zip(Xb, Xb2))
    for i in checked.values():
        g = geoms[i]
        x_ref, _ = ita.ita(g, host_y[i], masks[i], Ks[i], iters)
        assert metrics.rel_l2(host(Xb[i]), x_ref) < 1e-3, shapes[i]


def dev_mask_float(mask):
    """The sampling mask as a complex64 CUDA tensor of 0/1 (zero-fills an echo)."""
    import torch
    return torch.from_numpy(mask.astype(np.complex64)).cuda()


@pytest.mark.parametrize("mu_mode", ["fixed", "niht"])
def test_batched_repass_and_selection_paths(mu_mode):
    """Patches whose threshold falls sharply between iterations (noiseless bright targets,
    95% and 80% sampling): the per-patch re-passes and the grid-wide selection run inside
    the batched launches (fixed step), or the per-patch branches run (NIHT step); every
    image equals that of a batch-member plan solved alone, and one patch of each matches
    the FP64 oracle."""
    import torch
    csar = lib()
    rng = np.random.default_rng(17)
    geoms, Ys, Ms, Ks, hosts = [], [], [], [], []
    for na, nr, rate, k in [(512, 512, 0.95, 60), (1024, 512, 0.8, 30), (512, 1024, 0.95, 90)]:
        g = synth.airborne(na, nr)
        x = np.zeros((na, nr), complex)
        idx = rng.choice(na * nr, k, replace=False)
        x.flat[idx] = 10 * np.exp(2j * np.pi * rng.random(k))
        mask = synth.bernoulli_mask(rng, na, nr, rate)
        y = mask * csa.observe_G(g, x)
        geoms.append(g)
        Ys.append(dev(y))
        Ms.append(dev_mask(mask))
        Ks.append(k)
        hosts.append((y, mask))
    iters = 4
    batch = csar.csar_batch_create(geoms)
    Xb = csar.csar_solve_batched(batch, Ys, Ms, Ks, iters, mu_mode=mu_mode)
    csar.csar_batch_check(batch)
    for i, g in enumerate(geoms):
        plan = csar.csar_plan_create(g, flags=csar.PLAN_BATCH_MEMBER)
        Xl = csar.csar_solve(plan, Ys[i], Ms[i], Ks[i], iters, mu_mode=mu_mode)
        assert torch.equal(Xb[i], Xl), i
        plan.close()
    y, mask = hosts[0]
    x_ref, _ = ita.ita(geoms[0], y, mask, Ks[0], iters, mu_mode=mu_mode)
    assert metrics.rel_l2(host(Xb[0]), x_ref) < 1e-3
