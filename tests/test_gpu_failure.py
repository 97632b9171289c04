"""Failure detection on the GPU without a fault: the bounded wait of the column-pass
cluster exchanges runs out on an mbarrier that nothing arrives at, the kernel returns with
a timeout status that the host reads, and the context stays usable."""
import numpy as np
import pytest

import synth
from gpu_helpers import crand, dev, host, lib
from oracle import csa, metrics

pytestmark = pytest.mark.gpu


def test_bounded_wait_times_out_and_context_survives():
    import time
    csar = lib()
    t0 = time.perf_counter()
    st = csar.csar_selftest_wait_timeout(20)
    dt = time.perf_counter() - t0
    assert st == 5, csar.lib.csar_last_error().decode()
    assert dt < 5.0
    # the device still runs the library's kernels correctly afterwards
    g = synth.airborne(256, 256)
    plan = csar.csar_plan_create(g)
    x = crand(np.random.default_rng(1), (256, 256))
    assert metrics.rel_l2(host(csar.csar_G(plan, dev(x))), csa.observe_G(g, x)) < 1e-5
    csar.csar_plan_check(plan)


def test_injected_allocation_failures_are_reported_without_leaks():
    """Host-side fault injection of the out-of-memory paths (csar_debug_fail_alloc):
    for every device allocation of plan creation in turn, creation fails with
    CSAR_E_OOM and leaves the device's free memory where it was; the lazily allocated
    workspaces (host-buffer staging, autofocus checkpoints, candidate growth) report
    CSAR_E_OOM the same way, and the next call succeeds and computes correctly."""
    import torch
    csar = lib()
    g = synth.airborne(1024, 1024)
    csar.csar_plan_create(g).close()     # loads the kernels this geometry uses
    torch.cuda.synchronize()
    free0 = torch.cuda.mem_get_info()[0]
    n = 1
    try:
        while True:
            csar.csar_debug_fail_alloc(n)
            try:
                plan = csar.csar_plan_create(g)
            except csar.CsarError as e:
                assert e.status == 3, e
                n += 1
                assert n < 200
                continue
            break
    finally:
        csar.csar_debug_fail_alloc(0)
    assert n > 10                        # every allocation of plan creation was hit once
    plan.close()
    torch.cuda.synchronize()
    assert abs(torch.cuda.mem_get_info()[0] - free0) < 4 * 2 ** 20
    plan = csar.csar_plan_create(g)
    rng = np.random.default_rng(2)
    x = synth.sparse_rayleigh(rng, 1024, 1024, 0.01)
    mask = synth.bernoulli_mask(rng, 1024, 1024, 0.5)
    y = (mask * csa.observe_G(g, x)).astype(np.complex64)
    bits = synth.pack_mask(mask)
    K = 10486
    for first in (1, 2, 3):             # each staging allocation fails once in turn
        csar.csar_debug_fail_alloc(first)
        try:
            with pytest.raises(csar.CsarError) as e:
                csar.csar_solve_host(plan, y, bits, K, 3)
            assert e.value.status == 3
        finally:
            csar.csar_debug_fail_alloc(0)
    xh = csar.csar_solve_host(plan, y, bits, K, 3)
    from oracle import ita
    x_ref, _ = ita.ita(g, y.astype(np.complex128), mask, K, 3)
    assert metrics.rel_l2(xh.reshape(1024, 1024).astype(np.complex128), x_ref) < 1e-3
    theta = torch.zeros(1024, dtype=torch.float32, device="cuda")
    csar.csar_debug_fail_alloc(2)
    try:
        with pytest.raises(csar.CsarError) as e:
            csar.csar_af_solve(plan, dev(y), torch.from_numpy(bits.view(np.int32)).cuda(), theta, K, 3)
        assert e.value.status == 3
    finally:
        csar.csar_debug_fail_alloc(0)
    csar.csar_af_solve(plan, dev(y), torch.from_numpy(bits.view(np.int32)).cuda(), theta, K, 3)
    csar.csar_plan_check(plan)


def test_checked_build_runs_the_parity_cases_without_index_faults():
    """The checked build (every guarded global index compared with its array's extent;
    an index out of range would be skipped and reported as CSAR_E_INTERNAL) runs small
    parity cases of G, M, the ITA (fixed and NIHT, both operator pairs) and the
    autofocus backward against the oracle, in a child process that loads it."""
    import os
    import subprocess
    import sys
    root = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
    r = subprocess.run([sys.executable, "-c",
                        "from paper_1302_3120_gb300 import build; print(build.build_checked())"],
                       cwd=root, capture_output=True, text=True, timeout=1200)
    assert r.returncode == 0, r.stderr[-2000:]
    env = dict(os.environ, CSAR_LIB_PATH=r.stdout.strip().splitlines()[-1])
    r = subprocess.run([sys.executable, os.path.join(root, "tests", "checked_cases.py")], cwd=root, env=env,
                       capture_output=True, text=True, timeout=1200)
    assert r.returncode == 0, (r.stdout[-2000:], r.stderr[-2000:])
    assert "checked build: all cases match" in r.stdout
