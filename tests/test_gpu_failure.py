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
