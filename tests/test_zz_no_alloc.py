"""csar_G_noalloc: G for callers that cannot allocate device memory (no plan; tables in
a static device array).  Checked against the plan-based csar_G on two calls in a row,
through the C ABI.  Collected last so that a stop-at-first-failure run has already run
every other test."""
import ctypes

import numpy as np
import pytest

import synth
from gpu_helpers import crand, dev, host, lib
from oracle import metrics

pytestmark = pytest.mark.gpu


def test_noalloc_G_matches_plan_G_on_consecutive_calls():
    import torch
    csar = lib()
    rng = np.random.default_rng(21)
    cases = [synth.spaceborne(2048, 1024), synth.airborne(512, 4096)]
    for g in cases:                     # two calls in a row, different geometries
        x = dev(crand(rng, (g.n_az, g.n_rg)))
        y_ref = csar.csar_G(csar.csar_plan_create(g), x)
        p = csar.params_of(g)
        y = torch.empty_like(x)
        st = csar.lib.csar_G_noalloc(ctypes.byref(p), ctypes.c_void_p(x.data_ptr()),
                                     ctypes.c_void_p(y.data_ptr()),
                                     ctypes.c_void_p(torch.cuda.current_stream().cuda_stream))
        assert st == 0, csar.lib.csar_last_error().decode()
        torch.cuda.synchronize()
        assert metrics.rel_l2(host(y), host(y_ref)) < 1e-5
    # in place, and the size limit is enforced with a clear error
    x = dev(crand(rng, (256, 256)))
    g = synth.airborne(256, 256)
    ref = csar.csar_G(csar.csar_plan_create(g), x)
    csar.csar_G_noalloc(g, x, x)
    torch.cuda.synchronize()
    assert metrics.rel_l2(host(x), host(ref)) < 1e-5
    # beyond the maximum size: rejected on the host, before any device access
    big = csar.params_of(synth.airborne(16384, 16))
    st = csar.lib.csar_G_noalloc(ctypes.byref(big), ctypes.c_void_p(x.data_ptr()),
                                 ctypes.c_void_p(x.data_ptr()), None)
    assert st != 0 and "8192" in csar.lib.csar_last_error().decode()
