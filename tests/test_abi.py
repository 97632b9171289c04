"""The C-ABI library builds for sm_103a, loads, and exports every entry point that
include/csar.h declares (no GPU needed: no compute call is made)."""
import ctypes
import os
import re

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
HEADER = os.path.join(ROOT, "include", "csar.h")


def declared_symbols():
    text = open(HEADER).read()
    text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
    return sorted(set(re.findall(r"\b(csar_[A-Za-z_0-9]+)\s*\(", text)))


def test_header_declares_the_boundary():
    syms = declared_symbols()
    for s in ("csar_plan_create", "csar_plan_destroy", "csar_G", "csar_M", "csar_ita_step",
              "csar_solve", "csar_solve_host", "csar_plan_check", "csar_last_error"):
        assert s in syms


def test_library_exports_every_declared_symbol():
    from paper_1302_3120_gb300 import build
    path = build.build()
    lib = ctypes.CDLL(path)
    for s in declared_symbols():
        assert hasattr(lib, s), s
    from paper_1302_3120_gb300 import csar
    assert csar.csar_version() >= 10000
    for s in csar.EXPORTS:
        assert s in declared_symbols()


def test_invalid_arguments_rejected_on_host():
    """Parameter validation happens before any CUDA call, so it runs without a GPU."""
    import synth
    from paper_1302_3120_gb300 import csar
    bad = synth.airborne(100, 256)          # not a power of two
    try:
        csar.csar_plan_create(bad)
    except csar.CsarError as e:
        assert e.status == 1 and "power of two" in str(e)
    else:
        raise AssertionError("plan accepted n_az = 100")
    neg = synth.Geometry(64, 64, -0.03, 150.0, 10e3, 200.0, 60e6, 1e-6, 72e6, 2.0)
    try:
        csar.csar_plan_create(neg)
    except csar.CsarError as e:
        assert e.status == 1 and "wavelength" in str(e)
    else:
        raise AssertionError("plan accepted a negative wavelength")
    p = csar.params_of(synth.airborne(64, 64))
    h = ctypes.c_void_p()
    assert csar.lib.csar_plan_create(ctypes.byref(p), 7, ctypes.byref(h)) == 1
    assert h.value is None
    assert csar.lib.csar_plan_create(None, 0, ctypes.byref(h)) == 1


def test_echo_simulator_and_tile_flags_rejected_on_host():
    """Host-side validation of the echo simulator and of the plan's column-tile flags
    (no CUDA call is reached)."""
    import dataclasses
    import numpy as np
    import synth
    from paper_1302_3120_gb300 import csar
    g = synth.airborne(64, 64)
    p = csar.params_of(g)
    rows = np.array([64], np.int32)          # off the grid
    cols = np.array([0], np.int32)
    amp = np.array([1.0, 0.0], np.float32)
    fake = ctypes.c_void_p(16)               # never dereferenced: validation fails first
    st = csar.lib.csar_echo_points(ctypes.byref(p), rows.ctypes.data, cols.ctypes.data,
                                   amp.ctypes.data, 1, fake, 0, None)
    assert st == 1 and "off the grid" in csar.lib.csar_last_error().decode()
    p0 = csar.params_of(dataclasses.replace(g, antenna_len=0.0))
    rows[0] = 10
    st = csar.lib.csar_echo_points(ctypes.byref(p0), rows.ctypes.data, cols.ctypes.data,
                                   amp.ctypes.data, 1, fake, 0, None)
    assert st == 1 and "antenna_len" in csar.lib.csar_last_error().decode()
    st = csar.lib.csar_echo_points(ctypes.byref(p), rows.ctypes.data, cols.ctypes.data,
                                   amp.ctypes.data, -1, fake, 0, None)
    assert st == 1
    h = ctypes.c_void_p()
    both = csar.PLAN_COL_HALF_TILE | csar.PLAN_COL_WIDE_TILE
    assert csar.lib.csar_plan_create(ctypes.byref(p), both, ctypes.byref(h)) == 2
    assert h.value is None


def test_rda_plan_checks_on_host():
    """A range-Doppler plan's tables are checked before any CUDA call: a migration
    slope above 1/2 (edge Doppler at 0.8 of 2V/lambda) or a Doppler beyond 2V/lambda is
    refused (CSAR_E_UNSUPPORTED) without a GPU."""
    import dataclasses
    import synth
    from paper_1302_3120_gb300 import csar
    for frac in (0.8, 1.2):
        g = dataclasses.replace(synth.airborne(64, 64), prf=frac * 4 * 150.0 / 0.03)
        p = csar.params_of(g)
        h = ctypes.c_void_p()
        assert csar.lib.csar_plan_create(ctypes.byref(p), csar.PLAN_RDA, ctypes.byref(h)) == 2
        assert h.value is None
        msg = csar.lib.csar_last_error().decode()
        assert ("slope" in msg) or ("Doppler" in msg) or ("phase" in msg), msg


def test_batch_member_flag_checked_on_host():
    """CSAR_PLAN_BATCH_MEMBER: sizes the one-launch-per-pass batch kernels do not serve
    are refused (CSAR_E_UNSUPPORTED), and so is the flag with another column flag
    (CSAR_E_INVALID), before any CUDA call."""
    import synth
    from paper_1302_3120_gb300 import csar
    h = ctypes.c_void_p()
    for na, nr in [(256, 512), (512, 8192), (8192, 1024)]:
        p = csar.params_of(synth.airborne(na, nr))
        assert csar.lib.csar_plan_create(ctypes.byref(p), csar.PLAN_BATCH_MEMBER, ctypes.byref(h)) == 2
        assert h.value is None and "batch member" in csar.lib.csar_last_error().decode()
    p = csar.params_of(synth.airborne(1024, 1024))
    for other in (csar.PLAN_COL_HALF_TILE, csar.plan_col_cluster(2), csar.PLAN_RDA, csar.PLAN_COL_PERSIST):
        assert csar.lib.csar_plan_create(ctypes.byref(p), csar.PLAN_BATCH_MEMBER | other, ctypes.byref(h)) == 1
        assert h.value is None
