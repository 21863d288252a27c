"""The C ABI: the library loads on a machine without a GPU, exports every
symbol include/gbr.h declares, and rejects bad arguments before touching the
device."""
import ctypes
import os
import re

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.fixture(scope="module")
def lib():
    from paper_2305_00762_gb300 import build, gbr
    build.build()
    return gbr.load()


def declared():
    text = open(os.path.join(ROOT, "include", "gbr.h")).read()
    text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
    return sorted(set(re.findall(r"\b(gbr_\w+)\s*\(", text)))


def test_every_declared_symbol_is_exported(lib):
    names = declared()
    assert "gbr_create" in names and "gbr_step" in names and len(names) >= 14
    for n in names:
        assert hasattr(lib, n), n


def test_error_strings(lib):
    from paper_2305_00762_gb300 import gbr
    for rc in (0, -1, -2, -3, -4, -5, -6, -7):
        assert gbr.error_string(rc)
    assert gbr.error_string(-3).startswith("non-physical")


def test_bad_arguments_rejected_without_device(lib):
    from paper_2305_00762_gb300 import gbr
    out = ctypes.c_void_p()
    ok = gbr.gbr_bc(0, 0, 0, 0, 0.1, 0.1)
    assert lib.gbr_create(5, 64, 1.4, 0.0, 0.72, ctypes.byref(ok), ctypes.byref(out)) == gbr.GBR_ERR_ARG
    assert lib.gbr_create(64, 64, 1.0, 0.0, 0.72, ctypes.byref(ok), ctypes.byref(out)) == gbr.GBR_ERR_ARG
    assert lib.gbr_create(64, 64, 1.4, -1.0, 0.72, ctypes.byref(ok), ctypes.byref(out)) == gbr.GBR_ERR_ARG
    mixed = gbr.gbr_bc(0, 1, 0, 0, 0.1, 0.1)   # periodic must be paired
    assert lib.gbr_create(64, 64, 1.4, 0.0, 0.72, ctypes.byref(mixed), ctypes.byref(out)) == gbr.GBR_ERR_ARG
    neg = gbr.gbr_bc(0, 0, 0, 0, -0.1, 0.1)
    assert lib.gbr_create(64, 64, 1.4, 0.0, 0.72, ctypes.byref(neg), ctypes.byref(out)) == gbr.GBR_ERR_ARG
    assert lib.gbr_step(None, 0.1) == gbr.GBR_ERR_ARG
    assert lib.gbr_destroy(None) == gbr.GBR_OK


def test_degenerate_sizes_and_options_rejected(lib):
    """Empty and oversized grids, unknown boundary kinds and options, and the
    other entry points' argument checks, all before any device call."""
    from paper_2305_00762_gb300 import gbr
    out = ctypes.c_void_p()
    ok = gbr.gbr_bc(1, 1, 1, 1, 0.1, 0.1)
    for nx, ny in ((0, 64), (64, 0), (-3, 64), (5, 5), (1 << 16, 1 << 16)):  # last: > 2^31 cells
        assert lib.gbr_create(nx, ny, 1.4, 0.0, 0.72, ctypes.byref(ok), ctypes.byref(out)) == gbr.GBR_ERR_ARG
    for k in (5, 6, -1):   # GBR_BC_FIXED only inside a gbr_side; 6, -1 unknown
        bad = gbr.gbr_bc(k, 1, 1, 1, 0.1, 0.1)
        assert lib.gbr_create(64, 64, 1.4, 0.0, 0.72, ctypes.byref(bad), ctypes.byref(out)) == gbr.GBR_ERR_ARG
    assert lib.gbr_create(64, 64, 1.4, 0.0, 0.0, ctypes.byref(ok), ctypes.byref(out)) == gbr.GBR_ERR_ARG
    assert lib.gbr_create(64, 64, 1.4, 0.0, 0.72, None, ctypes.byref(out)) == gbr.GBR_ERR_ARG
    assert lib.gbr_set_option(None, gbr.GBR_OPT_PRECISION, ctypes.c_double(32.0)) == gbr.GBR_ERR_ARG
    assert lib.gbr_residual(None, None, 0) == gbr.GBR_ERR_ARG
    assert lib.gbr_step_cfl(None, ctypes.c_double(0.5), ctypes.c_double(1.0)) == gbr.GBR_ERR_ARG
    assert lib.gbr_set_sensor_weights(None, None, 0) == gbr.GBR_ERR_ARG
    assert lib.gbr_set_side(None, 0, None) == gbr.GBR_ERR_ARG
    # batches: no grids, a grid below the ghost width
    nx = (ctypes.c_int * 1)(5)
    ny = (ctypes.c_int * 1)(64)
    d = (ctypes.c_double * 1)(0.1)
    bcs = (ctypes.c_int * 4)(1, 1, 1, 1)
    bout = ctypes.c_void_p()
    assert lib.gbr_batch_create(0, nx, ny, d, d, bcs, ctypes.c_double(1.4), ctypes.byref(bout)) == gbr.GBR_ERR_ARG
    assert lib.gbr_batch_create(1, nx, ny, d, d, bcs, ctypes.c_double(1.4), ctypes.byref(bout)) == gbr.GBR_ERR_ARG
    # the allocation-free step: a grid larger than its fixed scratch
    big = gbr.gbr_bc(1, 1, 1, 1, 0.1, 0.1)
    assert lib.gbr_step_static(ctypes.c_void_p(16), ctypes.c_void_p(16), 4096, 4096, ctypes.c_double(1.4),
                               ctypes.c_double(0.0), ctypes.c_double(0.72), ctypes.byref(big),
                               ctypes.c_double(1e-3), None) == gbr.GBR_ERR_ARG


def test_fma_probe_library_exports_its_entry():
    """The benchmark's FMA-throughput probe is its own library; it builds and
    exports gbr_probe_fma_gflops (no compute without a GPU)."""
    import ctypes
    from paper_2305_00762_gb300 import build as B
    B.build()
    L = ctypes.CDLL(B.PROBE_LIB)
    assert hasattr(L, "gbr_probe_fma_gflops")
