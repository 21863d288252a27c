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
