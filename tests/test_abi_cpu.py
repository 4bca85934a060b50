"""Host-side checks of the C-ABI library that need no GPU: it loads, it
exports every entry point that include/*.h declares, and its argument
checks fail cleanly (status + message, no crash) without a device."""
import ctypes
import glob
import os
import re

import numpy as np
import pytest

from paper_2001_01473_gb300 import an5d, inputs

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def declared_functions():
    names = []
    for h in glob.glob(os.path.join(ROOT, "include", "*.h")):
        src = open(h).read()
        src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
        src = re.sub(r"//[^\n]*", "", src)
        names += re.findall(r"\b(an5d_\w+)\s*\(", src)
    return sorted(set(names))


@pytest.fixture(scope="module")
def lib():
    if not os.path.exists(an5d.LIB_PATH):
        from paper_2001_01473_gb300 import build
        build.build()
    return an5d.load()


def test_header_declares_entry_points():
    names = declared_functions()
    for n in ("an5d_plan_create", "an5d_run", "an5d_plan_destroy"):
        assert n in names


def test_library_exports_every_declared_symbol(lib):
    missing = [n for n in declared_functions() if not hasattr(lib, n)]
    assert not missing, missing


def test_coeff_count(lib):
    for ndim in (2, 3):
        for R in (1, 2, 3, 4):
            assert an5d.an5d_coeff_count(ndim, inputs.STAR, R) == 2 * ndim * R + 1
            assert an5d.an5d_coeff_count(ndim, inputs.BOX, R) == (2 * R + 1) ** ndim
    with pytest.raises(an5d.An5dError) as e:
        an5d.an5d_coeff_count(4, inputs.STAR, 1)
    assert e.value.status == an5d.AN5D_ERR_UNSUPPORTED
    with pytest.raises(an5d.An5dError):
        an5d.an5d_coeff_count(2, inputs.STAR, 9)


def test_plan_create_rejects_bad_arguments(lib):
    c = np.ones(5)
    P = ctypes.c_void_p
    assert not lib.an5d_plan_create(2, 0, 1, None, 0, np.array([8, 8], np.int64).ctypes.data)
    assert an5d.an5d_last_status() == an5d.AN5D_ERR_INVALID_ARG
    assert "NULL" in an5d.an5d_last_error()
    with pytest.raises(an5d.An5dError) as e:
        an5d.an5d_plan_create(2, inputs.STAR, 1, c, "f32", [0, 8])
    assert e.value.status == an5d.AN5D_ERR_INVALID_ARG
    with pytest.raises(an5d.An5dError) as e:
        an5d.an5d_plan_create(2, inputs.STAR, 1, c, "f32", [70000, 70000])
    assert e.value.status == an5d.AN5D_ERR_UNSUPPORTED
    with pytest.raises(an5d.An5dError) as e:
        an5d.an5d_plan_create(2, inputs.STAR, 1, c, 9, [8, 8])
    assert e.value.status == an5d.AN5D_ERR_INVALID_ARG
    _ = P


def test_null_plan_calls_fail_cleanly(lib):
    assert lib.an5d_run(None, None, None, 1, None) == an5d.AN5D_ERR_INVALID_ARG
    assert lib.an5d_plan_status(None) == an5d.AN5D_ERR_INVALID_ARG
    assert lib.an5d_plan_set_config(None, 1, 0) == an5d.AN5D_ERR_INVALID_ARG
    assert lib.an5d_plan_set_tile(None, 0) == an5d.AN5D_ERR_INVALID_ARG
    assert lib.an5d_plan_launches(None, 5) == an5d.AN5D_ERR_INVALID_ARG
    lib.an5d_plan_destroy(None)   # NULL-safe
    assert an5d.an5d_version().startswith("an5d")


def test_plan_create_without_device_reports_cuda_error(lib):
    try:
        import torch
        if torch.cuda.is_available():
            pytest.skip("a device is present")
    except ImportError:
        pass
    with pytest.raises(an5d.An5dError) as e:
        an5d.an5d_plan_create(2, inputs.STAR, 1, np.ones(5), "f32", [16, 16])
    assert e.value.status in (an5d.AN5D_ERR_CUDA, an5d.AN5D_ERR_OOM)


def test_plan_create_div_rejects_bad_arguments(lib):
    c = np.ones(5)
    for kw, status in ((dict(divisor=7.0, post=3, dtype="f32"), an5d.AN5D_ERR_INVALID_ARG),
                       (dict(divisor=0.0, post="div", dtype="f32"), an5d.AN5D_ERR_INVALID_ARG),
                       (dict(divisor=float("inf"), post="rcp", dtype="f64"), an5d.AN5D_ERR_INVALID_ARG),
                       (dict(divisor=1e-300, post="div", dtype="f32"), an5d.AN5D_ERR_INVALID_ARG),
                       (dict(divisor=7.0, post="div", dtype="f16"), an5d.AN5D_ERR_UNSUPPORTED),
                       (dict(divisor=7.0, post="div", dtype="f32c"), an5d.AN5D_ERR_UNSUPPORTED)):
        with pytest.raises(an5d.An5dError) as e:
            an5d.an5d_plan_create_div(2, inputs.STAR, 1, c, kw["divisor"], kw["post"], kw["dtype"],
                                      [8, 8])
        assert e.value.status == status, kw
