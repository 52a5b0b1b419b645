"""Host-side checks of the C ABI that need no GPU: the library loads, exports
every entry point include/cgh.h declares, and rejects bad arguments before
touching the device."""
import ctypes
import os
import re

import pytest

from paper_1309_2734_gb300 import _lib
from paper_1309_2734_gb300.build import build

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.fixture(scope="module")
def lib():
    build()
    return _lib.load()


def _declared():
    text = open(os.path.join(ROOT, "include", "cgh.h")).read()
    text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
    return sorted(set(re.findall(r"\b(cgh_[a-z0-9_]+)\s*\(", text)))


def test_header_declares_the_abi():
    names = _declared()
    for required in ("cgh_create", "cgh_destroy", "cgh_point_cloud", "cgh_batch", "cgh_quantize8", "cgh_sync"):
        assert required in names


def test_every_declared_symbol_is_exported(lib):
    for name in _declared():
        assert hasattr(lib, name), name
    assert set(_lib.EXPORTS) >= set(_declared())


def test_abi_version_and_strings(lib):
    assert lib.cgh_abi_version() == 1
    for code in range(7):
        assert lib.cgh_status_string(code)
    assert b"unknown" in lib.cgh_status_string(99)


@pytest.mark.parametrize("w,h,p,lam", [(0, 10, 8e-6, 5e-7), (10, 0, 8e-6, 5e-7), (16385, 4, 8e-6, 5e-7),
                                       (10, 10, 0.0, 5e-7), (10, 10, 8e-6, -1.0),
                                       (10, 10, float("nan"), 5e-7), (10, 10, 8e-6, float("inf"))])
def test_create_rejects_bad_arguments(lib, w, h, p, lam):
    out = ctypes.c_void_p(1)
    assert lib.cgh_create(w, h, p, lam, ctypes.byref(out)) == _lib.CGH_EINVAL
    assert out.value is None


def test_create_null_out(lib):
    assert lib.cgh_create(10, 10, 8e-6, 5e-7, None) == _lib.CGH_EINVAL


def test_null_context_everywhere(lib):
    assert lib.cgh_point_cloud(None, None, None, 0, None) == _lib.CGH_EINVAL
    assert lib.cgh_point_cloud_host(None, None, None, 0, None) == _lib.CGH_EINVAL
    assert lib.cgh_quantize8(None, None, 0, 0, None) == _lib.CGH_EINVAL
    assert lib.cgh_factors(None, None, None, 0, 3, None, None, 64) == _lib.CGH_EINVAL
    assert lib.cgh_batch(None, None, 0) == _lib.CGH_EINVAL
    assert lib.cgh_sync(None) == _lib.CGH_EINVAL
    assert lib.cgh_set_form(None, 1) == _lib.CGH_EINVAL
    assert lib.cgh_set_option(None, 1, 1) == _lib.CGH_EINVAL
    assert lib.cgh_set_stream(None, None) == _lib.CGH_EINVAL
    assert lib.cgh_set_reference(None, 0.0, 0.0, 0.0) == _lib.CGH_EINVAL
    assert lib.cgh_wave(None, None, None, 0, None) == _lib.CGH_EINVAL
    assert lib.cgh_fresnel(None, None, 0.1, None) == _lib.CGH_EINVAL
    assert lib.cgh_wrp(None, None, None, 0, 0.5, None) == _lib.CGH_EINVAL
    assert lib.cgh_wrp_record(None, None, None, 0, 0.5, None) == _lib.CGH_EINVAL
    assert lib.cgh_autotune(None, 0) == _lib.CGH_EINVAL
    n = ctypes.c_int(0)
    assert lib.cgh_batch_forms(None, None, 0, ctypes.byref(n)) == _lib.CGH_EINVAL
    v = ctypes.c_double(0.0)
    assert lib.cgh_measure_mufu(None, ctypes.byref(v)) == _lib.CGH_EINVAL
    assert lib.cgh_destroy(None) == _lib.CGH_OK


def test_create_without_gpu_fails_loudly(lib):
    import torch
    if torch.cuda.is_available():
        pytest.skip("a GPU is present")
    out = ctypes.c_void_p()
    assert lib.cgh_create(64, 64, 8e-6, 532e-9, ctypes.byref(out)) == _lib.CGH_ECUDA
