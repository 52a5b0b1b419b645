"""The GEMM's launch-shape choice (cgh_gemm_layout, host only): argument checks, the invariants every layout
keeps, and the choices at hologram shapes whose layouts were all timed on a GB300."""
import ctypes
import itertools

import pytest

from paper_1309_2734_gb300 import _lib
from paper_1309_2734_gb300.build import build

GEMM_FORMS = (_lib.CGH_GEMM_F16, _lib.CGH_GEMM_BF16, _lib.CGH_GEMM_SPLIT16)


@pytest.fixture(scope="module")
def lib():
    build()
    return _lib.load()


@pytest.mark.parametrize("w,h,n,form,sms", [(0, 10, 5, 3, 152), (10, 16385, 5, 3, 152), (10, 10, 0, 3, 152),
                                             (10, 10, 5, _lib.CGH_DIRECT_SFU, 152), (10, 10, 5, 6, 152),
                                             (10, 10, 5, 3, 0)])
def test_rejects_bad_arguments(lib, w, h, n, form, sms):
    out = (ctypes.c_int * 4)()
    assert lib.cgh_gemm_layout(w, h, n, form, sms, out) == _lib.CGH_EINVAL


def test_rejects_null_layout(lib):
    assert lib.cgh_gemm_layout(10, 10, 5, _lib.CGH_GEMM_F16, 152, None) == _lib.CGH_EINVAL


@pytest.mark.parametrize("form", GEMM_FORMS)
def test_layout_invariants(lib, form):
    sides = (1, 7, 128, 300, 1024, 1080, 1920, 2160, 3840, 4096, 16384)
    for w, h, n in itertools.product(sides, sides, (1, 33, 1000, 50000, 10 ** 6)):
        lay = _lib.cgh_gemm_layout(w, h, n, form, 152)
        assert lay["bn"] in (128, 192, 224, 240, 256)
        assert not (lay["pair"] and lay["bn"] == 240)   # the two-SM form splits B into whole 32-row halves
        kb = (2 * n + 63) // 64
        assert 1 <= lay["splits"] <= min(16, kb)   # every split has k-blocks of its own


# Layouts timed on a GB300 (every tile width, 1-16 K splits, both orientations, both forms; kernel time plus the
# split reduction): the choice at each of these shapes was the fastest or within 1 % of it.
@pytest.mark.parametrize("w,h,n,form,want", [
    (1920, 1080, 50000, _lib.CGH_GEMM_F16, (True, 224, 2, False)),
    (1920, 1080, 50000, _lib.CGH_GEMM_SPLIT16, (True, 224, 2, False)),
    (1920, 1080, 10000, _lib.CGH_GEMM_SPLIT16, (True, 224, 2, False)),
    (1024, 1024, 95015, _lib.CGH_GEMM_F16, (True, 256, 9, True)),
    (1024, 1024, 8000, _lib.CGH_GEMM_F16, (True, 256, 4, True)),
])
def test_layout_at_timed_shapes(lib, w, h, n, form, want):
    lay = _lib.cgh_gemm_layout(w, h, n, form, 152)
    assert (lay["transposed"], lay["bn"], lay["splits"], lay["pair"]) == want
