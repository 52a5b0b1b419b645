"""The autotuner's cache file, checked on the host (no GPU): the tuner accepts a cache only when it names the
device and the ABI and holds a complete table of finite, non-negative time coefficients; a truncated, edited or
foreign file is ignored (the tuner then calibrates and rewrites it)."""
import math
import os

import pytest

from paper_1309_2734_gb300 import _lib

DEVICE = "NVIDIA GB300:152"


def _text(device=DEVICE, abi=1, coef=None, bn='"1920x1080:3": 224, "4096x4096:5": 256'):
    coef = coef or [[1.5e-6 * (i + 1), 2.0e-13, 3.0e-11] for i in range(6)]
    rows = ", ".join("[" + ", ".join(f"{v:.9e}" if math.isfinite(v) else str(v).lower() for v in r) + "]"
                     for r in coef)
    return '{\n "abi": %d,\n "device": "%s",\n "coef": [%s],\n "bn": {%s}\n}\n' % (abi, device, rows, bn)


@pytest.fixture(scope="module")
def lib():
    try:
        return _lib.load()
    except OSError as e:   # pragma: no cover - the library is built by __graft_entry__.build()
        pytest.skip(f"libcgh.so not built: {e}")


def _check(tmp_path, text, device=DEVICE):
    path = tmp_path / "tune.json"
    path.write_text(text)
    return _lib.cgh_tune_cache_check(str(path), device)


def test_a_written_cache_is_accepted(lib, tmp_path):
    assert _check(tmp_path, _text())


def test_other_device_or_abi_is_refused(lib, tmp_path):
    assert not _check(tmp_path, _text(device="NVIDIA B200:148"))
    assert not _check(tmp_path, _text(abi=2))
    assert not _check(tmp_path, _text(abi=12))


@pytest.mark.parametrize("bad", [float("nan"), -1.0e-9, float("inf")])
def test_non_finite_or_negative_coefficients_are_refused(lib, tmp_path, bad):
    coef = [[1.0e-6, 1.0e-13, 1.0e-11] for _ in range(6)]
    coef[3][1] = bad
    assert not _check(tmp_path, _text(coef=coef))


def test_every_truncation_that_loses_data_is_refused(lib, tmp_path):
    text = _text()
    end = text.index("}\n}") + 1   # the tile-width table is complete from here on
    for cut in range(0, end):
        assert not _check(tmp_path, text[:cut]), cut


def test_missing_tables_and_garbage_are_refused(lib, tmp_path):
    text = _text()
    assert not _check(tmp_path, text.replace('"bn": {', '"tiles": {'))
    assert not _check(tmp_path, text.replace('"coef": [', '"coefs": ['))
    assert not _check(tmp_path, "\x00\xff garbage")
    assert not _check(tmp_path, "")


def test_unreadable_path_is_not_an_error(lib, tmp_path):
    assert not _lib.cgh_tune_cache_check(str(tmp_path / "missing" / "tune.json"), DEVICE)


def test_unsupported_tile_widths_are_skipped_not_fatal(lib, tmp_path):
    assert _check(tmp_path, _text(bn='"1920x1080:3": 200, "640x480:5": 224'))
