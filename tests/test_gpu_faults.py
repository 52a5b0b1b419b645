"""Failures injected on the host, recovered from without any device fault: an autotuner cache that is
corrupted, truncated or foreign (the tuner ignores it, calibrates and rewrites it), a save/load round trip
of the cache, and a refused workspace allocation (CGH_ENOMEM, then the context works again)."""
import os
import re

import numpy as np
import pytest

import oracle
from paper_1309_2734_gb300 import CghError, Hologram, batch, workloads
from paper_1309_2734_gb300 import _lib

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")


@pytest.fixture(scope="module", autouse=True)
def _built():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1309_2734_gb300.build import build
    build()
    torch.cuda.set_device(0)


@pytest.fixture
def cache(tmp_path, monkeypatch):
    path = tmp_path / "tune.json"
    monkeypatch.setenv("CGH_TUNE_CACHE", str(path))
    return path


def _device_of(path):
    return re.search(r'"device": "([^"]*)"', path.read_text()).group(1)


def _auto_hologram_ok(tol_e9=10000):
    c = workloads.random_cloud(910, 320, 180, 3000)
    xyz, amp = torch.from_numpy(c.xyz).cuda(), torch.from_numpy(c.amp).cuda()
    with Hologram(c.width, c.height, c.pitch_m, c.lambda_m, form="auto") as h:
        h.set_option(_lib.CGH_OPT_TOLERANCE_E9, tol_e9)
        f = h.point_cloud(xyz, amp)
        h.sync()
    ref = oracle.field(c.pitch_m, c.lambda_m, c.xyz, c.amp, c.width, c.height)
    assert oracle.nrms(f.cpu().numpy(), ref) <= tol_e9 * 1e-9


def test_cache_round_trip(cache):
    """Calibration writes the cache; a new context loads it instead of calibrating (the file is not rewritten)."""
    with Hologram(8, 8, 8e-6, 532e-9, form="auto") as h:
        _lib.check(_lib.cgh_autotune(h.ctx, 1), "cgh_autotune")
    assert cache.exists()
    assert _lib.cgh_tune_cache_check(str(cache), _device_of(cache))
    stamp = cache.stat().st_mtime_ns
    text = cache.read_text()
    with Hologram(8, 8, 8e-6, 532e-9, form="auto") as h:
        _lib.check(_lib.cgh_autotune(h.ctx, 0), "cgh_autotune")
    assert cache.stat().st_mtime_ns == stamp and cache.read_text() == text
    _auto_hologram_ok()


@pytest.mark.parametrize("damage", ["nan", "negative", "truncated", "device", "abi"])
def test_damaged_cache_is_recalibrated(cache, damage):
    """A damaged cache is refused: the tuner calibrates, rewrites a valid cache, and its choices meet the
    tolerance."""
    with Hologram(8, 8, 8e-6, 532e-9, form="auto") as h:
        _lib.check(_lib.cgh_autotune(h.ctx, 1), "cgh_autotune")
    text = cache.read_text()
    device = _device_of(cache)
    if damage == "nan":
        bad = re.sub(r"\[([0-9.e+-]+),", "[nan,", text, count=1)
    elif damage == "negative":
        bad = re.sub(r"\[([0-9.e+-]+),", "[-1.0e-03,", text, count=1)
    elif damage == "truncated":
        bad = text[: len(text) // 2]
    elif damage == "device":
        bad = text.replace(device, "another device:1")
    else:
        bad = text.replace('"abi": ', '"abi": 9')
    assert bad != text
    cache.write_text(bad)
    assert not _lib.cgh_tune_cache_check(str(cache), device)
    with Hologram(8, 8, 8e-6, 532e-9, form="auto") as h:
        _lib.check(_lib.cgh_autotune(h.ctx, 0), "cgh_autotune")
    assert _lib.cgh_tune_cache_check(str(cache), device)
    _auto_hologram_ok()


@pytest.mark.parametrize("form", ["direct_sfu", "gemm_split16"])
def test_refused_allocation_then_recovery(form):
    """The first workspace growth is refused (as a failed cudaMalloc): CGH_ENOMEM, nothing launched; the same
    context then computes the hologram."""
    c = workloads.random_cloud(911, 300, 140, 2500)
    xyz, amp = torch.from_numpy(c.xyz).cuda(), torch.from_numpy(c.amp).cuda()
    with Hologram(c.width, c.height, c.pitch_m, c.lambda_m, form=form) as h:
        h.set_option(_lib.CGH_OPT_TEST_ALLOC_FAIL, 1)
        out = torch.full((c.height, c.width), 7.0, device="cuda")
        with pytest.raises(CghError) as ei:
            h.point_cloud(xyz, amp, out)
        assert ei.value.code == _lib.CGH_ENOMEM
        h.sync()
        f = h.point_cloud(xyz, amp, out)
        h.sync()
    ref = oracle.field(c.pitch_m, c.lambda_m, c.xyz, c.amp, c.width, c.height)
    assert oracle.nrms(f.cpu().numpy(), ref) <= 1e-5


def test_refused_batch_arena_then_recovery():
    clouds = [workloads.random_cloud(912, 200, 100, 900), workloads.random_cloud(913, 96, 64, 300)]
    dev = [(torch.from_numpy(c.xyz).cuda(), torch.from_numpy(c.amp).cuda(), c.width, c.height, c.pitch_m,
            c.lambda_m) for c in clouds]
    outs = [torch.zeros((c.height, c.width), device="cuda") for c in clouds]
    with Hologram(8, 8, 8e-6, 532e-9, form="direct_sfu") as h:
        h.set_option(_lib.CGH_OPT_TEST_ALLOC_FAIL, 1)
        with pytest.raises(CghError) as ei:
            batch(h, dev, outs)
        assert ei.value.code == _lib.CGH_ENOMEM
        batch(h, dev, outs)
        h.sync()
    for c, o in zip(clouds, outs):
        ref = oracle.field(c.pitch_m, c.lambda_m, c.xyz, c.amp, c.width, c.height)
        assert oracle.nrms(o.cpu().numpy(), ref) <= 1e-5
