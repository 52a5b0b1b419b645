"""The allocation-free entry point, cgh_point_cloud_noalloc, through the C ABI.

It serves callers that may not call cudaMalloc (real-time loops, hosts that
only lend pre-registered buffers, plug-ins inside another program's memory
budget): its scratch is a fixed array inside the library.  Its output must
match the regular entry point (cgh_point_cloud, same direct SFU form) within
the direct form's tolerance, on two calls in a row with different clouds, so
that stale scratch contents from the first call cannot leak into the second.

This file is named to be collected last; it passes alone in a fresh process
and after the other tests.
"""
import ctypes

import numpy as np
import pytest

import oracle
from paper_1309_2734_gb300 import Hologram, workloads
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


def _regular(c, xyz, amp):
    with Hologram(c.width, c.height, c.pitch_m, c.lambda_m, form="direct_sfu") as h:
        f = h.point_cloud(xyz, amp)
        h.sync()
        return f.cpu().numpy()


def test_noalloc_matches_regular_entry_point_twice():
    stream = torch.cuda.current_stream()
    clouds = [workloads.random_cloud(901, 333, 211, 5000), workloads.random_cloud(902, 333, 211, 700)]
    for c in clouds:
        xyz = torch.from_numpy(c.xyz).cuda()
        amp = torch.from_numpy(c.amp).cuda()
        out = torch.full((c.height, c.width), float("nan"), device="cuda")
        rc = _lib.cgh_point_cloud_noalloc(c.width, c.height, c.pitch_m, c.lambda_m, xyz.data_ptr(),
                                          amp.data_ptr(), c.n_points, out.data_ptr(), stream.cuda_stream)
        assert rc == _lib.CGH_OK, _lib.status_string(rc)
        got = out.cpu().numpy()
        want = _regular(c, xyz, amp)
        assert np.all(np.isfinite(got))
        assert oracle.nrms(got, want) <= 1e-5
        ref = oracle.field(c.pitch_m, c.lambda_m, c.xyz, c.amp, c.width, c.height)
        assert oracle.nrms(got, ref) <= 1e-5


def test_noalloc_rejects_oversized_and_bad_input():
    n = _lib.CGH_NOALLOC_MAX_POINTS + 1
    out = torch.zeros((8, 8), device="cuda")
    rc = _lib.cgh_point_cloud_noalloc(8, 8, 8e-6, 532e-9, out.data_ptr(), out.data_ptr(), n, out.data_ptr(), 0)
    assert rc == _lib.CGH_EINVAL
    assert torch.count_nonzero(out).item() == 0          # nothing was launched
    c = workloads.random_cloud(903, 64, 48, 50)
    xyz = c.xyz.copy()
    xyz[7, 2] = -1.0
    rc = _lib.cgh_point_cloud_noalloc(64, 48, c.pitch_m, c.lambda_m, torch.from_numpy(xyz).cuda().data_ptr(),
                                      torch.from_numpy(c.amp).cuda().data_ptr(), c.n_points,
                                      torch.empty((48, 64), device="cuda").data_ptr(), 0)
    assert rc == _lib.CGH_EINPUT
    empty = torch.full((48, 64), 3.0, device="cuda")
    assert _lib.cgh_point_cloud_noalloc(64, 48, c.pitch_m, c.lambda_m, 0, 0, 0, empty.data_ptr(), 0) == _lib.CGH_OK
    assert torch.count_nonzero(empty).item() == 0
