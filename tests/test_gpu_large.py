"""The large depth-layered case: a 4096x4096 hologram of 10^6 points on 16
depth planes, split FP16 GEMM form (grouped by plane and column), its 8-bit
quantised output.  The oracle is checked on the central 512x512 crop (about
five minutes of oracle time on 16 cores; CGH_LARGE_CROP sets another size)."""
import os

import numpy as np
import pytest

import oracle
from paper_1309_2734_gb300 import Hologram, workloads

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")

CROP = int(os.environ.get("CGH_LARGE_CROP", "512"))


@pytest.fixture(scope="module")
def large():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1309_2734_gb300.build import build
    build()
    torch.cuda.set_device(0)
    c = workloads.large_layered()
    xyz, amp = torch.from_numpy(c.xyz).cuda(), torch.from_numpy(c.amp).cuda()
    with Hologram(4096, 4096, c.pitch_m, c.lambda_m, form="gemm_split16", timeout_ms=60000) as h:
        h.profile(True)
        f = h.point_cloud(xyz, amp)
        q = h.quantize8(f)
        h.sync()
        names = set(h.profile_read())
        field, q = f.cpu().numpy(), q.cpu().numpy()
    return c, field, q, names


def test_large_runs_grouped(large):
    assert "group_factors" in large[3]


def test_large_quantised_field_bit_exact_on_same_field(large):
    """The whole 4096x4096 field: GPU uint8 equals the oracle's quantisation of the same float field."""
    _, field, q, _ = large
    assert np.array_equal(q, oracle.quantize8(field)[0])


def test_large_crop_field_and_quantisation(large):
    """Central crop: the float field within 1e-5 NRMS of the FP64 oracle, and the uint8 crop
    (min/max of the crop) equal to the oracle's quantisation of its own field away from ties."""
    c, field, _, _ = large
    r0, c0, rows, cols = workloads.large_crop(4096, CROP)
    ref = oracle.field(c.pitch_m, c.lambda_m, c.xyz, c.amp, 4096, 4096, window=(r0, c0, rows, cols))
    got = np.ascontiguousarray(field[r0:r0 + rows, c0:c0 + cols])
    assert oracle.nrms(got, ref) <= 1e-5
    with Hologram(8, 8, 8e-6, 532e-9) as h:
        qg = h.quantize8(torch.from_numpy(got).cuda())
        h.sync()
    qg = qg.cpu().numpy()
    ref32 = ref.astype(np.float32)
    qr, (lo, hi, s) = oracle.quantize8(ref32)
    scaled = (ref - lo) * s
    delta = (np.max(np.abs(got.astype(np.float64) - ref)) + abs(float(got.min()) - lo)
             + np.abs(ref32.astype(np.float64) - ref).max()) * s * 2.0 + 2.0 ** -20
    ties = np.abs(scaled - np.round(scaled)) <= delta
    mism = qg != qr
    assert not np.any(mism & ~ties), int(np.sum(mism & ~ties))
    assert ties.mean() < 0.02
