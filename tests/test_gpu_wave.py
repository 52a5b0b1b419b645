"""The complex object wave (cgh_wave) and the kinoform of Eq. 3 (CGH_Q_PHASE)
against the FP64 oracle.  This is the workload the paper times in Tables 3-4
(phase-only CGH, 1920x1080, 10^3..10^5 points)."""
import numpy as np
import pytest

import oracle
from paper_1309_2734_gb300 import Hologram, workloads
from paper_1309_2734_gb300 import _lib

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")

NRMS = {"direct_sfu": 1e-5, "gemm_f16": 2e-3, "gemm_bf16": 1e-2, "gemm_split16": 1e-5}


@pytest.fixture(scope="module", autouse=True)
def _built():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1309_2734_gb300.build import build
    build()
    torch.cuda.set_device(0)


def _wave(c, form, opts=None):
    xyz, amp = torch.from_numpy(c.xyz).cuda(), torch.from_numpy(c.amp).cuda()
    with Hologram(c.width, c.height, c.pitch_m, c.lambda_m, form=form, timeout_ms=5000) as h:
        for k, v in (opts or {}).items():
            h.set_option(k, v)
        w = h.wave(xyz, amp)
        q = h.kinoform8(w)
        h.sync()
    w = w.cpu().numpy().astype(np.float64)
    return w[0] + 1j * w[1], q.cpu().numpy()


def _check_wave(got, ref, tol):
    assert oracle.nrms(got.real, ref.real) <= tol
    assert oracle.nrms(got.imag, ref.imag) <= tol


def _check_kinoform(q, got, ref):
    """Bit-exact against the oracle's kinoform of the FP64 wave, except at ties: pixels whose
    scaled phase lies within the wave's measured error of a quantisation step."""
    want = oracle.kinoform8(ref)
    psi = np.mod(np.angle(ref), 2 * np.pi)
    scaled = 255.0 * psi / (2 * np.pi)
    rel = np.abs(got - ref) / np.maximum(np.abs(ref), 1e-30)
    delta = 255.0 / (2 * np.pi) * (rel + 1e-6) + 1e-4
    dist = np.abs(scaled - np.round(scaled))
    wrap = (scaled > 255.0 - delta) | (scaled < delta)          # 0 and 255 meet at psi = 0
    ties = (dist <= delta) | wrap
    mism = q != want
    assert not np.any(mism & ~ties), int(np.sum(mism & ~ties))
    assert ties.mean() < 0.02


@pytest.mark.parametrize("form", ["direct_sfu", "gemm_f16", "gemm_bf16", "gemm_split16"])
@pytest.mark.parametrize("w,h,n", [(256, 256, 1024), (257, 33, 300), (31, 130, 77)])
def test_wave_vs_oracle(form, w, h, n):
    c = workloads.random_cloud(300 + w + n, w, h, n)
    ref = oracle.wave(c.pitch_m, c.lambda_m, c.xyz, c.amp, w, h)
    got, q = _wave(c, form)
    _check_wave(got, ref, NRMS[form])
    if form in ("direct_sfu", "gemm_split16"):
        _check_kinoform(q, got, ref)


@pytest.mark.parametrize("split", [2, 5])
def test_wave_point_splits(split):
    c = workloads.random_cloud(311, 300, 90, 2500)
    ref = oracle.wave(c.pitch_m, c.lambda_m, c.xyz, c.amp, 300, 90)
    got, _ = _wave(c, "direct_sfu", {_lib.CGH_OPT_POINT_SPLIT: split})
    _check_wave(got, ref, 1e-5)


def test_wave_gemm_point_chunks_and_splits():
    c = workloads.random_cloud(312, 320, 200, 3000)
    ref = oracle.wave(c.pitch_m, c.lambda_m, c.xyz, c.amp, 320, 200)
    got, _ = _wave(c, "gemm_split16", {_lib.CGH_OPT_FACTOR_BUDGET_MB: 1, _lib.CGH_OPT_GEMM_SPLITK: 3})
    _check_wave(got, ref, 1e-5)


def test_paper_workload_kinoform_display_size_sampled():
    """1920x1080, 10^4 points: the phase-only CGH of the paper's Table 3, sampled rows."""
    c = workloads.display_direct()
    rows = (0, 333, 1079)
    refs = [oracle.wave(c.pitch_m, c.lambda_m, c.xyz, c.amp, 1920, 1080, window=(r, 0, 1, 1920)) for r in rows]
    for form in ("direct_sfu", "gemm_split16"):
        got, q = _wave(c, form)
        for r, ref in zip(rows, refs):
            _check_wave(got[r:r + 1], ref, 1e-5)
            _check_kinoform(q[r:r + 1], got[r:r + 1], ref)


def test_wave_many_points_sampled_rows():
    """10^5 points on a 1920x1080 hologram: the direct wave's row walks by complex rotation (restarted at every
    point and row) leave no error that grows with the number of points; sampled rows at both edges and the middle."""
    c = workloads.random_cloud(313, 1920, 1080, 100000)
    rows = (0, 541, 1079)
    got, _ = _wave(c, "direct_sfu")
    for r in rows:
        ref = oracle.wave(c.pitch_m, c.lambda_m, c.xyz, c.amp, 1920, 1080, window=(r, 0, 1, 1920))
        _check_wave(got[r:r + 1], ref, 1e-5)


def test_wave_wide_block_sampled_rows():
    """4096 x 32 with 10^5 points: the layout model gives the wave the wide block (16 tiles of 256 x 32 against 32
    of 128 x 64), whose threads take their own sines and cosines; sampled rows against the oracle."""
    c = workloads.random_cloud(314, 4096, 32, 100000)
    got, _ = _wave(c, "direct_sfu")
    for r in (0, 31):
        ref = oracle.wave(c.pitch_m, c.lambda_m, c.xyz, c.amp, 4096, 32, window=(r, 0, 1, 4096))
        _check_wave(got[r:r + 1], ref, 1e-5)


def test_kinoform_quantiser_same_field():
    """The GPU phase rule on given float fields against the oracle's on the same values."""
    rng = np.random.default_rng(9)
    re = rng.standard_normal(5000).astype(np.float32)
    im = rng.standard_normal(5000).astype(np.float32)
    re[:4] = [1, 0, -1, 0]
    im[:4] = [0, 1, 0, -1]
    dev = torch.from_numpy(np.stack([re, im])).cuda()
    with Hologram(8, 8, 8e-6, 532e-9) as h:
        q = h.kinoform8(dev)
        h.sync()
    q = q.cpu().numpy()
    ref = re.astype(np.float64) + 1j * im.astype(np.float64)
    want = oracle.kinoform8(ref)
    scaled = 255.0 * np.mod(np.angle(ref), 2 * np.pi) / (2 * np.pi)
    ties = np.abs(scaled - np.round(scaled)) < 1e-4
    assert np.array_equal(q[~ties], want[~ties])
    assert list(q[:4]) == [0, 63, 127, 191]


@pytest.mark.parametrize("trans", [1, 2])
def test_wave_gemm_orientations(trans):
    c = workloads.random_cloud(313, 300, 140, 1200)
    ref = oracle.wave(c.pitch_m, c.lambda_m, c.xyz, c.amp, 300, 140)
    got, _ = _wave(c, "gemm_split16", {_lib.CGH_OPT_GEMM_TRANSPOSE: trans})
    _check_wave(got, ref, 1e-5)
