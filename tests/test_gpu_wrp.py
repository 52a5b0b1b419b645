"""Fresnel diffraction (Eq. 10) and the wavefront-recording method (Section 2.3)
against the FP64 oracle.  Tolerance: NRMS <= 1e-5 (single-precision FFT and
hardware sine and cosine; both are a few 1e-7 here)."""
import math

import numpy as np
import pytest

import oracle
from paper_1309_2734_gb300 import Hologram, workloads
from paper_1309_2734_gb300 import _lib

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")

TOL = 1e-5


@pytest.fixture(scope="module", autouse=True)
def _built():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1309_2734_gb300.build import build
    build()
    torch.cuda.set_device(0)


def _cplx(t):
    a = t.cpu().numpy().astype(np.float64)
    return a[0] + 1j * a[1]


def _nrms_c(got, ref):
    return float(np.sqrt(np.sum(np.abs(got - ref) ** 2) / np.sum(np.abs(ref) ** 2)))


@pytest.mark.parametrize("w,h,z", [(48, 64, 0.05), (128, 128, 0.2), (300, 200, -0.1), (1, 37, 0.02)])
def test_fresnel_vs_oracle(w, h, z):
    u = workloads.complex_plane(900 + w, w, h)
    ref = oracle.fresnel(u[0].astype(np.float64) + 1j * u[1], 8e-6, 532e-9, z)
    with Hologram(w, h, 8e-6, 532e-9) as hol:
        got = _cplx(hol.fresnel(torch.from_numpy(u).cuda(), z))
        hol.sync()
    assert _nrms_c(got, ref) <= TOL


@pytest.mark.parametrize("w,h,z", [(40, 100, 0.03), (3, 100, 0.03), (70, 250, -0.05), (160, 400, 0.08),
                                   (9, 700, 0.1), (300, 700, 0.12)])
def test_fresnel_fused_column_forms(w, h, z):
    """Padded grids of 256, 512, 1024 and 2048 rows, whose columns take the one-pass strip transform (strips of
    32, 16, 8 and 8 columns), ragged widths, and a plane too narrow for its strip (3 x 100: the four-step passes),
    against the oracle; the same context then alternates distances (the spectrum, in natural order, rebuilt)."""
    u = workloads.complex_plane(930 + w + h, w, h)
    uc = u[0].astype(np.float64) + 1j * u[1]
    with Hologram(w, h, 8e-6, 532e-9) as hol:
        for zz in (z, 1.5 * z, z):
            got = _cplx(hol.fresnel(torch.from_numpy(u).cuda(), zz))
            hol.sync()
            assert _nrms_c(got, oracle.fresnel(uc, 8e-6, 532e-9, zz)) <= TOL


def test_fresnel_wide_plane_uses_the_library_fft():
    """A plane wider than the own FFT's longest transform (2W - 1 > 16384): the cuFFT path, same result."""
    u = workloads.complex_plane(909, 8200, 3)
    ref = oracle.fresnel(u[0].astype(np.float64) + 1j * u[1], 8e-6, 532e-9, 0.2)
    with Hologram(8200, 3, 8e-6, 532e-9) as hol:
        hol.profile(True)
        got = _cplx(hol.fresnel(torch.from_numpy(u).cuda(), 0.2))
        hol.sync()
        names = set(hol.profile_read())
    assert "cufft_c2c" in names
    assert _nrms_c(got, ref) <= TOL


def test_fresnel_own_fft_on_display_sizes():
    """1920 x 1080 (padded to 4096 x 4096 by the own FFT): sampled pixels against the direct sum."""
    u = workloads.complex_plane(908, 1920, 1080)
    uc = u[0].astype(np.float64) + 1j * u[1]
    rng = np.random.default_rng(907)
    cols = np.concatenate([rng.integers(0, 1920, 24), [0, 1919]])
    rows = np.concatenate([rng.integers(0, 1080, 24), [1079, 0]])
    ref = oracle.fresnel_at(uc, 8e-6, 532e-9, 0.25, cols, rows)
    with Hologram(1920, 1080, 8e-6, 532e-9) as hol:
        hol.profile(True)
        got = _cplx(hol.fresnel(torch.from_numpy(u).cuda(), 0.25))
        hol.sync()
        names = set(hol.profile_read())
    assert "fresnel_fft" in names and "cufft_c2c" not in names
    assert _nrms_c(got[rows, cols], ref) <= TOL


@pytest.mark.parametrize("w,h", [(4100, 2100), (4200, 64)])
def test_fresnel_own_fft_long_rows_and_columns(w, h):
    """Planes padded to 8192 x 8192 (rows of 8192 points, columns split 128 x 64) and 16384 x 128 (rows of 16384
    points): sampled pixels, edges included, against the direct sum."""
    u = workloads.complex_plane(920 + h, w, h)
    uc = u[0].astype(np.float64) + 1j * u[1]
    rng = np.random.default_rng(921)
    cols = np.concatenate([rng.integers(0, w, 24), [0, w - 1]])
    rows = np.concatenate([rng.integers(0, h, 24), [h - 1, 0]])
    ref = oracle.fresnel_at(uc, 8e-6, 532e-9, 0.4, cols, rows)
    with Hologram(w, h, 8e-6, 532e-9) as hol:
        hol.profile(True)
        got = _cplx(hol.fresnel(torch.from_numpy(u).cuda(), 0.4))
        hol.sync()
        names = set(hol.profile_read())
    assert "fresnel_fft" in names and "cufft_c2c" not in names
    assert _nrms_c(got[rows, cols], ref) <= TOL


def test_fresnel_in_place_and_cached_spectra():
    """d_out == d_in, and spectra for alternating distances (the cache must follow z)."""
    u = workloads.complex_plane(910, 96, 80)
    uc = u[0].astype(np.float64) + 1j * u[1]
    with Hologram(96, 80, 8e-6, 532e-9) as hol:
        for z in (0.05, 0.11, 0.05):
            buf = torch.from_numpy(u).cuda()
            hol.fresnel(buf, z, out=buf)
            hol.sync()
            assert _nrms_c(_cplx(buf), oracle.fresnel(uc, 8e-6, 532e-9, z)) <= TOL


def test_fresnel_gaussian_beam():
    """The GPU propagation of a Gaussian beam against the closed form (see the oracle pin)."""
    N, p, lam, z = 256, 8e-6, 532e-9, 0.1
    w0 = 20 * p
    yy, xx = np.meshgrid((np.arange(N) - N // 2) * p, (np.arange(N) - N // 2) * p, indexing="ij")
    u = np.stack([np.exp(-(xx ** 2 + yy ** 2) / w0 ** 2), np.zeros((N, N))]).astype(np.float32)
    with Hologram(N, N, p, lam) as hol:
        got = _cplx(hol.fresnel(torch.from_numpy(u).cuda(), z))
        hol.sync()
    a, b = 1.0 / w0 ** 2, math.pi / (lam * z)
    zt = z / lam
    pre = np.exp(2j * math.pi * (zt - round(zt))) / (1j * lam * z)
    r2 = xx ** 2 + yy ** 2
    want = pre * (math.pi / (a - 1j * b)) * np.exp(1j * b * r2 - b * b * r2 / (a - 1j * b))
    core = r2 <= (40 * p) ** 2
    assert np.abs(got - want)[core].max() <= 2e-6 * np.abs(want).max()


def test_fresnel_display_size_sampled():
    """1024 x 1024 plane: sampled pixels against the direct sum of Eq. 10."""
    u = workloads.complex_plane(911, 1024, 1024)
    uc = u[0].astype(np.float64) + 1j * u[1]
    rng = np.random.default_rng(912)
    cols = np.concatenate([rng.integers(0, 1024, 40), [0, 1023]])
    rows = np.concatenate([rng.integers(0, 1024, 40), [1023, 0]])
    ref = oracle.fresnel_at(uc, 8e-6, 532e-9, 0.3, cols, rows)
    with Hologram(1024, 1024, 8e-6, 532e-9) as hol:
        got = _cplx(hol.fresnel(torch.from_numpy(u).cuda(), 0.3))
        hol.sync()
    assert _nrms_c(got[rows, cols], ref) <= TOL


@pytest.mark.parametrize("model", [0, 1])
@pytest.mark.parametrize("w,h,n", [(256, 200, 500), (97, 130, 300)])
def test_wrp_record_vs_oracle(model, w, h, n):
    c = workloads.wrp_cloud(913 + n, w, h, n)
    ref = oracle.wrp_record(model, c.pitch_m, c.lambda_m, 0.5, c.xyz, c.amp, w, h)
    xyz, amp = torch.from_numpy(c.xyz).cuda(), torch.from_numpy(c.amp).cuda()
    with Hologram(w, h, c.pitch_m, c.lambda_m) as hol:
        hol.set_phase_model(model)
        got = _cplx(hol.wrp_record(xyz, amp, 0.5))
        hol.sync()
    assert np.array_equal(got != 0, ref != 0)          # the same windows, pixel for pixel
    assert _nrms_c(got, ref) <= TOL


@pytest.mark.parametrize("model", [0, 1])
def test_wrp_vs_oracle(model):
    c = workloads.wrp_cloud(914, 256, 256, 1000)
    ref = oracle.wrp(model, c.pitch_m, c.lambda_m, 0.5, c.xyz, c.amp, 256, 256)
    xyz, amp = torch.from_numpy(c.xyz).cuda(), torch.from_numpy(c.amp).cuda()
    with Hologram(256, 256, c.pitch_m, c.lambda_m) as hol:
        hol.set_phase_model(model)
        o = hol.wrp(xyz, amp, 0.5)
        q = hol.kinoform8(o)
        hol.sync()
    got = _cplx(o)
    assert _nrms_c(got, ref) <= TOL
    k = oracle.kinoform8(ref)
    psi = np.mod(np.angle(ref), 2 * np.pi) * 255.0 / (2 * np.pi)
    rel = np.abs(got - ref) / np.maximum(np.abs(ref), 1e-30)
    delta = 255.0 / (2 * np.pi) * (rel + 1e-6) + 1e-4
    ties = (np.abs(psi - np.round(psi)) <= delta) | (psi > 255.0 - delta) | (psi < delta)
    assert not np.any((q.cpu().numpy() != k) & ~ties)
    assert ties.mean() < 0.02


def test_wrp_1024_full_plane():
    """1024 x 1024, 5000 points 2-10 mm behind the plane: the whole object wave against the oracle."""
    c = workloads.wrp_cloud(915, 1024, 1024, 5000)
    ref = oracle.wrp(1, c.pitch_m, c.lambda_m, 0.5, c.xyz, c.amp, 1024, 1024)
    xyz, amp = torch.from_numpy(c.xyz).cuda(), torch.from_numpy(c.amp).cuda()
    with Hologram(1024, 1024, c.pitch_m, c.lambda_m) as hol:
        hol.set_phase_model("fresnel_piston")
        got = _cplx(hol.wrp(xyz, amp, 0.5))
        hol.sync()
    assert _nrms_c(got, ref) <= TOL


def test_wrp_rejects_points_in_front_and_other_models():
    c = workloads.wrp_cloud(916, 64, 64, 50)
    c.xyz[3, 2] = np.float32(0.4)                        # in front of the plane at 0.5 m
    xyz, amp = torch.from_numpy(c.xyz).cuda(), torch.from_numpy(c.amp).cuda()
    out = torch.empty((2, 64, 64), device="cuda")
    with Hologram(64, 64, c.pitch_m, c.lambda_m) as hol:
        assert _lib.load().cgh_wrp(hol.ctx, xyz.data_ptr(), amp.data_ptr(), 50, 0.5, out.data_ptr()) == _lib.CGH_OK
        assert _lib.load().cgh_sync(hol.ctx) == _lib.CGH_EINPUT
        assert _lib.load().cgh_wrp(hol.ctx, xyz.data_ptr(), amp.data_ptr(), 50, -1.0, out.data_ptr()) == \
            _lib.CGH_EINVAL
        hol.set_phase_model("spherical")
        assert _lib.load().cgh_wrp(hol.ctx, xyz.data_ptr(), amp.data_ptr(), 50, 0.5, out.data_ptr()) == \
            _lib.CGH_ENOTSUP
        hol.set_phase_model("fresnel")
        hol.set_reference(0.01, 0.0, 0.0)
        assert _lib.load().cgh_wrp(hol.ctx, xyz.data_ptr(), amp.data_ptr(), 50, 0.5, out.data_ptr()) == \
            _lib.CGH_ENOTSUP
        assert _lib.load().cgh_fresnel(hol.ctx, out.data_ptr(), 0.0, out.data_ptr()) == _lib.CGH_EINVAL


def test_wrp_empty_cloud_gives_zeros():
    with Hologram(40, 30, 8e-6, 532e-9) as hol:
        e = torch.empty(0, device="cuda")
        o = hol.wrp(e, e, 0.5)
        hol.sync()
        assert torch.count_nonzero(o).item() == 0


def test_numerical_reconstruction_focuses_on_the_point():
    """Back-propagating the hologram's object wave by the point's distance (Fresnel diffraction with a negative
    distance, the numerical reconstruction of the paper's Fig. 4) brings the light back to the point: the
    intensity peaks at (x_j, y_j), with most of the energy of the reconstructed plane there."""
    z_wrp, d = 0.05, 0.004
    N = 512
    xyz = np.array([[200.0, 310.0, z_wrp + d]], dtype=np.float32)
    amp = np.ones(1, dtype=np.float32)
    with Hologram(N, N, 8e-6, 532e-9) as hol:
        hol.set_phase_model("fresnel_piston")
        o = hol.wrp(torch.from_numpy(xyz).cuda(), torch.from_numpy(amp).cuda(), z_wrp)
        back = hol.fresnel(o, -(z_wrp + d))
        hol.sync()
    inten = np.abs(_cplx(back)) ** 2
    r, c = np.unravel_index(np.argmax(inten), inten.shape)
    assert (r, c) == (310, 200)
    assert inten[305:316, 195:206].sum() > 0.5 * inten.sum()
