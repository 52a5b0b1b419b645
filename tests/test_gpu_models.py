"""Phase models beyond the restricted Fresnel form (Section 2.1) against the
FP64 oracle: the piston of Eq. 2, the plane-wave reference phase of Eqs. 4-5
(every form), and the exact spherical wave of Eq. 1 (direct SFU form)."""
import numpy as np
import pytest

import oracle
from paper_1309_2734_gb300 import Hologram, workloads
from paper_1309_2734_gb300 import _lib

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")

NRMS = {"direct_sfu": 1e-5, "direct_accurate": 1e-5, "gemm_f16": 2e-3, "gemm_bf16": 1e-2, "gemm_split16": 1e-5}
REF = (0.0123, -0.0071, 0.7)


@pytest.fixture(scope="module", autouse=True)
def _built():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1309_2734_gb300.build import build
    build()
    torch.cuda.set_device(0)


def _run(c, form, model, ref=None, wave=False, opts=None):
    xyz, amp = torch.from_numpy(c.xyz).cuda(), torch.from_numpy(c.amp).cuda()
    with Hologram(c.width, c.height, c.pitch_m, c.lambda_m, form=form, timeout_ms=10000) as h:
        h.set_phase_model(model)
        if ref is not None:
            h.set_reference(*ref)
        for k, v in (opts or {}).items():
            h.set_option(k, v)
        h.profile(True)
        if wave:
            w = h.wave(xyz, amp)
            q = h.kinoform8(w)
            h.sync()
            w = w.cpu().numpy().astype(np.float64)
            return w[0] + 1j * w[1], q.cpu().numpy(), set(h.profile_read())
        f = h.point_cloud(xyz, amp)
        h.sync()
        return f.cpu().numpy(), None, set(h.profile_read())


@pytest.mark.parametrize("form", ["direct_sfu", "direct_accurate", "gemm_f16", "gemm_split16"])
@pytest.mark.parametrize("model,ref", [(1, None), (0, REF), (1, REF)])
def test_piston_and_reference_vs_oracle(form, model, ref):
    c = workloads.random_cloud(801, 260, 190, 1500)
    want = oracle.model_wave(model, c.pitch_m, c.lambda_m, c.xyz, c.amp, 260, 190,
                             reference=ref or (0.0, 0.0, 0.0)).real
    got, _, _ = _run(c, form, model, ref)
    assert oracle.nrms(got, want) <= NRMS[form]


@pytest.mark.parametrize("form", ["direct_sfu", "gemm_split16"])
def test_piston_and_reference_wave(form):
    c = workloads.random_cloud(802, 200, 130, 1200)
    want = oracle.model_wave(1, c.pitch_m, c.lambda_m, c.xyz, c.amp, 200, 130, reference=REF)
    got, _, _ = _run(c, form, 1, REF, wave=True)
    assert oracle.nrms(got.real, want.real) <= NRMS[form]
    assert oracle.nrms(got.imag, want.imag) <= NRMS[form]


def test_steep_reference_and_far_columns():
    """sin_x = 0.5 (7.5 turns per pixel), points far outside the aperture, a 1000-wide hologram."""
    c = workloads.random_cloud(803, 1000, 40, 600)
    c.xyz[:100, 0] = np.float32(-9000.0)
    c.xyz[100:200, 0] = np.float32(12000.0)
    ref = (0.5, -0.25, -2.0)
    want = oracle.model_wave(1, c.pitch_m, c.lambda_m, c.xyz, c.amp, 1000, 40, reference=ref).real
    for form in ("direct_sfu", "gemm_split16"):
        got, _, _ = _run(c, form, 1, ref)
        assert oracle.nrms(got, want) <= NRMS[form], form
    # the exact distance too: at 72-96 mm from the aperture's edge u reaches 0.1 and the remainder at the tile
    # centres hundreds of turns, whose fraction the double-float evaluation must keep
    want = oracle.model_wave(2, c.pitch_m, c.lambda_m, c.xyz, c.amp, 1000, 40, reference=ref).real
    got, _, _ = _run(c, "direct_sfu", 2, ref)
    assert oracle.nrms(got, want) <= 1e-5


@pytest.mark.parametrize("form", ["gemm_f16", "gemm_split16"])
def test_grouped_with_reference(form):
    c = workloads.layered_cloud(804, 300, 180, 8000, 4)
    want = oracle.model_wave(0, c.pitch_m, c.lambda_m, c.xyz, c.amp, 300, 180, reference=REF).real
    got, _, names = _run(c, form, 0, REF, opts={_lib.CGH_OPT_GEMM_GROUP: 2})
    assert "group_factors" in names
    assert oracle.nrms(got, want) <= NRMS[form]


def test_piston_turns_grouping_off():
    c = workloads.layered_cloud(805, 200, 120, 4000, 3)
    want = oracle.model_wave(1, c.pitch_m, c.lambda_m, c.xyz, c.amp, 200, 120).real
    got, _, names = _run(c, "gemm_split16", 1, opts={_lib.CGH_OPT_GEMM_GROUP: 2})
    assert "group_factors" not in names and "factors" in names
    assert oracle.nrms(got, want) <= NRMS["gemm_split16"]


@pytest.mark.parametrize("form", ["direct_sfu", "auto"])
@pytest.mark.parametrize("w,h,n,z", [(256, 256, 1024, (0.5, 1.0)), (301, 77, 900, (0.3, 1.0)),
                                     (640, 480, 700, (0.1, 0.3))])
def test_spherical_vs_oracle(form, w, h, n, z):
    c = workloads.random_cloud(806 + n, w, h, n, z_range=z)
    want = oracle.model_wave(2, c.pitch_m, c.lambda_m, c.xyz, c.amp, w, h).real
    got, _, names = _run(c, form, 2)
    assert "spherical" in names
    assert oracle.nrms(got, want) <= 1e-5
    # the result is the exact distance, not its Fresnel approximation (which differs by 3e-5 .. 1e-1 here)
    fres = oracle.model_wave(1, c.pitch_m, c.lambda_m, c.xyz, c.amp, w, h).real
    assert oracle.nrms(got, want) < 0.3 * oracle.nrms(got, fres)


def test_spherical_closed_form_branch():
    """Points 4-6 mm from a 160 x 160 hologram: u = r^2/z^2 reaches 0.13 and the remainder ~20 turns at the
    corners, beyond the quadratic's bounds, so every point takes the per-term form."""
    c = workloads.random_cloud(812, 160, 160, 400, z_range=(0.004, 0.006))
    mix = _remainder_forms(c)
    assert mix["term_series"] + mix["term_closed"] == 400, mix
    want = oracle.model_wave(2, c.pitch_m, c.lambda_m, c.xyz, c.amp, 160, 160).real
    got, _, _ = _run(c, "direct_sfu", 2)
    assert oracle.nrms(got, want) <= 1e-5


def _remainder_forms(c, tile_cols=8, tile_rows=8):
    """Which remainder form the point preparation selects per point for the amplitude hologram (thread tiles of
    8 rows x 8 columns; the same bounds, in FP64): the quadratic about each thread tile's centre or the per-term
    form, each with the series (u < 0.05) or the closed form."""
    x, y, z = (c.xyz[:, k].astype(np.float64) for k in range(3))
    qz, zh = (c.pitch_m / z) ** 2, z / (2 * c.lambda_m)
    hx, hy = (tile_cols - 1) / 2, (tile_rows - 1) / 2
    cx = np.maximum(np.abs(x), np.abs(c.width - 1 - x)) + hx
    cy = np.maximum(np.abs(y), np.abs(c.height - 1 - y)) + hy
    umax, wmax = (cx * cx + cy * cy) * qz, (2 * hx * cx + hx * hx + 2 * hy * cy + hy * hy) * qz
    quad = (zh * wmax ** 3 / 8 <= 2.0 ** -25) & (zh * umax / 2 * wmax + zh / 4 * wmax ** 2 <= 0.45)
    series = umax < 0.05
    return {"quad_series": int((quad & series).sum()), "quad_closed": int((quad & ~series).sum()),
            "term_series": int((~quad & series).sum()), "term_closed": int((~quad & ~series).sum())}


@pytest.mark.parametrize("wave", [False, True])
@pytest.mark.parametrize("w,h,n,z,forms", [
    (8192, 2048, 2000, (0.15, 0.3), ("quad_series", "quad_closed", "term_closed")),
    (1920, 1080, 2000, (0.05, 0.1), ("quad_series", "term_series", "term_closed"))])
def test_spherical_every_remainder_form(w, h, n, z, forms, wave):
    """Close points on wide holograms: each point's remainder takes the form its bounds allow (the amplitude
    hologram's 8 x 8 thread tiles; the complex wave's 4 x 4 tiles shift the mix); sampled pixels (corners
    included) against the oracle."""
    c = workloads.random_cloud(813 + w, w, h, n, z_range=z)
    mix = _remainder_forms(c)
    assert all(mix[f] >= 50 for f in forms), mix
    if wave:
        assert sum(v > 0 for v in _remainder_forms(c, tile_cols=4, tile_rows=4).values()) >= 3
    rng = np.random.default_rng(814)
    cols = np.concatenate([rng.integers(0, w, 400), [0, w - 1, 0, w - 1]])
    rows = np.concatenate([rng.integers(0, h, 400), [0, 0, h - 1, h - 1]])
    want = oracle.model_wave_at(2, c.pitch_m, c.lambda_m, c.xyz, c.amp, cols, rows)
    got, _, _ = _run(c, "direct_sfu", 2, wave=wave)
    assert oracle.nrms(got.real[rows, cols], want.real) <= 1e-5
    if wave:
        assert oracle.nrms(got.imag[rows, cols], want.imag) <= 1e-5


def test_spherical_wave_kinoform_and_reference():
    c = workloads.random_cloud(807, 330, 210, 1300, z_range=(0.2, 0.6))
    want = oracle.model_wave(2, c.pitch_m, c.lambda_m, c.xyz, c.amp, 330, 210, reference=REF)
    got, q, _ = _run(c, "direct_sfu", 2, REF, wave=True)
    assert oracle.nrms(got.real, want.real) <= 1e-5
    assert oracle.nrms(got.imag, want.imag) <= 1e-5
    k = oracle.kinoform8(want)
    psi = np.mod(np.angle(want), 2 * np.pi) * 255.0 / (2 * np.pi)
    rel = np.abs(got - want) / np.maximum(np.abs(want), 1e-30)
    delta = 255.0 / (2 * np.pi) * (rel + 1e-6) + 1e-4
    ties = (np.abs(psi - np.round(psi)) <= delta) | (psi > 255.0 - delta) | (psi < delta)
    assert not np.any((q != k) & ~ties)
    assert ties.mean() < 0.02


@pytest.mark.parametrize("split", [1, 3])
def test_spherical_point_splits(split):
    c = workloads.random_cloud(808, 200, 100, 2000, z_range=(0.3, 0.8))
    want = oracle.model_wave(2, c.pitch_m, c.lambda_m, c.xyz, c.amp, 200, 100).real
    got, _, _ = _run(c, "direct_sfu", 2, opts={_lib.CGH_OPT_POINT_SPLIT: split})
    assert oracle.nrms(got, want) <= 1e-5


def test_spherical_display_size_sampled():
    """1920x1080, 10^4 points (z ~ U[0.3, 1.0] m): sampled pixels of Eq. 1 against the oracle."""
    c = workloads.display_direct()
    rng = np.random.default_rng(809)
    cols = np.concatenate([rng.integers(0, 1920, 300), [0, 1919, 0, 1919]])
    rows = np.concatenate([rng.integers(0, 1080, 300), [0, 0, 1079, 1079]])
    want = oracle.model_wave_at(2, c.pitch_m, c.lambda_m, c.xyz, c.amp, cols, rows).real
    got, _, _ = _run(c, "direct_sfu", 2)
    assert oracle.nrms(got[rows, cols], want) <= 1e-5


@pytest.mark.parametrize("form", ["direct_accurate", "gemm_f16", "gemm_split16"])
def test_spherical_other_forms_not_supported(form):
    c = workloads.random_cloud(810, 64, 64, 100)
    with Hologram(64, 64, c.pitch_m, c.lambda_m, form=form) as h:
        h.set_phase_model("spherical")
        xyz, amp = torch.from_numpy(c.xyz).cuda(), torch.from_numpy(c.amp).cuda()
        out = torch.empty((64, 64), device="cuda")
        assert _lib.cgh_point_cloud(h.ctx, xyz.data_ptr(), amp.data_ptr(), 100, out.data_ptr()) == _lib.CGH_ENOTSUP


def test_batch_rejects_models_and_reference():
    c = workloads.random_cloud(811, 64, 64, 100)
    xyz, amp = torch.from_numpy(c.xyz).cuda(), torch.from_numpy(c.amp).cuda()
    out = torch.empty((64, 64), device="cuda")
    inst = (_lib.cgh_instance * 1)()
    inst[0].width, inst[0].height, inst[0].pitch_m, inst[0].lambda_m = 64, 64, c.pitch_m, c.lambda_m
    inst[0].d_xyz, inst[0].d_amp, inst[0].n_points, inst[0].d_out = xyz.data_ptr(), amp.data_ptr(), 100, out.data_ptr()
    for setup in (lambda h: h.set_phase_model("fresnel_piston"), lambda h: h.set_reference(0.01, 0.0, 0.0)):
        with Hologram(64, 64, c.pitch_m, c.lambda_m) as h:
            setup(h)
            assert _lib.load().cgh_batch(h.ctx, inst, 1) == _lib.CGH_ENOTSUP


def test_reference_argument_checks():
    with Hologram(16, 16, 8e-6, 532e-9) as h:
        for bad in ((1.5, 0.0, 0.0), (0.0, float("nan"), 0.0), (0.0, 0.0, float("inf"))):
            assert _lib.load().cgh_set_reference(h.ctx, *bad) == _lib.CGH_EINVAL
        assert _lib.load().cgh_set_option(h.ctx, _lib.CGH_OPT_PHASE_MODEL, 3) == _lib.CGH_EINVAL
