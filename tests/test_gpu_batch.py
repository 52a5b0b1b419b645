"""Batched holograms (one persistent launch for the whole batch, or per-kind
launches, captured in a CUDA graph) and the autotuner, through the C ABI,
against the FP64 oracle."""
import numpy as np
import pytest

import oracle
from paper_1309_2734_gb300 import CghError, Hologram, batch, workloads
from paper_1309_2734_gb300 import _lib

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")

NRMS = {"direct_sfu": 1e-5, "direct_accurate": 1e-5, "gemm_f16": 2e-3, "gemm_bf16": 1e-2, "gemm_split16": 1e-5}


@pytest.fixture(scope="module", autouse=True)
def _built():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1309_2734_gb300.build import build
    build()
    torch.cuda.set_device(0)


def _clouds():
    return [workloads.random_cloud(700, 300, 200, 1500), workloads.random_cloud(701, 128, 130, 300),
            workloads.random_cloud(702, 257, 65, 0), workloads.random_cloud(703, 500, 120, 2100),
            workloads.random_cloud(704, 64, 64, 5)]


def _dev(clouds):
    return [(torch.from_numpy(c.xyz).cuda(), torch.from_numpy(c.amp).cuda(), c.width, c.height, c.pitch_m,
             c.lambda_m) for c in clouds]


def _check_all(clouds, outs, tol):
    for c, o in zip(clouds, outs):
        got = o.cpu().numpy()
        if c.n_points == 0:
            assert np.count_nonzero(got) == 0
            continue
        ref = oracle.field(c.pitch_m, c.lambda_m, c.xyz, c.amp, c.width, c.height)
        assert oracle.nrms(got, ref) <= tol, (c.name, oracle.nrms(got, ref))


@pytest.mark.parametrize("mode", [0, 1])
@pytest.mark.parametrize("form", ["direct_sfu", "direct_accurate", "gemm_f16", "gemm_bf16", "gemm_split16"])
def test_batch_each_form_vs_oracle(form, mode):
    """Every form through the persistent launch (mode 0) and the per-kind launches (mode 1)."""
    clouds = _clouds()
    dev = _dev(clouds)
    outs = [torch.full((c.height, c.width), 5.0, device="cuda") for c in clouds]
    with Hologram(8, 8, 8e-6, 532e-9, form=form, timeout_ms=5000) as h:
        h.set_option(_lib.CGH_OPT_BATCH_MODE, mode)
        batch(h, dev, outs)
        h.sync()
        assert _lib.cgh_batch_forms(h.ctx)[:2] == [getattr(_lib, "CGH_" + form.upper())] * 2
    _check_all(clouds, outs, NRMS[form])


def _mixed_clouds():
    # direct jobs of several point chunks (their parts are folded), ragged shapes, an empty instance
    return [workloads.random_cloud(720, 300, 200, 5000), workloads.random_cloud(721, 1000, 70, 700),
            workloads.random_cloud(722, 130, 257, 9000), workloads.random_cloud(723, 64, 64, 0),
            workloads.random_cloud(724, 513, 129, 3)]


@pytest.mark.parametrize("form", ["direct_sfu", "direct_accurate", "gemm_split16"])
def test_persistent_batch_is_deterministic_and_matches_kinds(form):
    """Two replays of the persistent launch give the same bits (the parts of a direct tile are summed in chunk
    order, whoever finishes last); the per-kind launches agree within single-precision rounding."""
    clouds = _mixed_clouds()
    dev = _dev(clouds)
    outs = [torch.full((c.height, c.width), 3.0, device="cuda") for c in clouds]
    with Hologram(8, 8, 8e-6, 532e-9, form=form) as h:
        batch(h, dev, outs)
        h.sync()
        first = [o.clone() for o in outs]
        batch(h, dev, outs)
        h.sync()
        for a, b in zip(first, outs):
            assert torch.equal(a, b)
        h.set_option(_lib.CGH_OPT_BATCH_MODE, 1)
        batch(h, dev, outs)
        h.sync()
    for c, a, b in zip(clouds, first, outs):
        if c.n_points:
            assert oracle.nrms(a.cpu().numpy(), b.cpu().numpy()) < 1e-6
    _check_all(clouds, first, NRMS[form])


@pytest.mark.parametrize("form", ["gemm_f16", "gemm_split16"])
def test_persistent_batch_k_chunks(form):
    """CGH_OPT_BATCH_CHUNK_MB: GEMM units of short K chunks whose results reach each tile in K order (sequence
    flags), against the default units (here: the K splits of a batch with few tiles) -- other summation order,
    equal within single-precision rounding -- and bit-equal on a replay."""
    clouds = _mixed_clouds()
    dev = _dev(clouds)
    outs = [torch.full((c.height, c.width), 2.0, device="cuda") for c in clouds]
    with Hologram(8, 8, 8e-6, 532e-9, form=form) as h:
        batch(h, dev, outs)
        h.sync()
        plain = [o.clone() for o in outs]
        h.set_option(_lib.CGH_OPT_BATCH_CHUNK_MB, 1)
        batch(h, dev, outs)
        h.sync()
        first = [o.clone() for o in outs]
        batch(h, dev, outs)
        h.sync()
    for c, a, b, p in zip(clouds, first, outs, plain):
        assert torch.equal(a, b)
        if c.n_points:
            assert oracle.nrms(a.cpu().numpy(), p.cpu().numpy()) < (3e-6 if form == "gemm_split16" else 2e-4)
    _check_all(clouds, first, NRMS[form])


@pytest.mark.parametrize("pct", [40, 100])
def test_persistent_batch_premade_factors(pct):
    """CGH_OPT_BATCH_PREMADE_PCT: the first GEMM jobs' points and factors come from the plain kernels before the
    persistent launch (the same device functions as the SIMT units, so the same bits)."""
    clouds = _mixed_clouds()
    dev = _dev(clouds)
    outs = [torch.full((c.height, c.width), 2.0, device="cuda") for c in clouds]
    with Hologram(8, 8, 8e-6, 532e-9, form="gemm_split16") as h:
        batch(h, dev, outs)
        h.sync()
        plain = [o.clone() for o in outs]
        h.set_option(_lib.CGH_OPT_BATCH_PREMADE_PCT, pct)
        batch(h, dev, outs)
        h.sync()
    for a, b in zip(plain, outs):
        assert torch.equal(a, b)
    _check_all(clouds, outs, NRMS["gemm_split16"])


@pytest.mark.parametrize("form", ["direct_sfu", "gemm_f16"])
def test_persistent_batch_wait_times_out_and_context_recovers(form):
    """Test hook: the first job waits for one unit more than exists, so its bounded wait runs out; the launch
    ends with a timeout status instead of hanging, and the next plan (hook off) computes the batch."""
    clouds = _clouds()
    dev = _dev(clouds)
    outs = [torch.zeros((c.height, c.width), device="cuda") for c in clouds]
    with Hologram(8, 8, 8e-6, 532e-9, form=form, timeout_ms=300) as h:
        h.set_option(_lib.CGH_OPT_TEST_DROP_TILE, 0)
        batch(h, dev, outs)
        with pytest.raises(CghError) as ei:
            h.sync()
        assert ei.value.code == _lib.CGH_ETIMEOUT
        h.set_option(_lib.CGH_OPT_TEST_DROP_TILE, -1)
        batch(h, dev, outs)
        h.sync()
    _check_all(clouds, outs, NRMS[form])


def test_batch_replays_graph_on_new_data():
    clouds = _clouds()
    dev = _dev(clouds)
    outs = [torch.zeros((c.height, c.width), device="cuda") for c in clouds]
    with Hologram(8, 8, 8e-6, 532e-9, form="gemm_split16") as h:
        batch(h, dev, outs)
        h.sync()
        first = [o.clone() for o in outs]
        batch(h, dev, outs)                    # same plan: graph replay
        h.sync()
        for a, b in zip(first, outs):
            assert torch.equal(a, b)
        # new point data in the same buffers: the replay recomputes
        fresh = [workloads.random_cloud(800 + i, c.width, c.height, c.n_points) for i, c in enumerate(clouds)]
        for (xyz, amp, *_), c in zip(dev, fresh):
            xyz.copy_(torch.from_numpy(c.xyz))
            amp.copy_(torch.from_numpy(c.amp))
        batch(h, dev, outs)
        h.sync()
    _check_all(fresh, outs, NRMS["gemm_split16"])


def test_batch_matches_single_calls():
    clouds = _clouds()
    dev = _dev(clouds)
    outs = [torch.zeros((c.height, c.width), device="cuda") for c in clouds]
    with Hologram(8, 8, 8e-6, 532e-9, form="direct_sfu") as h:
        batch(h, dev, outs)
        h.sync()
    for c, (xyz, amp, *_), o in zip(clouds, dev, outs):
        with Hologram(c.width, c.height, c.pitch_m, c.lambda_m, form="direct_sfu") as h1:
            one = h1.point_cloud(xyz, amp)
            h1.sync()
        assert oracle.nrms(o.cpu().numpy(), one.cpu().numpy()) < 1e-6 or c.n_points == 0


@pytest.mark.parametrize("tol_e9,allowed", [(10000, {"direct_sfu", "direct_accurate", "gemm_split16"}),
                                            (10_000_000, set(NRMS))])
def test_autotuned_batch_meets_tolerance(tol_e9, allowed):
    clouds = _clouds()
    dev = _dev(clouds)
    outs = [torch.zeros((c.height, c.width), device="cuda") for c in clouds]
    with Hologram(8, 8, 8e-6, 532e-9, form="auto") as h:
        assert _lib.cgh_autotune(h.ctx, False) == _lib.CGH_OK
        h.set_option(_lib.CGH_OPT_TOLERANCE_E9, tol_e9)
        batch(h, dev, outs)
        h.sync()
    _check_all(clouds, outs, tol_e9 * 1e-9)


def test_auto_single_hologram_meets_tolerance():
    c = workloads.random_cloud(710, 640, 360, 6000)
    xyz, amp = torch.from_numpy(c.xyz).cuda(), torch.from_numpy(c.amp).cuda()
    with Hologram(c.width, c.height, c.pitch_m, c.lambda_m, form="auto") as h:
        f = h.point_cloud(xyz, amp)
        h.sync()
    ref = oracle.field(c.pitch_m, c.lambda_m, c.xyz, c.amp, c.width, c.height)
    assert oracle.nrms(f.cpu().numpy(), ref) <= 1e-5


@pytest.mark.parametrize("tol_e9", [10000, 2_000_000])
def test_video_batch_64_frames_sampled(tol_e9):
    """64 frames of uneven size (1024^2 / 1920x1080 / 3840x2160, 10^3..2x10^5 points), one
    batch call at NRMS 1e-5 and at 2e-3 (autotuned forms), sampled pixels of every frame vs the oracle."""
    frames = workloads.video_batch()
    dev = _dev(frames)
    outs = [torch.empty((c.height, c.width), device="cuda") for c in frames]
    with Hologram(8, 8, 8e-6, 532e-9, form="auto", timeout_ms=20000) as h:
        h.set_option(_lib.CGH_OPT_TOLERANCE_E9, tol_e9)
        batch(h, dev, outs)
        h.sync()
    rng = np.random.default_rng(64)
    for c, o in zip(frames, outs):
        cols = rng.integers(0, c.width, 24)
        rows = rng.integers(0, c.height, 24)
        ref = oracle.field_at(c.pitch_m, c.lambda_m, c.xyz, c.amp, cols, rows)
        got = o[torch.from_numpy(rows).cuda(), torch.from_numpy(cols).cuda()].cpu().numpy()
        assert oracle.nrms(got, ref) <= tol_e9 * 1e-9, c.name
