"""Parity of the direct form (prep + direct kernel + chunk reduction) and of
the quantiser against the FP64 oracle, through the C ABI on the GPU.

Tolerances (NRMS = ||I_gpu - I_ref|| / ||I_ref||): 1e-5 for the FP32 direct
forms.  Per pixel the error may not exceed 1e-5 * sqrt(sum_j A_j^2), the RMS
size of a pixel of a random-phase sum times ~1.4e-5.
"""
import math

import numpy as np
import pytest

import oracle
from paper_1309_2734_gb300 import CghError, Hologram, workloads
from paper_1309_2734_gb300 import _lib

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")

NRMS_DIRECT = 1e-5


@pytest.fixture(scope="module", autouse=True)
def _built():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1309_2734_gb300.build import build
    build()
    torch.cuda.set_device(0)


def _dev(c):
    return torch.from_numpy(c.xyz).cuda(), torch.from_numpy(c.amp).cuda()


def _run(c, form, split=None, xyz=None, amp=None, timeout_ms=None):
    if xyz is None:
        xyz, amp = _dev(c)
    with Hologram(c.width, c.height, c.pitch_m, c.lambda_m, form=form, timeout_ms=timeout_ms) as h:
        if split:
            h.set_option(_lib.CGH_OPT_POINT_SPLIT, split)
        f = h.point_cloud(xyz, amp)
        h.sync()
        return f.cpu().numpy()


def _check(got, ref, amp, tol=NRMS_DIRECT):
    err = oracle.nrms(got, ref)
    assert err <= tol, f"NRMS {err:.3e} > {tol:.1e}"
    per_pixel = 1e-5 * math.sqrt(float(np.sum(amp.astype(np.float64) ** 2)))
    worst = float(np.max(np.abs(got.astype(np.float64) - ref))) if ref.size else 0.0
    assert worst <= per_pixel, f"max abs error {worst:.3e} > {per_pixel:.3e}"
    return err


@pytest.mark.parametrize("form", ["direct_sfu", "direct_accurate"])
def test_small_direct_full_field(form):
    c = workloads.small_direct()
    ref = oracle.field(c.pitch_m, c.lambda_m, c.xyz, c.amp, c.width, c.height)
    _check(_run(c, form), ref, c.amp)


@pytest.mark.parametrize("form", ["direct_sfu", "direct_accurate"])
@pytest.mark.parametrize("w,h,n", [(1, 1, 1), (257, 33, 300), (300, 37, 513), (31, 300, 256),
                                   (1000, 3, 77), (258, 35, 1)])
def test_ragged_shapes(form, w, h, n):
    c = workloads.random_cloud(1000 + w + n, w, h, n)
    ref = oracle.field(c.pitch_m, c.lambda_m, c.xyz, c.amp, w, h)
    _check(_run(c, form), ref, c.amp)


def test_points_outside_the_hologram_and_negative_coordinates():
    rng = np.random.default_rng(11)
    n = 400
    xyz = np.stack([rng.integers(-16384, 16385, n), rng.integers(-16384, 16385, n),
                    rng.uniform(0.05, 2.0, n)], 1).astype(np.float32)
    xyz[:4, :2] = [[-16384, -16384], [16384, 16384], [-16384, 16384], [0, 0]]
    amp = rng.uniform(-1.0, 1.0, n).astype(np.float32)
    c = workloads.Cloud(96, 80, 8e-6, 532e-9, xyz, amp, "far")
    ref = oracle.field(c.pitch_m, c.lambda_m, xyz, amp, 96, 80)
    for form in ("direct_sfu", "direct_accurate"):
        _check(_run(c, form), ref, amp)


@pytest.mark.parametrize("w,h", [(16384, 3), (3, 16384)])
def test_longest_side(w, h):
    """The longest side accepted (16384 pixels), points at both ends of the coordinate range (|x|, |y| = 16384,
    so distances reach 32767 pixels): direct and split-FP16 GEMM forms against the oracle; one more pixel is
    refused."""
    rng = np.random.default_rng(49)
    n = 300
    xyz = np.stack([rng.integers(0, w, n), rng.integers(0, h, n), rng.uniform(0.3, 1.0, n)], 1).astype(np.float32)
    xyz[:4, :2] = [[-16384, -16384], [16384, 16384], [-16384, 16384], [16384, -16384]]
    amp = rng.uniform(0.5, 1.0, n).astype(np.float32)
    c = workloads.Cloud(w, h, 8e-6, 532e-9, xyz, amp, "longest side")
    ref = oracle.field(c.pitch_m, c.lambda_m, xyz, amp, w, h)
    _check(_run(c, "direct_sfu"), ref, amp)
    assert oracle.nrms(_run(c, "gemm_split16"), ref) <= 1e-5
    with pytest.raises(CghError):
        Hologram(w + (w > h), h + (h > w), c.pitch_m, c.lambda_m)


def test_empty_cloud_writes_zeros():
    c = workloads.random_cloud(1, 70, 50, 0)
    with Hologram(70, 50, c.pitch_m, c.lambda_m, form="direct_sfu") as h:
        out = torch.full((50, 70), 7.0, device="cuda")
        h.point_cloud(torch.zeros((0, 3), device="cuda"), torch.zeros(0, device="cuda"), out=out)
        h.sync()
        assert torch.count_nonzero(out).item() == 0


@pytest.mark.parametrize("split", [2, 3, 7])
def test_point_split_matches_oracle(split):
    c = workloads.random_cloud(44, 300, 70, 2000)
    ref = oracle.field(c.pitch_m, c.lambda_m, c.xyz, c.amp, c.width, c.height)
    got = _run(c, "direct_sfu", split=split)
    _check(got, ref, c.amp)
    one = _run(c, "direct_sfu", split=1)
    assert oracle.nrms(got, one) < 2e-7


@pytest.mark.parametrize("split", [1, 3, 0])
def test_tall_cta_shape_with_point_splits(split):
    """640 x 64 takes the tall CTA shape (128 x 64-pixel tiles, 5 of them, against 6 wide ones): the whole field
    against the oracle, at forced and automatic point splits, and the same sums whatever the split."""
    c = workloads.random_cloud(47, 640, 64, 3000)
    ref = oracle.field(c.pitch_m, c.lambda_m, c.xyz, c.amp, c.width, c.height)
    got = _run(c, "direct_sfu", split=split)
    _check(got, ref, c.amp)
    assert oracle.nrms(got, _run(c, "direct_sfu", split=1)) < 2e-7


def test_deterministic():
    c = workloads.random_cloud(45, 333, 91, 3000)
    a = _run(c, "direct_sfu")
    b = _run(c, "direct_sfu")
    assert np.array_equal(a, b)


def test_display_size_sampled():
    """1920x1080, 10^4 points, in the launch configuration the benchmark times."""
    c = workloads.display_direct()
    rng = np.random.default_rng(5)
    cols = np.concatenate([rng.integers(0, 1920, 400), [0, 1919, 0, 1919, 1792, 1919]])
    rows = np.concatenate([rng.integers(0, 1080, 400), [0, 0, 1079, 1079, 1056, 1056]])
    ref = oracle.field_at(c.pitch_m, c.lambda_m, c.xyz, c.amp, cols, rows)
    for form in ("direct_sfu", "direct_accurate"):
        got = _run(c, form)
        _check(got[rows, cols], ref, c.amp)


@pytest.fixture(scope="module")
def layered():
    c = workloads.large_layered()
    rng = np.random.default_rng(6)
    cols = rng.integers(0, 4096, 48)
    rows = rng.integers(0, 4096, 48)
    return c, cols, rows, oracle.field_at(c.pitch_m, c.lambda_m, c.xyz, c.amp, cols, rows)


@pytest.mark.parametrize("form", ["direct_sfu", "direct_accurate"])
def test_layered_million_points_sampled(layered, form):
    """4096x4096, 10^6 points on 16 depth planes: sampled pixels vs the oracle.

    At this N a per-term bias of 1e-8 would already show as NRMS ~1e-5, so
    the mean error is checked as well as the NRMS.
    """
    c, cols, rows, ref = layered
    got = _run(c, form, timeout_ms=120000)[rows, cols].astype(np.float64)
    bias = float(np.mean(got - ref))
    assert abs(bias) < 3e-6 * math.sqrt(float(np.sum(c.amp.astype(np.float64) ** 2))), bias
    _check(got, ref, c.amp)


@pytest.mark.parametrize("bad", ["z0", "zneg", "nan", "frac", "range", "ampnan"])
def test_bad_points_are_reported(bad):
    c = workloads.random_cloud(3, 64, 64, 100)
    xyz, amp = c.xyz.copy(), c.amp.copy()
    if bad == "z0":
        xyz[10, 2] = 0.0
    elif bad == "zneg":
        xyz[10, 2] = -0.5
    elif bad == "nan":
        xyz[10, 0] = np.nan
    elif bad == "frac":
        xyz[10, 1] = 3.5
    elif bad == "range":
        xyz[10, 0] = 16385
    else:
        amp[10] = np.inf
    with Hologram(64, 64, c.pitch_m, c.lambda_m, form="direct_sfu") as h:
        h.point_cloud(torch.from_numpy(xyz).cuda(), torch.from_numpy(amp).cuda())
        with pytest.raises(CghError) as ei:
            h.sync()
        assert ei.value.code == _lib.CGH_EINPUT
        # the status is cleared and the context stays usable
        xg, ag = _dev(c)
        f = h.point_cloud(xg, ag)
        h.sync()
        ref = oracle.field(c.pitch_m, c.lambda_m, c.xyz, c.amp, 64, 64)
        _check(f.cpu().numpy(), ref, c.amp)


def test_host_buffer_entry_point():
    c = workloads.random_cloud(12, 128, 96, 600)
    ref = oracle.field(c.pitch_m, c.lambda_m, c.xyz, c.amp, 128, 96)
    out = torch.empty((96, 128), dtype=torch.float32).pin_memory()
    with Hologram(128, 96, c.pitch_m, c.lambda_m, form="direct_sfu") as h:
        h.point_cloud_host(torch.from_numpy(c.xyz), torch.from_numpy(c.amp), out)
    _check(out.numpy(), ref, c.amp)


# ---- quantiser -------------------------------------------------------------

def _q_gpu(field_np, offset=0):
    buf = torch.zeros(field_np.size + offset, dtype=torch.float32, device="cuda")
    buf[offset:] = torch.from_numpy(field_np.reshape(-1)).cuda()
    out = torch.zeros(field_np.size + offset, dtype=torch.uint8, device="cuda")
    with Hologram(8, 8, 8e-6, 532e-9) as h:
        rc = _lib.cgh_quantize8(h.ctx, buf[offset:].data_ptr(), field_np.size, 0, out[offset:].data_ptr())
        assert rc == 0
        h.sync()
    return out[offset:].cpu().numpy()


@pytest.mark.parametrize("n,offset", [(65536, 0), (1000, 0), (1000, 1), (17, 3), (1, 0)])
def test_quantize_bit_exact_on_same_field(n, offset):
    rng = np.random.default_rng(n + offset)
    f = (rng.standard_normal(n) * 50).astype(np.float32)
    want, _ = oracle.quantize8(f)
    assert np.array_equal(_q_gpu(f, offset), want)


def test_quantize_special_fields():
    f = np.full(100, 3.25, np.float32)
    assert np.all(_q_gpu(f) == 0)
    k = np.arange(256, dtype=np.float64)
    v = (k / 256.0).astype(np.float32)
    assert np.array_equal(_q_gpu(v), np.arange(256, dtype=np.uint8))
    g = np.linspace(-1, 1, 999).astype(np.float32)
    g[[3, 500]] = np.nan
    want, _ = oracle.quantize8(g)
    assert np.array_equal(_q_gpu(g), want)


def test_quantize_hologram_vs_oracle_quantisation():
    """uint8 of the GPU field equals the oracle's quantisation of the FP64 field away from ties."""
    c = workloads.small_direct()
    ref = oracle.field(c.pitch_m, c.lambda_m, c.xyz, c.amp, c.width, c.height)
    got = _run(c, "direct_sfu")
    with Hologram(8, 8, 8e-6, 532e-9) as h:
        q = h.quantize8(torch.from_numpy(got).cuda())
        h.sync()
    q = q.cpu().numpy()
    assert np.array_equal(q, oracle.quantize8(got)[0])
    ref32 = ref.astype(np.float32)
    qr, (lo, hi, s) = oracle.quantize8(ref32)
    scaled = (ref.astype(np.float64) - lo) * s
    delta = (np.max(np.abs(got.astype(np.float64) - ref)) + abs(float(got.min()) - lo)) * s + 2.0 ** -20 + \
        np.abs(ref32.astype(np.float64) - ref).max() * s
    ties = np.abs(scaled - np.round(scaled)) <= delta
    mism = q != qr
    assert not np.any(mism & ~ties)
    assert ties.mean() < 0.01


@pytest.mark.parametrize("w,h,n", [(300, 70, 2000), (1920, 1080, 777), (129, 65, 3), (640, 200, 4099)])
def test_balanced_split_cta_counts_and_determinism(w, h, n):
    """The SFU form's default layout: equal shares of the (pixel tile, point) pairs per CTA, a tile's parts
    summed by the last CTA to finish it.  Two runs give the same bits; other CTA counts (other part boundaries,
    so other single-precision rounding: O(eps sqrt(N)) relative) agree within 1e-6; the result meets the oracle
    and agrees with the chunked layout within 1e-6."""
    c = workloads.random_cloud(4400 + n, w, h, n)
    xyz, amp = _dev(c)
    outs = []
    for ctas in (0, 0, 97, 1):
        with Hologram(w, h, c.pitch_m, c.lambda_m, form="direct_sfu") as hg:
            hg.set_option(_lib.CGH_OPT_DIRECT_CTAS, ctas)
            f = hg.point_cloud(xyz, amp)
            hg.sync()
            outs.append(f.cpu().numpy())
    assert np.array_equal(outs[0], outs[1])
    for other in outs[2:]:
        assert oracle.nrms(outs[0], other) < 1e-6
    if w * h * n <= 2e8:
        ref = oracle.field(c.pitch_m, c.lambda_m, c.xyz, c.amp, w, h)
        _check(outs[0], ref, c.amp)
    chunked = _run(c, "direct_sfu", split=3)
    assert oracle.nrms(outs[0], chunked) < 1e-6


@pytest.mark.parametrize("shape", [1, 2, 3, 4, 5, 6])
@pytest.mark.parametrize("w,h,n", [(300, 70, 2000), (515, 129, 301)])
def test_balanced_layout_every_thread_block(shape, w, h, n):
    """CGH_OPT_DIRECT_SHAPE: 8 x 4 pixels a thread in 32 x 8 or 16 x 16 threads (totals in registers), 8 x 8 in
    16 x 8 or 32 x 4 (totals in shared memory), 8 x 4 in 16 x 16 or 32 x 8 with the CTA's tables of the column and
    row sines; ragged in both directions, against the oracle, and within single-precision rounding of one another
    (the same terms in the same point order)."""
    c = workloads.random_cloud(4600 + n, w, h, n)
    xyz, amp = _dev(c)
    with Hologram(w, h, c.pitch_m, c.lambda_m, form="direct_sfu") as hg:
        hg.set_option(_lib.CGH_OPT_DIRECT_SHAPE, shape)
        got = hg.point_cloud(xyz, amp)
        hg.sync()
        got = got.cpu().numpy()
    ref = oracle.field(c.pitch_m, c.lambda_m, c.xyz, c.amp, w, h)
    _check(got, ref, c.amp)
    assert oracle.nrms(got, _run(c, "direct_sfu")) < 1e-6


def test_sfu_error_does_not_grow_with_points():
    """The separable SFU evaluation alternates a half turn between points so that the hardware cosine's mean error
    cancels: the field's NRMS stays at the 10^4-point level with 2 10^5 points (it grew 3.4x without)."""
    errs = []
    for n in (10000, 200000):
        c = workloads.random_cloud(4700, 640, 360, n)
        xyz, amp = _dev(c)
        with Hologram(640, 360, c.pitch_m, c.lambda_m, form="direct_sfu") as hg:
            got = hg.point_cloud(xyz, amp)
            hg.sync()
            got = got.cpu().numpy()
        rng = np.random.default_rng(12)
        cols, rows = rng.integers(0, 640, 500), rng.integers(0, 360, 500)
        ref = oracle.field_at(c.pitch_m, c.lambda_m, c.xyz, c.amp, cols, rows)
        errs.append(oracle.nrms(got[rows, cols], ref))
    assert errs[0] < 1.5e-6
    assert errs[1] < 1.5 * errs[0] + 3e-7, errs


def test_balanced_split_wait_times_out_and_context_recovers():
    """The default layout with a point tile that CTA 0 never loads (test hook): the bounded wait runs out, the
    launch ends with a timeout status, no other CTA waits on the missing part, and the context keeps working."""
    c = workloads.random_cloud(47, 300, 100, 1000)
    xyz, amp = _dev(c)
    with Hologram(c.width, c.height, c.pitch_m, c.lambda_m, form="direct_sfu", timeout_ms=300) as h:
        h.set_option(_lib.CGH_OPT_TEST_DROP_TILE, 0)
        h.point_cloud(xyz, amp)
        with pytest.raises(CghError) as ei:
            h.sync()
        assert ei.value.code == _lib.CGH_ETIMEOUT
        h.set_option(_lib.CGH_OPT_TEST_DROP_TILE, -1)
        f = h.point_cloud(xyz, amp)
        h.sync()
    ref = oracle.field(c.pitch_m, c.lambda_m, c.xyz, c.amp, c.width, c.height)
    _check(f.cpu().numpy(), ref, c.amp)


def test_device_wait_times_out_and_context_recovers():
    """A point tile that is never loaded (host-side test hook): the kernel's bounded
    wait runs out, the launch ends with a timeout status, and the context keeps working."""
    c = workloads.random_cloud(46, 300, 100, 1000)
    xyz, amp = _dev(c)
    with Hologram(c.width, c.height, c.pitch_m, c.lambda_m, form="direct_sfu", timeout_ms=300) as h:
        h.set_option(_lib.CGH_OPT_POINT_SPLIT, 1)
        h.set_option(_lib.CGH_OPT_TEST_DROP_TILE, 1)
        h.point_cloud(xyz, amp)
        with pytest.raises(CghError) as ei:
            h.sync()
        assert ei.value.code == _lib.CGH_ETIMEOUT
        h.set_option(_lib.CGH_OPT_TEST_DROP_TILE, -1)
        f = h.point_cloud(xyz, amp)
        h.sync()
    ref = oracle.field(c.pitch_m, c.lambda_m, c.xyz, c.amp, c.width, c.height)
    _check(f.cpu().numpy(), ref, c.amp)


def test_measured_mufu_rate_is_plausible():
    """The hardware-sine probe behind the roofline: within (0.5, 1.1) x 16 results/clk/SM x SMs x max clock."""
    props = torch.cuda.get_device_properties(0)
    with Hologram(8, 8, 8e-6, 532e-9) as h:
        r = _lib.cgh_measure_mufu(h.ctx)
    nominal = 16 * props.multi_processor_count * 2.07e9
    assert 0.5 * nominal < r < 1.1 * nominal, r
