"""Parity of the separable tensor-core form: factor generation (cgh_factors)
against the oracle's FP64 factors, the tcgen05 GEMM against a plain PyTorch
FP32 matmul of the very same 16-bit operands, and the whole GEMM form
against the FP64 oracle field.

NRMS tolerances of the GEMM forms against the oracle: 2e-3 (FP16), 1e-2
(BF16), 1e-5 (split hi+lo FP16).
"""
import math

import numpy as np
import pytest

import oracle
from paper_1309_2734_gb300 import Hologram, workloads
from paper_1309_2734_gb300 import _lib

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")

NRMS = {"gemm_f16": 2e-3, "gemm_bf16": 1e-2, "gemm_split16": 1e-5}


@pytest.fixture(scope="module", autouse=True)
def _built():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1309_2734_gb300.build import build
    build()
    torch.cuda.set_device(0)


def _dev(c):
    return torch.from_numpy(c.xyz).cuda(), torch.from_numpy(c.amp).cuda()


def _run(c, form, bn=None, splitk=None, chunk=None, budget_mb=None, trans=None, pair=None):
    xyz, amp = _dev(c)
    with Hologram(c.width, c.height, c.pitch_m, c.lambda_m, form=form, timeout_ms=3000) as h:
        if pair:
            h.set_option(_lib.CGH_OPT_GEMM_PAIR, pair)
        if trans:
            h.set_option(_lib.CGH_OPT_GEMM_TRANSPOSE, trans)
        if budget_mb:
            h.set_option(_lib.CGH_OPT_FACTOR_BUDGET_MB, budget_mb)
        if bn:
            h.set_option(_lib.CGH_OPT_GEMM_BN, bn)
        if splitk:
            h.set_option(_lib.CGH_OPT_GEMM_SPLITK, splitk)
        if chunk:
            h.set_option(_lib.CGH_OPT_GEMM_CHUNK, chunk)
        f = h.point_cloud(xyz, amp)
        h.sync()
        return f.cpu().numpy()


# ---- a3: factors -----------------------------------------------------------

@pytest.mark.parametrize("form", ["gemm_f16", "gemm_bf16", "gemm_split16"])
def test_factors_match_fp64_oracle(form):
    c = workloads.random_cloud(31, 70, 45, 150)
    Pr, Qr = oracle.factors(c.pitch_m, c.lambda_m, c.xyz, c.amp, c.width, c.height)
    xyz, amp = _dev(c)
    with Hologram(c.width, c.height, c.pitch_m, c.lambda_m) as h:
        P, Q = h.factors(xyz, amp, form)
        h.sync()
    k = 2 * c.n_points
    if form == "gemm_split16":
        Pg = (P[0].float() + P[1].float()).cpu().numpy().astype(np.float64)
        Qg = (Q[0].float() + Q[1].float()).cpu().numpy().astype(np.float64)
        pad_p, pad_q = P[:, :, k:], Q[:, :, k:]
        rel, floor = 2.0 ** -21, 6e-7
    else:
        Pg = P.float().cpu().numpy().astype(np.float64)
        Qg = Q.float().cpu().numpy().astype(np.float64)
        pad_p, pad_q = P[:, k:], Q[:, k:]
        # FP16 / BF16 factors walk the turn down a block's rows by the recurrence of Eqs. 6-8 (drift below
        # 31 * 32 / 2 = 496 units of 2^-32 turn) and convert its top 23 bits (rounding <= 2^-24 turn): the turn
        # is within 2^-24 + 496 * 2^-32 turn, 2 pi of that is 1.1e-6 rad
        rel = 2.0 ** -8 if form == "gemm_bf16" else 2.0 ** -11
        floor = 3.8e-7 + 2 * np.pi * (2.0 ** -24 + 496 * 2.0 ** -32)
    # floor: the hardware sine and cosine on [-pi, pi] (<= 3.8e-7) plus the turn's own error
    for got, ref in ((Pg[:, :k], Pr), (Qg[:, :k], Qr)):
        err = np.abs(got - ref)
        assert np.all(err <= rel * np.abs(ref) + floor), float(np.max(err - rel * np.abs(ref)))
    assert torch.count_nonzero(pad_p).item() == 0 and torch.count_nonzero(pad_q).item() == 0


# ---- a4: the GEMM kernel against an FP32 matmul of the same operands -------

@pytest.mark.parametrize("form", ["gemm_f16", "gemm_bf16", "gemm_split16"])
@pytest.mark.parametrize("shape", [(300, 200, 700), (1920, 131, 2048), (96, 260, 37)])
def test_gemm_matches_fp32_matmul_of_same_operands(form, shape):
    w, h, n = shape
    c = workloads.random_cloud(7 + w + n, w, h, n)
    c.amp[0] = 1.0            # max |A| = 1: the form's internal amplitude scale is exactly 1
    xyz, amp = _dev(c)
    with Hologram(w, h, c.pitch_m, c.lambda_m, form=form, timeout_ms=3000) as hh:
        P, Q = hh.factors(xyz, amp, form)
        f = hh.point_cloud(xyz, amp)
        hh.sync()
    P, Q = P.cpu().double(), Q.cpu().double()
    if form == "gemm_split16":
        ref = P[0] @ Q[0].t() + P[0] @ Q[1].t() + P[1] @ Q[0].t()
    else:
        ref = P @ Q.t()
    ref = ref.numpy()
    got = f.cpu().numpy().astype(np.float64)
    err = oracle.nrms(got, ref)
    # the tensor cores' own FP32 accumulation over a chain of 8 k-blocks (x3 passes
    # for split FP16) measured ~2.4e-6; an error in the kernel shows as >= 1e-3
    assert err < 5e-6, err


# ---- the whole form against the oracle ---------------------------------------

@pytest.mark.parametrize("form", ["gemm_f16", "gemm_bf16", "gemm_split16"])
@pytest.mark.parametrize("w,h,n", [(256, 256, 1024), (257, 129, 333), (130, 300, 64), (1, 1, 1), (1000, 3, 5)])
def test_gemm_form_vs_oracle(form, w, h, n):
    c = workloads.random_cloud(100 + w + h + n, w, h, n)
    ref = oracle.field(c.pitch_m, c.lambda_m, c.xyz, c.amp, w, h)
    got = _run(c, form)
    assert oracle.nrms(got, ref) <= NRMS[form]


@pytest.mark.parametrize("pair", [2, 1])
@pytest.mark.parametrize("bn", [128, 192, 224, 240, 256])
@pytest.mark.parametrize("splitk", [1, 2, 3, 5])
def test_tiles_and_splits(bn, splitk, pair):
    """Every tile width and a few K splits, in the one-CTA form (CGH_OPT_GEMM_PAIR 2) and the two-SM form (1; it
    has no 240-wide tile, where the one-CTA form runs)."""
    c = workloads.random_cloud(55, 500, 270, 1500)
    ref = oracle.field(c.pitch_m, c.lambda_m, c.xyz, c.amp, 500, 270)
    got = _run(c, "gemm_split16", bn=bn, splitk=splitk, pair=pair)
    assert oracle.nrms(got, ref) <= NRMS["gemm_split16"]


def test_split_results_agree_across_splits():
    """Same accumulation chunks, K split over 1 or 4 partial planes: only FP32 summation order differs."""
    c = workloads.random_cloud(56, 384, 256, 4096)
    a = _run(c, "gemm_f16", splitk=1, chunk=8)
    b = _run(c, "gemm_f16", splitk=4, chunk=8)
    assert oracle.nrms(b, a) < 1e-6
    assert np.array_equal(a, _run(c, "gemm_f16", splitk=1, chunk=8))     # deterministic


@pytest.mark.parametrize("chunk", [1, 3, 8, 16])
def test_accumulation_chunks(chunk):
    """Chunked TMEM accumulation (any chunk length, ragged last chunk) against the oracle."""
    c = workloads.random_cloud(58, 300, 140, 3000)
    ref = oracle.field(c.pitch_m, c.lambda_m, c.xyz, c.amp, 300, 140)
    got = _run(c, "gemm_split16", splitk=2, chunk=chunk)
    assert oracle.nrms(got, ref) <= NRMS["gemm_split16"]


@pytest.mark.parametrize("form", ["gemm_f16", "gemm_bf16", "gemm_split16"])
def test_display_size_50k_points_sampled(form):
    """1920x1080, 5x10^4 points, in the launch configuration the benchmark times."""
    c = workloads.display_gemm()
    rng = np.random.default_rng(8)
    cols = np.concatenate([rng.integers(0, 1920, 300), [0, 1919, 0, 1919]])
    rows = np.concatenate([rng.integers(0, 1080, 300), [0, 0, 1079, 1079]])
    ref = oracle.field_at(c.pitch_m, c.lambda_m, c.xyz, c.amp, cols, rows)
    got = _run(c, form)[rows, cols]
    assert oracle.nrms(got, ref) <= NRMS[form]


def test_large_amplitudes_are_scaled():
    """Amplitudes far outside the FP16 range still give the right field (scale by 1/max|A|)."""
    c = workloads.random_cloud(57, 200, 100, 500)
    c.amp *= np.float32(1e6)
    ref = oracle.field(c.pitch_m, c.lambda_m, c.xyz, c.amp, 200, 100)
    got = _run(c, "gemm_split16")
    assert oracle.nrms(got, ref) <= NRMS["gemm_split16"]


@pytest.mark.parametrize("form", ["gemm_f16", "gemm_split16"])
@pytest.mark.parametrize("splitk", [1, 3])
def test_point_chunks_accumulate(form, splitk):
    """A 1 MB factor budget cuts 3000 points into chunks whose GEMMs add up."""
    c = workloads.random_cloud(59, 320, 200, 3000)
    ref = oracle.field(c.pitch_m, c.lambda_m, c.xyz, c.amp, 320, 200)
    whole = _run(c, form, splitk=splitk)
    chunked = _run(c, form, splitk=splitk, budget_mb=1)
    assert oracle.nrms(chunked, ref) <= NRMS[form]
    assert oracle.nrms(chunked, whole) < 1e-5


def test_layered_million_points_split16_sampled():
    """4096x4096, 10^6 points on 16 planes, split FP16 in point chunks: sampled pixels vs the oracle."""
    c = workloads.large_layered()
    rng = np.random.default_rng(6)
    cols = rng.integers(0, 4096, 48)
    rows = rng.integers(0, 4096, 48)
    ref = oracle.field_at(c.pitch_m, c.lambda_m, c.xyz, c.amp, cols, rows)
    xyz, amp = _dev(c)
    with Hologram(4096, 4096, c.pitch_m, c.lambda_m, form="gemm_split16", timeout_ms=60000) as h:
        f = h.point_cloud(xyz, amp)
        h.sync()
        got = f[torch.from_numpy(rows).cuda(), torch.from_numpy(cols).cuda()].cpu().numpy()
    assert oracle.nrms(got, ref) <= NRMS["gemm_split16"]


@pytest.mark.parametrize("form", ["gemm_f16", "gemm_split16"])
def test_factor_gemm_pipeline_matches_unpipelined(form):
    """Factors of the next point chunk on a second stream while the GEMM of the current one runs:
    the same result as one chunk at a time."""
    c = workloads.random_cloud(60, 640, 360, 40000)
    xyz, amp = _dev(c)
    outs = []
    for depth in (1, 4):
        with Hologram(640, 360, c.pitch_m, c.lambda_m, form=form, timeout_ms=5000) as h:
            h.set_option(_lib.CGH_OPT_GEMM_PIPELINE, depth)
            outs.append(h.point_cloud(xyz, amp).cpu().numpy())
            h.sync()
    assert oracle.nrms(outs[1], outs[0]) < 1e-5
    rng = np.random.default_rng(61)
    cols, rows = rng.integers(0, 640, 200), rng.integers(0, 360, 200)
    ref = oracle.field_at(c.pitch_m, c.lambda_m, c.xyz, c.amp, cols, rows)
    assert oracle.nrms(outs[1][rows, cols], ref) <= NRMS[form]


@pytest.mark.parametrize("form", ["gemm_f16", "gemm_split16"])
@pytest.mark.parametrize("trans", [1, 2])
@pytest.mark.parametrize("bn,splitk", [(224, 1), (128, 3), (256, 2)])
def test_both_orientations(form, trans, bn, splitk):
    """128-row tiles of P or of Q (then written back transposed), ragged in both directions."""
    c = workloads.random_cloud(62, 500, 270, 1500)
    ref = oracle.field(c.pitch_m, c.lambda_m, c.xyz, c.amp, 500, 270)
    got = _run(c, form, bn=bn, splitk=splitk, trans=trans)
    assert oracle.nrms(got, ref) <= NRMS[form]


def test_transposed_point_chunks_accumulate():
    c = workloads.random_cloud(63, 333, 250, 3000)
    ref = oracle.field(c.pitch_m, c.lambda_m, c.xyz, c.amp, 333, 250)
    got = _run(c, "gemm_split16", splitk=2, budget_mb=1, trans=2)
    assert oracle.nrms(got, ref) <= NRMS["gemm_split16"]


# ---- the GEMM form of one hologram through the persistent kernel -----------

@pytest.mark.parametrize("form", ["gemm_f16", "gemm_bf16", "gemm_split16"])
@pytest.mark.parametrize("w,h,n", [(1920, 1080, 20000), (300, 77, 1000), (130, 257, 5), (1024, 64, 40000)])
def test_persistent_single_hologram(form, w, h, n):
    """CGH_OPT_GEMM_PERSISTENT: factors generated K chunk by K chunk beside the GEMM of the chunks already there,
    the chunks of a tile added in K order; against the oracle (sampled pixels at the large size) and the separate
    launches (same factors, other summation order: within single-precision rounding); a second call replays the
    graph and gives the same bits."""
    c = workloads.random_cloud(5100 + n, w, h, n)
    xyz, amp = _dev(c)
    with Hologram(w, h, c.pitch_m, c.lambda_m, form=form) as hg:
        hg.set_option(_lib.CGH_OPT_GEMM_PERSISTENT, 1)
        hg.profile(True)
        a = hg.point_cloud(xyz, amp)
        b = hg.point_cloud(xyz, amp)
        hg.sync()
        names = set(hg.profile_read())
        a, b = a.cpu().numpy(), b.cpu().numpy()
    assert "gemm_persist" in names
    assert np.array_equal(a, b)
    plain = _run(c, form)
    assert oracle.nrms(a, plain) < (3e-6 if form == "gemm_split16" else NRMS[form] / 4)
    if w * h * n <= 2e8:
        ref = oracle.field(c.pitch_m, c.lambda_m, c.xyz, c.amp, w, h)
        assert oracle.nrms(a, ref) <= NRMS[form]
    else:
        rng = np.random.default_rng(51)
        cols, rows = rng.integers(0, w, 256), rng.integers(0, h, 256)
        ref = oracle.field_at(c.pitch_m, c.lambda_m, c.xyz, c.amp, cols, rows)
        assert oracle.nrms(a[rows, cols], ref) <= NRMS[form]


# ---- the two-SM GEMM (clusters of two CTAs, 256-row tiles) -------------------

@pytest.mark.parametrize("form", ["gemm_f16", "gemm_bf16", "gemm_split16"])
@pytest.mark.parametrize("w,h,n,trans", [(300, 77, 1000, 0), (130, 257, 5, 0), (1920, 1080, 20000, 0),
                                         (1920, 1080, 20000, 2), (520, 300, 3000, 2)])
def test_pair_gemm(form, w, h, n, trans):
    """CGH_OPT_GEMM_PAIR: the tcgen05 MMA of a CTA pair (M = 256, each CTA half of B) against the oracle and the
    one-CTA form (the same products, so equal within single-precision rounding of the accumulation)."""
    c = workloads.random_cloud(5300 + n + w, w, h, n)
    xyz, amp = _dev(c)
    with Hologram(w, h, c.pitch_m, c.lambda_m, form=form, timeout_ms=3000) as hg:
        hg.set_option(_lib.CGH_OPT_GEMM_PAIR, 1)
        hg.set_option(_lib.CGH_OPT_GEMM_GROUP, 1)
        if trans:
            hg.set_option(_lib.CGH_OPT_GEMM_TRANSPOSE, trans)
        a = hg.point_cloud(xyz, amp)
        hg.sync()
        a = a.cpu().numpy()
    plain = _run(c, form, trans=trans or None, pair=2)
    assert oracle.nrms(a, plain) < (3e-6 if form == "gemm_split16" else NRMS[form] / 4)
    if w * h * n <= 2e8:
        ref = oracle.field(c.pitch_m, c.lambda_m, c.xyz, c.amp, w, h)
        assert oracle.nrms(a, ref) <= NRMS[form]
