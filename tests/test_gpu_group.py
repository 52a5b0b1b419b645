"""The grouped GEMM form (CGH_OPT_GEMM_GROUP): points on one depth plane and
one column summed into a single K unit before the tensor-core GEMM.  The sum
is the same (Eq. 5, regrouped), so it is held to the oracle at the tolerances
of the ungrouped forms, and it must fall back to the ungrouped form whenever
grouping does not apply."""
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


def _run(c, form, group, opts=None):
    """(field, profile kernel names) with CGH_OPT_GEMM_GROUP = group."""
    xyz, amp = torch.from_numpy(c.xyz).cuda(), torch.from_numpy(c.amp).cuda()
    with Hologram(c.width, c.height, c.pitch_m, c.lambda_m, form=form, timeout_ms=5000) as h:
        h.set_option(_lib.CGH_OPT_GEMM_GROUP, group)
        for k, v in (opts or {}).items():
            h.set_option(k, v)
        h.profile(True)
        f = h.point_cloud(xyz, amp)
        h.sync()
        names = set(h.profile_read())
    return f.cpu().numpy(), names


@pytest.mark.parametrize("form", ["gemm_f16", "gemm_bf16", "gemm_split16"])
@pytest.mark.parametrize("w,h,n,planes", [(320, 200, 3000, 4), (257, 130, 5000, 1), (64, 300, 2000, 16)])
def test_grouped_vs_oracle(form, w, h, n, planes):
    c = workloads.layered_cloud(700 + n + planes, w, h, n, planes)
    ref = oracle.field(c.pitch_m, c.lambda_m, c.xyz, c.amp, w, h)
    got, names = _run(c, form, 2)
    assert "group_factors" in names and "factors" not in names
    assert oracle.nrms(got, ref) <= NRMS[form]


@pytest.mark.parametrize("form", ["gemm_f16", "gemm_split16"])
def test_large_groups_and_offaperture_columns(form):
    """Few columns, some outside the hologram (x < 0, x >= W): groups of hundreds of points."""
    c = workloads.layered_cloud(710, 200, 160, 20000, 3, x_range=(-40, 240))
    c.xyz[:, 0] = np.round(c.xyz[:, 0] / 20.0) * 20.0       # 15 columns
    ref = oracle.field(c.pitch_m, c.lambda_m, c.xyz, c.amp, 200, 160)
    got, names = _run(c, form, 2)
    assert "group_factors" in names
    assert oracle.nrms(got, ref) <= NRMS[form]


def test_grouped_is_deterministic():
    """Members are summed in point order whatever order the scatter wrote them in."""
    c = workloads.layered_cloud(711, 300, 200, 30000, 8)
    a, _ = _run(c, "gemm_split16", 2)
    b, _ = _run(c, "gemm_split16", 2)
    assert np.array_equal(a, b)


def test_grouped_matches_ungrouped():
    c = workloads.layered_cloud(712, 256, 256, 8000, 5)
    g, ng = _run(c, "gemm_split16", 2)
    u, nu = _run(c, "gemm_split16", 1)
    assert "group_factors" in ng and "group_factors" not in nu and "factors" in nu
    assert oracle.nrms(g, u) < 1e-5


@pytest.mark.parametrize("splitk,budget", [(1, 1), (3, 1), (2, 0)])
def test_grouped_chunks_and_splits(splitk, budget):
    """Group chunks under a 1 MB factor budget, and K splits, add up to the same field."""
    c = workloads.layered_cloud(713, 320, 200, 12000, 6)
    ref = oracle.field(c.pitch_m, c.lambda_m, c.xyz, c.amp, 320, 200)
    opts = {_lib.CGH_OPT_GEMM_SPLITK: splitk}
    if budget:
        opts[_lib.CGH_OPT_FACTOR_BUDGET_MB] = budget
    got, names = _run(c, "gemm_split16", 2, opts)
    assert "group_factors" in names
    assert oracle.nrms(got, ref) <= NRMS["gemm_split16"]


@pytest.mark.parametrize("trans", [1, 2])
def test_grouped_orientations(trans):
    c = workloads.layered_cloud(714, 500, 270, 6000, 4)
    ref = oracle.field(c.pitch_m, c.lambda_m, c.xyz, c.amp, 500, 270)
    got, _ = _run(c, "gemm_split16", 2, {_lib.CGH_OPT_GEMM_TRANSPOSE: trans})
    assert oracle.nrms(got, ref) <= NRMS["gemm_split16"]


def test_too_many_planes_falls_back():
    """Continuous depths (more than 64 distinct constants): the ungrouped form runs."""
    c = workloads.random_cloud(715, 200, 120, 3000)
    ref = oracle.field(c.pitch_m, c.lambda_m, c.xyz, c.amp, 200, 120)
    got, names = _run(c, "gemm_split16", 2)
    assert "group_planes" in names and "group_count" not in names and "group_factors" not in names
    assert oracle.nrms(got, ref) <= NRMS["gemm_split16"]


@pytest.mark.parametrize("planes,grouped", [(64, True), (65, False)])
def test_plane_count_limit_over_many_blocks(planes, grouped):
    """The distinct depths are collected per thread block and then across blocks: 64 planes spread over every
    block of 20,000 points are grouped, 65 fall back to the ungrouped form."""
    c = workloads.layered_cloud(718 + planes, 180, 140, 20000, planes)
    got, names = _run(c, "gemm_split16", 2)
    assert ("group_factors" in names) == grouped
    rng = np.random.default_rng(5)
    cols, rows = rng.integers(0, 180, 300), rng.integers(0, 140, 300)
    ref = oracle.field_at(c.pitch_m, c.lambda_m, c.xyz, c.amp, cols, rows)
    assert oracle.nrms(got[rows, cols], ref) <= NRMS["gemm_split16"]


def test_oversized_group_falls_back():
    """A group above 1024 points (all points in one column of one plane): the ungrouped form runs."""
    c = workloads.layered_cloud(716, 150, 150, 2000, 1)
    c.xyz[:, 0] = 75.0
    ref = oracle.field(c.pitch_m, c.lambda_m, c.xyz, c.amp, 150, 150)
    got, names = _run(c, "gemm_split16", 2)
    assert "group_count" in names and "group_factors" not in names
    assert oracle.nrms(got, ref) <= NRMS["gemm_split16"]


def test_automatic_rule_keeps_small_clouds_ungrouped():
    c = workloads.layered_cloud(717, 200, 120, 3000, 2)
    _, names = _run(c, "gemm_f16", 0)
    assert "group_planes" not in names and "factors" in names


def test_single_point_and_zero_amplitudes():
    c = workloads.layered_cloud(718, 90, 70, 1, 1)
    ref = oracle.field(c.pitch_m, c.lambda_m, c.xyz, c.amp, 90, 70)
    got, names = _run(c, "gemm_split16", 2)
    assert "group_factors" in names
    assert oracle.nrms(got, ref) <= NRMS["gemm_split16"]
    c.amp[:] = 0.0
    got, _ = _run(c, "gemm_split16", 2)
    assert np.all(got == 0.0)


@pytest.mark.parametrize("form", ["gemm_f16", "gemm_split16"])
def test_layered_million_points_grouped_sampled(form):
    """4096x4096, 10^6 points on 16 planes: the automatic rule groups them; sampled pixels vs the oracle."""
    c = workloads.large_layered()
    rng = np.random.default_rng(16)
    cols = np.concatenate([rng.integers(0, 4096, 48), [0, 4095]])
    rows = np.concatenate([rng.integers(0, 4096, 48), [4095, 0]])
    ref = oracle.field_at(c.pitch_m, c.lambda_m, c.xyz, c.amp, cols, rows)
    xyz, amp = torch.from_numpy(c.xyz).cuda(), torch.from_numpy(c.amp).cuda()
    with Hologram(4096, 4096, c.pitch_m, c.lambda_m, form=form, timeout_ms=60000) as h:
        h.profile(True)
        f = h.point_cloud(xyz, amp)
        h.sync()
        names = set(h.profile_read())
        got = f[torch.from_numpy(rows).cuda(), torch.from_numpy(cols).cuda()].cpu().numpy()
    assert "group_factors" in names
    assert oracle.nrms(got, ref) <= NRMS[form]
