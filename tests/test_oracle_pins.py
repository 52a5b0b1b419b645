"""Pins of the FP64 oracle against what the paper and the mathematics fix.

Each test checks the oracle against something other than itself: exact
rational brute force, closed-form special values, the zone-plate zeros of a
single point (Eq. 2/5), linearity of the sum, mirror and translation
symmetry, the separable factorisation, the recurrence of Eqs. 6-8, and hand
cases of the quantiser.  A plausible slip in the oracle (a dropped term, a
wrong sign, pi for 2 pi, lambda in the numerator as printed in the paper's
listings, transposed m/n) fails at least one of them.
"""
import math
from fractions import Fraction

import numpy as np
import pytest

import oracle
from paper_1309_2734_gb300 import workloads

P8 = 8e-6
L532 = 532e-9


def _cloud(pts, amps=None):
    xyz = np.asarray(pts, dtype=np.float32).reshape(-1, 3)
    a = np.ones(xyz.shape[0], np.float32) if amps is None else np.asarray(amps, np.float32)
    return xyz, a


def _exact_pixel(pitch, lam, xyz, amp, m, n):
    """Brute force: exact rational phase in turns, reduced exactly, then math.cos; fsum."""
    p = Fraction(pitch)
    L = Fraction(lam)
    terms = []
    for (x, y, z), a in zip(xyz.astype(np.float64), amp.astype(np.float64)):
        c = p * p / (2 * L * Fraction(float(z)))
        dx = Fraction(m) - Fraction(float(x))
        dy = Fraction(n) - Fraction(float(y))
        t = c * (dx * dx + dy * dy)
        f = t - round(t)
        terms.append(float(a) * math.cos(2 * math.pi * float(f)))
    return math.fsum(terms)


@pytest.mark.parametrize("seed", [1, 2, 3])
def test_brute_force_tiny(seed):
    """Eq. 5 (restricted form) on W, H <= 5 and N <= 3, exact rational arithmetic."""
    rng = np.random.default_rng(seed)
    W, H = 5, 4
    n = 3
    xyz = np.stack([rng.integers(-3, 8, n), rng.integers(-3, 7, n), rng.uniform(0.2, 1.0, n)], 1)
    if seed == 3:
        xyz[:, 0] += 0.5      # non-integer positions: the definition still holds
    xyz = xyz.astype(np.float32)
    amp = rng.uniform(0.1, 1.0, n).astype(np.float32)
    pitch = [8e-6, 6.4e-6, 3.74e-6][seed - 1]
    lam = [532e-9, 633e-9, 488e-9][seed - 1]
    got = oracle.field(pitch, lam, xyz, amp, W, H)
    for nn in range(H):
        for mm in range(W):
            assert abs(got[nn, mm] - _exact_pixel(pitch, lam, xyz, amp, mm, nn)) < 1e-12


def test_quarter_turn_closed_form():
    """c = p^2/(2 lambda z) = 1/8 turn/px^2: cos(pi r^2 / 4) takes 8 textbook values."""
    table = {0: 1.0, 1: math.sqrt(0.5), 2: 0.0, 3: -math.sqrt(0.5), 4: -1.0,
             5: -math.sqrt(0.5), 6: 0.0, 7: math.sqrt(0.5)}
    x0, y0 = 1, 2
    xyz, amp = _cloud([[x0, y0, 4.0]])
    W, H = 7, 5                  # not square, point off-centre: catches m/n transposition
    got = oracle.field(1.0, 1.0, xyz, amp, W, H)
    for n in range(H):
        for m in range(W):
            r2 = (m - x0) ** 2 + (n - y0) ** 2
            assert abs(got[n, m] - table[r2 % 8]) < 1e-13, (m, n)


def test_half_turn_closed_form():
    """c = 1/2 turn/px^2: every pixel is (-1)^(r^2), scaled by A."""
    xyz, amp = _cloud([[3, 0, 1.0]], [0.75])
    got = oracle.field(0.5, 0.25, xyz, amp, 6, 3)
    for n in range(3):
        for m in range(6):
            r2 = (m - 3) ** 2 + n * n
            assert abs(got[n, m] - 0.75 * (-1) ** r2) < 1e-14


def test_zone_plate_zero_crossings():
    """A single point gives a Fresnel zone plate: I = cos(pi p^2 r^2/(lambda z)).

    Along the point's row the sign changes exactly between the pixels that
    bracket r_k = sqrt((2k+1) lambda z / 2) / p (pitch units), for every r_k
    below the sampling (Nyquist) radius lambda z / (2 p^2).
    """
    z = 0.5
    x0, y0 = 1000, 3
    xyz, amp = _cloud([[x0, y0, z]])
    W = 2048
    row = oracle.field(P8, L532, xyz, amp, W, 8, window=(y0, 0, 1, W))[0]
    nyq = L532 * z / (2 * P8 * P8)
    radii = []
    k = 0
    while True:
        r = math.sqrt((2 * k + 1) * L532 * z / 2) / P8
        if r >= min(nyq, W - 1 - x0) - 2:
            break
        radii.append(r)
        k += 1
    assert len(radii) > 100
    right = row[x0:]
    signs = np.sign(right)
    changes = np.nonzero(signs[1:] != signs[:-1])[0]       # change between d and d+1
    rmax = int(math.floor(radii[-1])) + 1
    changes = changes[changes < rmax]
    assert len(changes) == len(radii)
    for d, r in zip(changes, radii):
        assert d < r < d + 1
    # the same zeros on the left, and the closed form value at the centre
    assert row[x0] == pytest.approx(1.0, abs=1e-15)
    assert np.allclose(row[x0 - 500:x0], row[x0 + 500:x0:-1], atol=1e-12)


def test_lambda_placement_matters():
    """The listings' phase pi*lambda*r^2/z would not give these zeros (Section 4.1)."""
    z = 0.8
    xyz, amp = _cloud([[0, 0, z]])
    row = oracle.field(P8, L532, xyz, amp, 400, 1)[0]
    r0 = math.sqrt(L532 * z / 2) / P8          # first zero, ~36.5 px
    d = int(math.floor(r0))
    assert row[d] > 0 > row[d + 1]


def test_linearity_points_and_amplitudes():
    c = workloads.random_cloud(77, 40, 30, 200)
    a, b = c.amp.copy(), c.amp.copy()
    a[100:] = 0
    b[:100] = 0
    full = oracle.field(c.pitch_m, c.lambda_m, c.xyz, c.amp, 40, 30)
    pa = oracle.field(c.pitch_m, c.lambda_m, c.xyz[:100], c.amp[:100], 40, 30)
    pb = oracle.field(c.pitch_m, c.lambda_m, c.xyz[100:], c.amp[100:], 40, 30)
    assert np.allclose(full, pa + pb, rtol=0, atol=1e-11 * np.abs(full).max())
    za = oracle.field(c.pitch_m, c.lambda_m, c.xyz, a, 40, 30)
    assert np.allclose(za, pa, atol=1e-12)
    scaled = oracle.field(c.pitch_m, c.lambda_m, c.xyz, (c.amp * 0.5).astype(np.float32), 40, 30)
    assert np.allclose(scaled, 0.5 * full, atol=1e-12 * np.abs(full).max())
    empty = oracle.field(c.pitch_m, c.lambda_m, c.xyz[:0], c.amp[:0], 40, 30)
    assert np.all(empty == 0.0)


def test_mirror_symmetry():
    W, H = 33, 21
    c = workloads.random_cloud(5, W, H, 60)
    mx = c.xyz.copy()
    mx[:, 0] = (W - 1) - mx[:, 0]
    xyz = np.concatenate([c.xyz, mx])
    amp = np.concatenate([c.amp, c.amp])
    I = oracle.field(c.pitch_m, c.lambda_m, xyz, amp, W, H)
    assert np.allclose(I, I[:, ::-1], atol=1e-11)
    my = c.xyz.copy()
    my[:, 1] = (H - 1) - my[:, 1]
    I2 = oracle.field(c.pitch_m, c.lambda_m, np.concatenate([c.xyz, my]), amp, W, H)
    assert np.allclose(I2, I2[::-1, :], atol=1e-11)
    # an asymmetric cloud is not symmetric (the test can fail)
    I3 = oracle.field(c.pitch_m, c.lambda_m, c.xyz, c.amp, W, H)
    assert not np.allclose(I3, I3[:, ::-1], atol=1e-3)


def test_integer_translation():
    W, H = 48, 40
    c = workloads.random_cloud(9, 32, 24, 80)
    dx, dy = 7, 5
    sh = c.xyz.copy()
    sh[:, 0] += dx
    sh[:, 1] += dy
    a = oracle.field(c.pitch_m, c.lambda_m, c.xyz, c.amp, W, H)
    b = oracle.field(c.pitch_m, c.lambda_m, sh, c.amp, W, H)
    assert np.allclose(b[dy:, dx:], a[:H - dy, :W - dx], atol=1e-11)


def test_separable_factors_reproduce_field():
    """P Q^T with P[n][2j] = cos b, P[n][2j+1] = sin b, Q = A(cos a, -sin a) equals I."""
    c = workloads.random_cloud(21, 37, 29, 150)
    P, Q = oracle.factors(c.pitch_m, c.lambda_m, c.xyz, c.amp, 37, 29)
    I = oracle.field(c.pitch_m, c.lambda_m, c.xyz, c.amp, 37, 29)
    assert P.shape == (29, 300) and Q.shape == (37, 300)
    assert np.allclose(P @ Q.T, I, atol=1e-10)
    # each factor entry against the exact single-axis phase
    p, L = Fraction(c.pitch_m), Fraction(c.lambda_m)
    for j in (0, 77, 149):
        x, y, z = (float(v) for v in c.xyz[j])
        cc = p * p / (2 * L * Fraction(z))
        for n in (0, 13, 28):
            t = cc * (Fraction(n) - Fraction(y)) ** 2
            b = 2 * math.pi * float(t - round(t))
            assert abs(P[n, 2 * j] - math.cos(b)) < 1e-13
            assert abs(P[n, 2 * j + 1] - math.sin(b)) < 1e-13
        for m in (0, 20, 36):
            t = cc * (Fraction(m) - Fraction(x)) ** 2
            a = 2 * math.pi * float(t - round(t))
            assert abs(Q[m, 2 * j] - float(c.amp[j]) * math.cos(a)) < 1e-13
            assert abs(Q[m, 2 * j + 1] + float(c.amp[j]) * math.sin(a)) < 1e-13


def test_wave_real_part_and_modulus():
    c = workloads.random_cloud(4, 20, 16, 50)
    O = oracle.wave(c.pitch_m, c.lambda_m, c.xyz, c.amp, 20, 16)
    I = oracle.field(c.pitch_m, c.lambda_m, c.xyz, c.amp, 20, 16)
    assert np.allclose(O.real, I, atol=1e-12)
    one = oracle.wave(c.pitch_m, c.lambda_m, c.xyz[:1], c.amp[:1], 20, 16)
    assert np.allclose(np.abs(one), float(c.amp[0]), atol=1e-13)


def test_recurrence_reproduces_quadratic_phase():
    """Eqs. 6-8: Gamma_{k+1} = Gamma_k + delta_k, delta_{k+1} = delta_k + Delta, exactly."""
    c = Fraction(P8) ** 2 / (2 * Fraction(L532) * Fraction(float(np.float32(0.37))))
    for dx0, dy in ((-20, 3), (0, 0), (5, -17)):
        g = oracle.recurrence_phases(c, dx0, dy, 40)
        for k, gk in enumerate(g):
            assert gk == c * ((dx0 + k) ** 2 + dy * dy)
    # and the oracle's cosine of that phase at those pixels
    z = float(np.float32(0.37))
    xyz, amp = _cloud([[30, 10, z]])
    row = oracle.field(P8, L532, xyz, amp, 80, 20, window=(13, 0, 1, 80))[0]
    g = oracle.recurrence_phases(c, 10 - 30, 13 - 10, 40)
    for k in range(40):
        f = g[k] - round(g[k])
        assert abs(row[10 + k] - math.cos(2 * math.pi * float(f))) < 1e-12


def test_field_at_matches_window():
    c = workloads.random_cloud(8, 50, 40, 64)
    I = oracle.field(c.pitch_m, c.lambda_m, c.xyz, c.amp, 50, 40)
    rng = np.random.default_rng(0)
    cols = rng.integers(0, 50, 30)
    rows = rng.integers(0, 40, 30)
    v = oracle.field_at(c.pitch_m, c.lambda_m, c.xyz, c.amp, cols, rows)
    assert np.array_equal(v, I[rows, cols])
    win = oracle.field(c.pitch_m, c.lambda_m, c.xyz, c.amp, 50, 40, window=(7, 11, 9, 13))
    assert np.array_equal(win, I[7:16, 11:24])


def test_accumulation_at_display_point_count():
    """FP64 sum over 10^4 points agrees with exact-phase fsum to 1e-11 relative."""
    c = workloads.display_direct()
    cols = np.array([0, 959, 1919, 1234])
    rows = np.array([0, 539, 1079, 77])
    v = oracle.field_at(c.pitch_m, c.lambda_m, c.xyz, c.amp, cols, rows)
    scale = math.sqrt(np.sum(c.amp.astype(np.float64) ** 2))
    for i in range(2):
        ref = _exact_pixel(c.pitch_m, c.lambda_m, c.xyz, c.amp, int(cols[i]), int(rows[i]))
        assert abs(v[i] - ref) < 1e-11 * scale


# ---- quantiser ------------------------------------------------------------

def test_quantize_endpoints_and_constant():
    f = np.array([-3.5, 0.0, 2.25, 7.125, -3.5], np.float32)
    q, (lo, hi, s) = oracle.quantize8(f)
    assert lo == -3.5 and hi == 7.125
    assert q[0] == 0 and q[4] == 0 and q[3] == 255
    assert s >= 255.0 / (7.125 + 3.5)
    c, _ = oracle.quantize8(np.full(17, 4.0, np.float32))
    assert np.all(c == 0)
    e, _ = oracle.quantize8(np.zeros(0, np.float32))
    assert e.shape == (0,)


def test_quantize_exact_bins():
    """lo = 0, hi = 255/256: s = 256 exactly, so v = k/256 maps to k and just below to k-1."""
    k = np.arange(256, dtype=np.float64)
    v = (k / 256.0).astype(np.float32)
    q, (lo, hi, s) = oracle.quantize8(v)
    assert s == 256.0
    assert np.array_equal(q, np.arange(256, dtype=np.uint8))
    below = np.nextafter(v[1:], np.float32(-1)).astype(np.float32)
    qb, _ = oracle.quantize8(np.concatenate([v[:1], below, v[-1:]]))
    assert np.array_equal(qb[1:-1], np.arange(255, dtype=np.uint8))


def test_quantize_properties_random():
    rng = np.random.default_rng(3)
    f = (rng.standard_normal(10000) * 37.0).astype(np.float32)
    q, (lo, hi, s) = oracle.quantize8(f)
    order = np.argsort(f, kind="stable")
    assert np.all(np.diff(q[order].astype(int)) >= 0)          # monotone
    assert q[np.argmin(f)] == 0 and q[np.argmax(f)] == 255
    ideal = np.floor(255.0 * (f.astype(np.float64) - lo) / (float(hi) - float(lo)))
    assert np.max(np.abs(q.astype(np.float64) - np.minimum(ideal, 255))) <= 1
    perm = rng.permutation(f.shape[0])
    q2, lh2 = oracle.quantize8(f[perm])
    assert np.array_equal(q2, q[perm]) and lh2 == (lo, hi, s)
    fn = f.copy()
    fn[5] = np.nan
    qn, _ = oracle.quantize8(fn)
    assert qn[5] == 0


def test_kinoform_hand_cases():
    """Eq. 3 with the listings' rule: floor(255 psi / 2 pi), psi in [0, 2 pi)."""
    w = np.array([1 + 0j, 1j, -1 + 0j, -1j, 1 - 1e-9j, 1 + 1j, -1 - 1j, 0j, 2.5 + 0j])
    q = oracle.kinoform8(w)
    # psi: 0, pi/2, pi, 3pi/2, ~2pi, pi/4, 5pi/4, atan2(0,0)=0, 0
    assert list(q) == [0, 63, 127, 191, 254, 31, 159, 0, 0]
    # the phase of a single point's wave is its own Fresnel phase (Eq. 2)
    xyz = np.array([[3, 2, 0.5]], np.float32)
    amp = np.array([1.0], np.float32)
    O = oracle.wave(8e-6, 532e-9, xyz, amp, 16, 8)
    c = (8e-6) ** 2 / (2 * 532e-9 * float(np.float32(0.5)))
    m, n = np.meshgrid(np.arange(16), np.arange(8))
    t = c * ((m - 3.0) ** 2 + (n - 2.0) ** 2)
    want = np.floor(255.0 * (t - np.floor(t)))
    got = oracle.kinoform8(O).astype(np.float64)
    frac = 255.0 * (t - np.floor(t))
    safe = np.abs(frac - np.round(frac)) > 1e-6
    assert np.array_equal(got[safe], want[safe])


# ---- phase models of Eq. 1 / Eq. 2 and the plane-wave reference of Eqs. 4-5 ----

def _decimal_model_pixel(model, pitch, lam, ref, xyz, amp, m, n):
    """Brute force in 60-digit decimal arithmetic: the phase of model 0/1/2 plus phi_r, reduced exactly."""
    from decimal import Decimal, getcontext
    getcontext().prec = 60
    D = lambda v: Decimal(repr(float(v)))
    p, L = D(pitch), D(lam)
    sx, sy, ph = (D(v) for v in ref)
    two_pi = Decimal("6.283185307179586476925286766559005768394338798750211641949889")
    reft = (D(m) * p * sx + D(n) * p * sy) / L + ph / two_pi
    acc = 0.0
    for (x, y, z), a in zip(xyz.astype(np.float64), amp.astype(np.float64)):
        dx = (D(m) - D(x)) * p
        dy = (D(n) - D(y)) * p
        zz = D(z)
        r2 = dx * dx + dy * dy
        if model == 2:
            t = (r2 + zz * zz).sqrt() / L
        elif model == 1:
            t = (zz + r2 / (2 * zz)) / L
        else:
            t = r2 / (2 * L * zz)
        t = t + reft
        f = t - t.to_integral_value()
        acc += a * math.cos(2 * math.pi * float(f))
    return acc


def _model_tol(xyz, amp, lam, turns_extra=1e3):
    """The oracle's own rounding: phases of up to max z/lambda turns carry a few ulps of that size each,
    so the field is off by at most 2 pi * 8 ulp(t_max) * sum|A| (t_max: the piston plus the quadratic part)."""
    t_max = float(np.max(xyz[:, 2].astype(np.float64))) / lam + turns_extra
    return 2 * math.pi * 8 * float(np.spacing(t_max)) * float(np.sum(np.abs(amp.astype(np.float64)))) + 1e-12


@pytest.mark.parametrize("model", [0, 1, 2])
@pytest.mark.parametrize("ref", [(0.0, 0.0, 0.0), (0.0123, -0.0071, 0.7)])
def test_models_brute_force_tiny(model, ref):
    rng = np.random.default_rng(40 + model)
    xyz = np.stack([rng.integers(-20, 40, 5), rng.integers(-20, 40, 5), rng.uniform(0.05, 0.6, 5)], 1)
    xyz, amp = _cloud(xyz, rng.uniform(0.2, 1.0, 5))
    w = oracle.model_wave(model, P8, L532, xyz, amp, 7, 6, reference=ref, window=(1, 2, 4, 5))
    for r in range(4):
        for q in range(5):
            want = _decimal_model_pixel(model, P8, L532, ref, xyz, amp, 2 + q, 1 + r)
            assert abs(w[r, q].real - want) < _model_tol(xyz, amp, L532), (model, r, q, w[r, q].real, want)


def test_model0_equals_restricted_field_and_wave():
    """Model 0 without reference is the restricted form of Eq. 5 that the other pins fix."""
    c = workloads.random_cloud(91, 24, 17, 40)
    w = oracle.model_wave(0, c.pitch_m, c.lambda_m, c.xyz, c.amp, 24, 17)
    assert np.allclose(w, oracle.wave(c.pitch_m, c.lambda_m, c.xyz, c.amp, 24, 17), atol=1e-11, rtol=0)


def test_spherical_pythagorean_distance():
    """Eq. 1 at a pixel whose distance is exact: offset (3k, 4k) px, z = 12 k p gives distance 13 k p."""
    pitch = 2.0 ** -17          # exact in binary, so z = 12 * 1024 * pitch = 0.09375 is an exact float
    z = 12 * 1024 * pitch
    xyz, amp = _cloud([[5.0, 7.0, z]], [0.8])
    w = oracle.model_wave(2, pitch, L532, xyz, amp, 5 + 3072 + 1, 7 + 4096 + 1,
                          window=(7 + 4096, 5 + 3072, 1, 1))[0, 0]
    turns = Fraction(13 * 1024) * Fraction(pitch) / Fraction(L532)
    f = float(turns - round(turns))
    a = float(amp[0])                                   # 0.8 as stored in single precision
    tol = _model_tol(xyz, amp, L532)
    assert abs(w.real - a * math.cos(2 * math.pi * f)) < tol
    assert abs(w.imag - a * math.sin(2 * math.pi * f)) < tol
    # the Fresnel phase of Eq. 2 differs there by (12 + 25/24 - 13) * 1024 p / lambda turns (hundreds)
    w1 = oracle.model_wave(1, pitch, L532, xyz, amp, 5 + 3072 + 1, 7 + 4096 + 1,
                           window=(7 + 4096, 5 + 3072, 1, 1))[0, 0]
    t1 = (Fraction(12) + Fraction(25, 24)) * 1024 * Fraction(pitch) / Fraction(L532)
    assert abs(w1.real - a * math.cos(2 * math.pi * float(t1 - round(t1)))) < tol


def test_piston_is_the_depth_phase():
    """Eq. 2 with the piston = exp(i 2 pi z/lambda) times Eq. 2 without it, for a single depth plane."""
    c = workloads.layered_cloud(92, 30, 20, 60, 1)
    z = float(c.xyz[0, 2])
    w0 = oracle.model_wave(0, c.pitch_m, c.lambda_m, c.xyz, c.amp, 30, 20)
    w1 = oracle.model_wave(1, c.pitch_m, c.lambda_m, c.xyz, c.amp, 30, 20)
    t = Fraction(z) / Fraction(c.lambda_m)
    rot = np.exp(2j * math.pi * float(t - round(t)))
    assert np.allclose(w1, w0 * rot, atol=_model_tol(c.xyz, c.amp, c.lambda_m), rtol=0)


def test_spherical_tends_to_fresnel():
    """|t_sph - t_fresnel| <= r^4 / (8 lambda z^3) (Taylor remainder of sqrt(1+u) <= 1 + u/2 - u^2/8 + u^3/16),
    so the two fields differ by at most sum_j A_j 2 pi r_j^4 / (8 lambda z_j^3) at every pixel."""
    rng = np.random.default_rng(93)
    n = 12
    xyz, amp = _cloud(np.stack([rng.integers(0, 40, n), rng.integers(0, 30, n), rng.uniform(0.3, 1.0, n)], 1),
                      rng.uniform(0.5, 1.0, n))
    ws = oracle.model_wave(2, P8, L532, xyz, amp, 40, 30)
    wf = oracle.model_wave(1, P8, L532, xyz, amp, 40, 30)
    m, nn = np.meshgrid(np.arange(40), np.arange(30))
    bound = np.zeros((30, 40))
    for (x, y, z), a in zip(xyz.astype(np.float64), amp.astype(np.float64)):
        r2 = ((m - x) ** 2 + (nn - y) ** 2) * P8 * P8
        bound += a * 2 * math.pi * r2 * r2 / (8 * L532 * z ** 3)
    diff = np.abs(ws - wf)
    assert np.all(diff <= bound * 1.001 + 1e-10)
    assert np.max(diff) > 0.05 * np.max(bound)      # the quartic term is really there


def test_reference_phase_rotates_every_pixel():
    """phi_r is added to every term (Eq. 5): O_ref = exp(i phi_r(m, n)) O, phi_r = 2 pi/lambda (x_h sin_x + y_h sin_y) + phase0;
    with sin_x = lambda / (4 p) the reference advances a quarter turn per column."""
    c = workloads.random_cloud(94, 20, 9, 30)
    sx = c.lambda_m / (4 * c.pitch_m)
    w0 = oracle.model_wave(0, c.pitch_m, c.lambda_m, c.xyz, c.amp, 20, 9)
    w = oracle.model_wave(0, c.pitch_m, c.lambda_m, c.xyz, c.amp, 20, 9, reference=(sx, 0.0, 0.25))
    cols = np.arange(20)[None, :]
    assert np.allclose(w, w0 * np.exp(1j * (0.5 * math.pi * cols + 0.25)), atol=1e-9, rtol=0)
    sy = -c.lambda_m / (2 * c.pitch_m)           # half a turn per row, backwards
    w = oracle.model_wave(0, c.pitch_m, c.lambda_m, c.xyz, c.amp, 20, 9, reference=(0.0, sy, 0.0))
    rows = np.arange(9)[:, None]
    assert np.allclose(w, w0 * np.exp(-1j * math.pi * rows), atol=1e-9, rtol=0)


def test_model_points_match_window():
    c = workloads.random_cloud(95, 16, 12, 25)
    ref = (0.01, 0.02, -1.0)
    w = oracle.model_wave(2, c.pitch_m, c.lambda_m, c.xyz, c.amp, 16, 12, reference=ref)
    cols, rows = np.array([0, 15, 7, 3]), np.array([0, 11, 5, 9])
    at = oracle.model_wave_at(2, c.pitch_m, c.lambda_m, c.xyz, c.amp, cols, rows, reference=ref)
    assert np.array_equal(at, w[rows, cols])


# ---- Fresnel diffraction (Eq. 10) and the wavefront-recording method (Section 2.3) ----

def test_fresnel_fft_equals_definition():
    """The numpy-FFT convolution (zero-padded to 2H x 2W) equals the direct sum of Eq. 10 on every pixel."""
    rng = np.random.default_rng(60)
    for (H, W, z) in ((20, 24, 0.05), (17, 9, -0.2), (1, 13, 0.01)):
        u = rng.standard_normal((H, W)) + 1j * rng.standard_normal((H, W))
        full = oracle.fresnel(u, P8, L532, z)
        m, n = np.meshgrid(np.arange(W), np.arange(H))
        direct = oracle.fresnel_at(u, P8, L532, z, m.ravel(), n.ravel()).reshape(H, W)
        assert np.allclose(full, direct, atol=1e-9 * np.abs(direct).max(), rtol=0)


def test_fresnel_gaussian_beam_closed_form():
    """A Gaussian beam exp(-r^2/w0^2) propagated by z has the closed form
    exp(i 2 pi z/lambda)/(i lambda z) * pi/(a - i b) * exp(i b r^2 - b^2 r^2/(a - i b)), a = 1/w0^2, b = pi/(lambda z)
    (the Gaussian integral); the grid sum with cells p^2 converges to it (w0 = 20 px, 200 x 200 grid)."""
    N, w0, z = 200, 20 * P8, 0.1
    yy, xx = np.meshgrid((np.arange(N) - N // 2) * P8, (np.arange(N) - N // 2) * P8, indexing="ij")
    u = np.exp(-(xx ** 2 + yy ** 2) / w0 ** 2)
    got = oracle.fresnel(u, P8, L532, z)
    a, b = 1.0 / w0 ** 2, math.pi / (L532 * z)
    zt = Fraction(z) / Fraction(L532)
    pre = np.exp(2j * math.pi * float(zt - round(zt))) / (1j * L532 * z)
    r2 = xx ** 2 + yy ** 2
    want = pre * (math.pi / (a - 1j * b)) * np.exp(1j * b * r2 - b * b * r2 / (a - 1j * b))
    core = r2 <= (40 * P8) ** 2
    err = np.abs(got - want)[core].max()
    assert err <= 1e-8 * np.abs(want).max(), err
    # a slip of the area element, the prefactor or the sign of the chirp is far larger
    assert np.abs(np.conj(got) - want)[core].max() > 1e-2 * np.abs(want).max()


def test_fresnel_translation_and_linearity():
    rng = np.random.default_rng(61)
    u = np.zeros((30, 30), complex)
    u[5:12, 6:14] = rng.standard_normal((7, 8)) + 1j * rng.standard_normal((7, 8))
    v = np.roll(np.roll(u, 9, axis=0), 7, axis=1)          # stays inside the plane
    fu, fv = oracle.fresnel(u, P8, L532, 0.03), oracle.fresnel(v, P8, L532, 0.03)
    assert np.allclose(fv[9:, 7:], fu[:-9, :-7], atol=1e-10 * np.abs(fu).max())
    w = oracle.fresnel(2.0 * u - 1j * v, P8, L532, 0.03)
    assert np.allclose(w, 2.0 * fu - 1j * fv, atol=1e-10 * np.abs(w).max())


def test_wrp_window_is_the_lattice_disk():
    """One point: the recorded plane is nonzero exactly on the integer points of the disk r^2 <= floor(w^2),
    w = d tan(asin(lambda / 2p)) / p, and equals there the point's wave at depth d (model_wave, pinned above)."""
    z_wrp, d = 0.4, 0.006
    xyz, amp = _cloud([[40.0, 37.0, z_wrp + d]], [0.9])
    u = oracle.wrp_record(1, P8, L532, z_wrp, xyz, amp, 90, 80)
    w = d * math.tan(math.asin(L532 / (2 * P8))) / P8
    W2 = oracle.wrp_window2(P8, L532, float(np.float64(xyz[0, 2]) - z_wrp))
    assert abs(W2 - math.floor(w * w)) <= 1            # same radius, up to the last rounding
    mm, nn = np.meshgrid(np.arange(90), np.arange(80))
    disk = (mm - 40) ** 2 + (nn - 37) ** 2 <= W2
    count = sum(1 for dx in range(-60, 61) for dy in range(-60, 61) if dx * dx + dy * dy <= W2)
    assert np.count_nonzero(u) == disk.sum() == count
    # inside: the quadratic phase at distance d (model 0 at a float32 depth of d: relative 1e-8 of a few turns)
    shifted = xyz.copy()
    shifted[0, 2] = np.float32(np.float64(xyz[0, 2]) - z_wrp)
    u0 = oracle.wrp_record(0, P8, L532, z_wrp, xyz, amp, 90, 80)
    ref0 = oracle.model_wave(0, P8, L532, shifted, amp, 90, 80)
    assert np.allclose(u0[disk], ref0[disk], atol=1e-6)
    # and the piston is that of d = z_j - z_wrp, exactly
    dt = (Fraction(float(xyz[0, 2])) - Fraction(z_wrp)) / Fraction(L532)
    rot = np.exp(2j * math.pi * float(dt - round(dt)))
    assert np.allclose(u[disk], u0[disk] * rot, atol=1e-9)


def test_wrp_rejects_points_in_front_of_the_plane():
    xyz, amp = _cloud([[3.0, 3.0, 0.2]])
    with pytest.raises(ValueError):
        oracle.wrp_record(0, P8, L532, 0.3, xyz, amp, 8, 8)
