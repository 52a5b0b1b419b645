"""FP64 CPU oracle for the point-cloud Fresnel hologram (test infrastructure).

TEST INFRASTRUCTURE ONLY: the tests, ``__graft_entry__.smoke()`` and the
CPU-baseline leg of ``bench.py`` may import this package; the library itself
never does, and it shares no code with the CUDA path.

The arithmetic lives in ``cgh_oracle.c`` (plain C, double precision, libm
cos/sin, OpenMP over rows).  This module compiles it with gcc on first use and
wraps it with ctypes.  Every function cites the passage it follows:

* ``field``/``field_at``: Eq. 2 and Eq. 5 of Section 2.1, without the per-point
  piston and reference phase,
  I(m, n) = sum_j A_j cos(pi p^2/(lambda z_j) ((m - x_j)^2 + (n - y_j)^2)).
* ``wave``: the complex object wave of Eq. 2 (same restriction), for Eq. 3.
* ``factors``: the separable factor matrices P, Q with I = P Q^T.
* ``quantize8``: the min/max 8-bit quantiser (the listings of Section 4.1
  quantise a phase with 255/(2 pi); this is the amplitude counterpart).
* ``kinoform8``: that phase rule for the kinoform of Eq. 3.
* ``recurrence_phases``: Eqs. 6-8 (Section 2.2) iterated in exact rationals.
* ``fresnel_at``/``fresnel``: Fresnel diffraction, Eq. 10 (definition; and
  by numpy FFT); ``wrp_record``/``wrp``: the wavefront-recording method of
  Section 2.3.
* ``model_wave``/``model_wave_at``: the phase models of Eq. 1 (exact spherical
  wave), Eq. 2 with and without the piston, and the plane-wave reference phase
  of Eqs. 4-5; the amplitude hologram is the real part.
"""
from __future__ import annotations

import ctypes
import os
import subprocess
import threading
from fractions import Fraction
from typing import Optional, Sequence

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "cgh_oracle.c")
_LIB_PATH = os.path.join(_HERE, "liboracle.so")
_lock = threading.Lock()
_lib = None

_F32P = ctypes.POINTER(ctypes.c_float)
_F64P = ctypes.POINTER(ctypes.c_double)
_I32P = ctypes.POINTER(ctypes.c_int32)
_U8P = ctypes.POINTER(ctypes.c_uint8)


def build(force: bool = False) -> str:
    """Compile cgh_oracle.c into liboracle.so (gcc, OpenMP, no FP contraction)."""
    if force or not os.path.exists(_LIB_PATH) or os.path.getmtime(_LIB_PATH) < os.path.getmtime(_SRC):
        tmp = _LIB_PATH + f".tmp{os.getpid()}"
        cmd = ["gcc", "-O2", "-fopenmp", "-fPIC", "-shared", "-ffp-contract=off",
               "-fno-fast-math", "-std=c11", _SRC, "-o", tmp, "-lm"]
        subprocess.run(cmd, check=True)
        os.replace(tmp, _LIB_PATH)
    return _LIB_PATH


def _load():
    global _lib
    with _lock:
        if _lib is None:
            lib = ctypes.CDLL(build())
            lib.oracle_threads.restype = ctypes.c_int
            lib.oracle_set_threads.argtypes = [ctypes.c_int]
            lib.oracle_field_window.argtypes = [ctypes.c_double, ctypes.c_double, _F32P, _F32P,
                                                ctypes.c_int64, ctypes.c_int, ctypes.c_int,
                                                ctypes.c_int, ctypes.c_int, _F64P]
            lib.oracle_field_points.argtypes = [ctypes.c_double, ctypes.c_double, _F32P, _F32P,
                                                ctypes.c_int64, _I32P, _I32P, ctypes.c_int64, _F64P]
            lib.oracle_wave_window.argtypes = [ctypes.c_double, ctypes.c_double, _F32P, _F32P,
                                               ctypes.c_int64, ctypes.c_int, ctypes.c_int,
                                               ctypes.c_int, ctypes.c_int, _F64P, _F64P]
            lib.oracle_factors.argtypes = [ctypes.c_int, ctypes.c_int, ctypes.c_double, ctypes.c_double,
                                           _F32P, _F32P, ctypes.c_int64, _F64P, _F64P]
            lib.oracle_quantize8.argtypes = [_F32P, ctypes.c_int64, _U8P, _F32P]
            lib.oracle_kinoform8.argtypes = [_F64P, _F64P, ctypes.c_int64, _U8P]
            lib.oracle_model_window.argtypes = [ctypes.c_int, ctypes.c_double, ctypes.c_double, ctypes.c_double,
                                                ctypes.c_double, ctypes.c_double, _F32P, _F32P, ctypes.c_int64,
                                                ctypes.c_int, ctypes.c_int, ctypes.c_int, ctypes.c_int, _F64P,
                                                _F64P]
            lib.oracle_fresnel_points.argtypes = [ctypes.c_int, ctypes.c_int, ctypes.c_double, ctypes.c_double,
                                                  ctypes.c_double, _F64P, _F64P, _I32P, _I32P, ctypes.c_int64,
                                                  _F64P, _F64P]
            lib.oracle_wrp_record.argtypes = [ctypes.c_int, ctypes.c_double, ctypes.c_double, ctypes.c_double,
                                              _F32P, _F32P, ctypes.c_int64, ctypes.c_int, ctypes.c_int,
                                              ctypes.c_int, ctypes.c_int, _F64P, _F64P]
            lib.oracle_model_points.argtypes = [ctypes.c_int, ctypes.c_double, ctypes.c_double, ctypes.c_double,
                                                ctypes.c_double, ctypes.c_double, _F32P, _F32P, ctypes.c_int64,
                                                _I32P, _I32P, ctypes.c_int64, _F64P, _F64P]
            _lib = lib
    return _lib


def _f32(a) -> np.ndarray:
    return np.ascontiguousarray(a, dtype=np.float32)


def _ptr(a: np.ndarray, t):
    return a.ctypes.data_as(t)


def threads() -> int:
    """OpenMP threads the oracle uses."""
    return int(_load().oracle_threads())


def set_threads(n: int) -> None:
    _load().oracle_set_threads(int(n))


def field(pitch_m: float, lambda_m: float, xyz, amp, width: int, height: int,
          window: Optional[Sequence[int]] = None) -> np.ndarray:
    """I(m, n) of Eq. 5 (restricted form) in FP64, [rows][cols].

    window = (row0, col0, rows, cols); default the whole width x height hologram.
    """
    xyz = _f32(xyz).reshape(-1, 3)
    amp = _f32(amp).reshape(-1)
    if window is None:
        window = (0, 0, height, width)
    r0, c0, rows, cols = (int(v) for v in window)
    out = np.empty((rows, cols), dtype=np.float64)
    rc = _load().oracle_field_window(float(pitch_m), float(lambda_m), _ptr(xyz, _F32P), _ptr(amp, _F32P),
                                     amp.shape[0], r0, rows, c0, cols, _ptr(out, _F64P))
    if rc != 0:
        raise ValueError("oracle_field_window rejected its arguments")
    return out


def field_at(pitch_m: float, lambda_m: float, xyz, amp, cols, rows) -> np.ndarray:
    """I at scattered pixels (cols[i], rows[i]) in FP64."""
    xyz = _f32(xyz).reshape(-1, 3)
    amp = _f32(amp).reshape(-1)
    pm = np.ascontiguousarray(cols, dtype=np.int32)
    pn = np.ascontiguousarray(rows, dtype=np.int32)
    out = np.empty(pm.shape[0], dtype=np.float64)
    rc = _load().oracle_field_points(float(pitch_m), float(lambda_m), _ptr(xyz, _F32P), _ptr(amp, _F32P),
                                     amp.shape[0], _ptr(pm, _I32P), _ptr(pn, _I32P), pm.shape[0],
                                     _ptr(out, _F64P))
    if rc != 0:
        raise ValueError("oracle_field_points rejected its arguments")
    return out


def wave(pitch_m: float, lambda_m: float, xyz, amp, width: int, height: int,
         window: Optional[Sequence[int]] = None) -> np.ndarray:
    """Complex object wave O(m, n) of Eq. 2 (restricted form), complex128 [rows][cols]."""
    xyz = _f32(xyz).reshape(-1, 3)
    amp = _f32(amp).reshape(-1)
    if window is None:
        window = (0, 0, height, width)
    r0, c0, rows, cols = (int(v) for v in window)
    re = np.empty((rows, cols), dtype=np.float64)
    im = np.empty((rows, cols), dtype=np.float64)
    rc = _load().oracle_wave_window(float(pitch_m), float(lambda_m), _ptr(xyz, _F32P), _ptr(amp, _F32P),
                                    amp.shape[0], r0, rows, c0, cols, _ptr(re, _F64P), _ptr(im, _F64P))
    if rc != 0:
        raise ValueError("oracle_wave_window rejected its arguments")
    return re + 1j * im


FRESNEL, FRESNEL_PISTON, SPHERICAL = 0, 1, 2


def model_wave(model: int, pitch_m: float, lambda_m: float, xyz, amp, width: int, height: int,
               reference=(0.0, 0.0, 0.0), window: Optional[Sequence[int]] = None) -> np.ndarray:
    """O(m, n) = sum_j A_j exp(i (2 pi t_j + phi_r)) in FP64, complex128 [rows][cols].

    model 0: t = r^2/(2 lambda z) (Eq. 2 without the piston), 1: t = (z + r^2/(2 z))/lambda (Eq. 2),
    2: t = sqrt(r^2 + z^2)/lambda (Eq. 1); r in metres.  reference = (sin_x, sin_y, phase0):
    phi_r = 2 pi/lambda (m p sin_x + n p sin_y) + phase0, added to every term as in Eq. 5.
    The amplitude hologram of Eq. 5 is the real part.
    """
    xyz = _f32(xyz).reshape(-1, 3)
    amp = _f32(amp).reshape(-1)
    if window is None:
        window = (0, 0, height, width)
    r0, c0, rows, cols = (int(v) for v in window)
    re = np.empty((rows, cols), dtype=np.float64)
    im = np.empty((rows, cols), dtype=np.float64)
    sx, sy, ph = (float(v) for v in reference)
    rc = _load().oracle_model_window(int(model), float(pitch_m), float(lambda_m), sx, sy, ph, _ptr(xyz, _F32P),
                                     _ptr(amp, _F32P), amp.shape[0], r0, rows, c0, cols, _ptr(re, _F64P),
                                     _ptr(im, _F64P))
    if rc != 0:
        raise ValueError("oracle_model_window rejected its arguments")
    return re + 1j * im


def model_wave_at(model: int, pitch_m: float, lambda_m: float, xyz, amp, cols, rows,
                  reference=(0.0, 0.0, 0.0)) -> np.ndarray:
    """model_wave at scattered pixels (cols[i], rows[i]), complex128."""
    xyz = _f32(xyz).reshape(-1, 3)
    amp = _f32(amp).reshape(-1)
    pm = np.ascontiguousarray(cols, dtype=np.int32)
    pn = np.ascontiguousarray(rows, dtype=np.int32)
    re = np.empty(pm.shape[0], dtype=np.float64)
    im = np.empty(pm.shape[0], dtype=np.float64)
    sx, sy, ph = (float(v) for v in reference)
    rc = _load().oracle_model_points(int(model), float(pitch_m), float(lambda_m), sx, sy, ph, _ptr(xyz, _F32P),
                                     _ptr(amp, _F32P), amp.shape[0], _ptr(pm, _I32P), _ptr(pn, _I32P),
                                     pm.shape[0], _ptr(re, _F64P), _ptr(im, _F64P))
    if rc != 0:
        raise ValueError("oracle_model_points rejected its arguments")
    return re + 1j * im


def _fresnel_prefactor(pitch_m: float, lambda_m: float, z_m: float) -> complex:
    """exp(i 2 pi z / lambda) / (i lambda z) * p^2 of Eq. 10 (the cell area p^2 turns the integral into a sum)."""
    zt = z_m / lambda_m
    a0 = 2 * np.pi * (zt - np.rint(zt))
    return np.exp(1j * a0) * (-1j) * pitch_m * pitch_m / (lambda_m * z_m)


def fresnel_at(u, pitch_m: float, lambda_m: float, z_m: float, cols, rows) -> np.ndarray:
    """Fresnel diffraction (Eq. 10) of the complex plane u [H][W] by z at scattered pixels, by its definition:
    O(m, n) = pre * sum_{m', n'} u(m', n') exp(i pi p^2 ((m - m')^2 + (n - n')^2) / (lambda z))."""
    u = np.asarray(u)
    H, W = u.shape
    ur = np.ascontiguousarray(u.real, dtype=np.float64)
    ui = np.ascontiguousarray(u.imag, dtype=np.float64)
    pm = np.ascontiguousarray(cols, dtype=np.int32)
    pn = np.ascontiguousarray(rows, dtype=np.int32)
    re = np.empty(pm.shape[0], dtype=np.float64)
    im = np.empty(pm.shape[0], dtype=np.float64)
    rc = _load().oracle_fresnel_points(W, H, float(pitch_m), float(lambda_m), float(z_m), _ptr(ur, _F64P),
                                       _ptr(ui, _F64P), _ptr(pm, _I32P), _ptr(pn, _I32P), pm.shape[0],
                                       _ptr(re, _F64P), _ptr(im, _F64P))
    if rc != 0:
        raise ValueError("oracle_fresnel_points rejected its arguments")
    return re + 1j * im


def fresnel(u, pitch_m: float, lambda_m: float, z_m: float) -> np.ndarray:
    """The same sum for every pixel: the linear convolution with the chirp evaluated by zero-padding to
    2H x 2W and numpy's complex128 FFT (a library step; pinned against fresnel_at), cropped to H x W."""
    u = np.asarray(u, dtype=np.complex128)
    H, W = u.shape
    n = np.arange(2 * H, dtype=np.int64)
    n = np.where(n < H, n, n - 2 * H)
    m = np.arange(2 * W, dtype=np.int64)
    m = np.where(m < W, m, m - 2 * W)
    c = pitch_m * pitch_m / (2.0 * lambda_m * z_m)
    t = c * (n[:, None] ** 2 + m[None, :] ** 2).astype(np.float64)
    h = np.exp(2j * np.pi * (t - np.rint(t)))
    pad = np.zeros((2 * H, 2 * W), dtype=np.complex128)
    pad[:H, :W] = u
    out = np.fft.ifft2(np.fft.fft2(pad) * np.fft.fft2(h))[:H, :W]
    return out * _fresnel_prefactor(pitch_m, lambda_m, z_m)


def wrp_window2(pitch_m: float, lambda_m: float, d_m: float) -> float:
    """floor(w^2), w = d s / sqrt(1 - s^2) / p, s = lambda / (2 p): the squared window radius in pixels
    (each operation rounded to double, as in the C oracle)."""
    s = lambda_m / (2.0 * pitch_m)
    w = ((d_m * s) / float(np.sqrt(1.0 - s * s))) / pitch_m
    return float(np.floor(w * w))


def wrp_record(model: int, pitch_m: float, lambda_m: float, z_wrp_m: float, xyz, amp, width: int, height: int,
               window: Optional[Sequence[int]] = None) -> np.ndarray:
    """WRP step 1 (Section 2.3): the windowed complex sum on the virtual plane at distance z_wrp from the
    hologram, model 0 or 1 at each point's distance d_j = z_j - z_wrp; complex128 [rows][cols]."""
    xyz = _f32(xyz).reshape(-1, 3)
    amp = _f32(amp).reshape(-1)
    if window is None:
        window = (0, 0, height, width)
    r0, c0, rows, cols = (int(v) for v in window)
    re = np.empty((rows, cols), dtype=np.float64)
    im = np.empty((rows, cols), dtype=np.float64)
    rc = _load().oracle_wrp_record(int(model), float(pitch_m), float(lambda_m), float(z_wrp_m), _ptr(xyz, _F32P),
                                   _ptr(amp, _F32P), amp.shape[0], r0, rows, c0, cols, _ptr(re, _F64P),
                                   _ptr(im, _F64P))
    if rc != 0:
        raise ValueError("oracle_wrp_record rejected its arguments")
    return re + 1j * im


def wrp(model: int, pitch_m: float, lambda_m: float, z_wrp_m: float, xyz, amp, width: int, height: int) -> np.ndarray:
    """The wavefront-recording method (Section 2.3): wrp_record, then Fresnel diffraction by z_wrp."""
    u = wrp_record(model, pitch_m, lambda_m, z_wrp_m, xyz, amp, width, height)
    return fresnel(u, pitch_m, lambda_m, z_wrp_m)


def factors(pitch_m: float, lambda_m: float, xyz, amp, width: int, height: int):
    """Separable factors (P [height][2N], Q [width][2N]) in FP64 with I = P Q^T."""
    xyz = _f32(xyz).reshape(-1, 3)
    amp = _f32(amp).reshape(-1)
    n = amp.shape[0]
    P = np.empty((height, 2 * n), dtype=np.float64)
    Q = np.empty((width, 2 * n), dtype=np.float64)
    rc = _load().oracle_factors(int(width), int(height), float(pitch_m), float(lambda_m),
                                _ptr(xyz, _F32P), _ptr(amp, _F32P), n, _ptr(P, _F64P), _ptr(Q, _F64P))
    if rc != 0:
        raise ValueError("oracle_factors rejected its arguments")
    return P, Q


def quantize8(field32) -> tuple:
    """Min/max 8-bit quantisation of a float32 field: (uint8 array, (lo, hi, s))."""
    f = _f32(field32)
    flat = f.reshape(-1)
    out = np.empty(flat.shape[0], dtype=np.uint8)
    lohi = np.zeros(3, dtype=np.float32)
    rc = _load().oracle_quantize8(_ptr(flat, _F32P), flat.shape[0], _ptr(out, _U8P), _ptr(lohi, _F32P))
    if rc != 0:
        raise ValueError("oracle_quantize8 rejected its arguments")
    return out.reshape(f.shape), (float(lohi[0]), float(lohi[1]), float(lohi[2]))


def kinoform8(wave_c) -> np.ndarray:
    """Phase-only 8-bit hologram of a complex field (Eq. 3; floor(255 psi/(2 pi)), psi in [0, 2 pi))."""
    w = np.asarray(wave_c)
    re = np.ascontiguousarray(w.real, dtype=np.float64).reshape(-1)
    im = np.ascontiguousarray(w.imag, dtype=np.float64).reshape(-1)
    out = np.empty(re.shape[0], dtype=np.uint8)
    rc = _load().oracle_kinoform8(_ptr(re, _F64P), _ptr(im, _F64P), re.shape[0], _ptr(out, _U8P))
    if rc != 0:
        raise ValueError("oracle_kinoform8 rejected its arguments")
    return out.reshape(w.shape)


def nrms(test, ref) -> float:
    """Normalised RMS error ||test - ref||_2 / ||ref||_2 in FP64."""
    t = np.asarray(test, dtype=np.float64)
    r = np.asarray(ref, dtype=np.float64)
    den = float(np.sqrt(np.sum(r * r)))
    num = float(np.sqrt(np.sum((t - r) ** 2)))
    return num / den if den > 0 else num


def recurrence_phases(c: Fraction, dx0: int, dy: int, steps: int):
    """Phases Gamma_1..Gamma_steps along a hologram row by Eqs. 6-8 (Section 2.2), exactly.

    Gamma_1 = P_j (dx0^2 + dy^2), delta_1 = P_j (2 dx0 + 1), Delta = 2 P_j with
    P_j = c the turn coefficient in px^-2; Gamma_{k+1} = Gamma_k + delta_k and
    delta_{k+1} = delta_k + Delta.  Gamma_k is the phase at dx = dx0 + k - 1.
    """
    g = c * (dx0 * dx0 + dy * dy)
    d = c * (2 * dx0 + 1)
    step = 2 * c
    out = []
    for _ in range(steps):
        out.append(g)
        g = g + d
        d = d + step
    return out
