"""GB300-native point-cloud Fresnel hologram library (Python side).

The compute path is libcgh.so (C ABI in include/cgh.h, CUDA kernels for
sm_103a).  This package marshals torch CUDA tensors into that ABI: PyTorch
provides device memory and streams only.

    import torch
    from paper_1309_2734_gb300 import Hologram
    h = Hologram(1920, 1080, pitch_m=8e-6, lambda_m=532e-9, form="direct_sfu")
    field = h.point_cloud(xyz_cuda, amp_cuda)          # float32 [1080][1920]
    codes = h.quantize8(field)                         # uint8   [1080][1920]
"""
from __future__ import annotations

from . import _lib
from ._lib import (CGH_DIRECT_ACCURATE, CGH_DIRECT_SFU, CGH_FORM_AUTO, CGH_GEMM_BF16, CGH_GEMM_F16,
                   CGH_GEMM_SPLIT16, CGH_OPT_GEMM_BN, CGH_OPT_GEMM_SPLITK, CGH_OPT_POINT_SPLIT,
                   CGH_OPT_TIMEOUT_MS, CGH_OPT_TOLERANCE_E9, CGH_Q_AMPLITUDE_MINMAX, FORMS, CghError)

__all__ = ["Hologram", "CghError", "FORMS", "build_library", "batch"]


def build_library(force: bool = False) -> str:
    from .build import build
    return build(force=force)


def _need_cuda_tensor(t, name, dtype=None):
    import torch
    if not isinstance(t, torch.Tensor) or not t.is_cuda:
        raise TypeError(f"{name} must be a CUDA tensor")
    if not t.is_contiguous():
        raise ValueError(f"{name} must be contiguous")
    if dtype is not None and t.dtype != dtype:
        raise TypeError(f"{name} must be {dtype}")


class Hologram:
    """One context of the C ABI: a width x height hologram of pitch p and wavelength lambda."""

    def __init__(self, width: int, height: int, pitch_m: float, lambda_m: float, form="auto",
                 stream=None, timeout_ms: int = None):
        import torch
        self.width, self.height = int(width), int(height)
        self.pitch_m, self.lambda_m = float(pitch_m), float(lambda_m)
        self.device = torch.device("cuda", torch.cuda.current_device())
        self.ctx = _lib.cgh_create(self.width, self.height, self.pitch_m, self.lambda_m)
        self._stream = None
        self.set_stream(stream if stream is not None else torch.cuda.current_stream())
        self.set_form(form)
        if timeout_ms is not None:
            _lib.cgh_set_option(self.ctx, CGH_OPT_TIMEOUT_MS, timeout_ms)

    # -- configuration
    def set_stream(self, stream) -> None:
        self._stream = stream
        _lib.cgh_set_stream(self.ctx, stream.cuda_stream if stream is not None else 0)

    def set_form(self, form) -> None:
        _lib.cgh_set_form(self.ctx, form)

    def set_option(self, key: int, value: int) -> None:
        _lib.cgh_set_option(self.ctx, key, value)

    def set_phase_model(self, model) -> None:
        """'fresnel' (Eq. 5 without the piston, default), 'fresnel_piston' (Eq. 2) or 'spherical' (Eq. 1)."""
        models = {"fresnel": _lib.CGH_PHASE_FRESNEL, "fresnel_piston": _lib.CGH_PHASE_FRESNEL_PISTON,
                  "spherical": _lib.CGH_PHASE_SPHERICAL}
        _lib.cgh_set_option(self.ctx, _lib.CGH_OPT_PHASE_MODEL, models[model] if isinstance(model, str) else model)

    def set_reference(self, sin_x: float = 0.0, sin_y: float = 0.0, phase0_rad: float = 0.0) -> None:
        """Plane-wave reference of Eqs. 4-5: phi_r = 2 pi/lambda (x_h sin_x + y_h sin_y) + phase0."""
        _lib.cgh_set_reference(self.ctx, sin_x, sin_y, phase0_rad)

    # -- compute
    def point_cloud(self, xyz, amp, out=None):
        """I(m, n) of Eq. 5 (restricted form) as a float32 [height][width] CUDA tensor."""
        import torch
        _need_cuda_tensor(xyz, "xyz", torch.float32)
        _need_cuda_tensor(amp, "amp", torch.float32)
        n = int(amp.numel())
        if xyz.numel() != 3 * n:
            raise ValueError("xyz must be [n][3] with n = amp.numel()")
        if out is None:
            out = torch.empty((self.height, self.width), dtype=torch.float32, device=self.device)
        _need_cuda_tensor(out, "out", torch.float32)
        if out.numel() != self.width * self.height:
            raise ValueError("out must hold height * width floats")
        _lib.check(_lib.cgh_point_cloud(self.ctx, xyz.data_ptr() if n else 0, amp.data_ptr() if n else 0, n,
                                        out.data_ptr()), "cgh_point_cloud")
        return out

    def wave(self, xyz, amp, out=None):
        """Complex object wave as a float32 [2][height][width] CUDA tensor (real, imaginary)."""
        import torch
        _need_cuda_tensor(xyz, "xyz", torch.float32)
        _need_cuda_tensor(amp, "amp", torch.float32)
        n = int(amp.numel())
        if out is None:
            out = torch.empty((2, self.height, self.width), dtype=torch.float32, device=self.device)
        _need_cuda_tensor(out, "out", torch.float32)
        if out.numel() != 2 * self.width * self.height:
            raise ValueError("out must hold 2 * height * width floats")
        _lib.check(_lib.cgh_wave(self.ctx, xyz.data_ptr() if n else 0, amp.data_ptr() if n else 0, n,
                                 out.data_ptr()), "cgh_wave")
        return out

    def _planes_out(self, out):
        import torch
        if out is None:
            out = torch.empty((2, self.height, self.width), dtype=torch.float32, device=self.device)
        _need_cuda_tensor(out, "out", torch.float32)
        if out.numel() != 2 * self.width * self.height:
            raise ValueError("out must hold 2 * height * width floats")
        return out

    def fresnel(self, plane, z_m: float, out=None):
        """Fresnel diffraction (Eq. 10) of a complex plane [2][height][width] by z_m metres."""
        import torch
        _need_cuda_tensor(plane, "plane", torch.float32)
        if plane.numel() != 2 * self.width * self.height:
            raise ValueError("plane must hold 2 * height * width floats")
        out = self._planes_out(out)
        _lib.check(_lib.cgh_fresnel(self.ctx, plane.data_ptr(), float(z_m), out.data_ptr()), "cgh_fresnel")
        return out

    def wrp_record(self, xyz, amp, z_wrp_m: float, out=None):
        """Wavefront-recording method, step 1: the windowed complex sum on the plane at z_wrp_m (Section 2.3)."""
        import torch
        _need_cuda_tensor(xyz, "xyz", torch.float32)
        _need_cuda_tensor(amp, "amp", torch.float32)
        n = int(amp.numel())
        out = self._planes_out(out)
        _lib.check(_lib.cgh_wrp_record(self.ctx, xyz.data_ptr() if n else 0, amp.data_ptr() if n else 0, n,
                                       float(z_wrp_m), out.data_ptr()), "cgh_wrp_record")
        return out

    def wrp(self, xyz, amp, z_wrp_m: float, out=None):
        """Wavefront-recording method: the complex object wave on the hologram, [2][height][width]."""
        import torch
        _need_cuda_tensor(xyz, "xyz", torch.float32)
        _need_cuda_tensor(amp, "amp", torch.float32)
        n = int(amp.numel())
        out = self._planes_out(out)
        _lib.check(_lib.cgh_wrp(self.ctx, xyz.data_ptr() if n else 0, amp.data_ptr() if n else 0, n,
                                float(z_wrp_m), out.data_ptr()), "cgh_wrp")
        return out

    def kinoform8(self, wave, out=None):
        """Phase-only 8-bit hologram of a complex wave [2][...] (Eq. 3, the listings' 255/(2 pi) rule)."""
        import torch
        _need_cuda_tensor(wave, "wave", torch.float32)
        n = wave.numel() // 2
        if out is None:
            out = torch.empty(wave.shape[1:], dtype=torch.uint8, device=wave.device)
        _need_cuda_tensor(out, "out", torch.uint8)
        _lib.check(_lib.cgh_quantize8(self.ctx, wave.data_ptr(), n, _lib.CGH_Q_PHASE, out.data_ptr()),
                   "cgh_quantize8")
        return out

    def point_cloud_host(self, xyz_host, amp_host, out_host):
        """Same through host buffers (torch CPU tensors); copies inside, waits at the end."""
        import torch
        for t, name in ((xyz_host, "xyz"), (amp_host, "amp"), (out_host, "out")):
            if t.is_cuda or not t.is_contiguous() or t.dtype != torch.float32:
                raise TypeError(f"{name} must be a contiguous float32 CPU tensor")
        n = int(amp_host.numel())
        _lib.check(_lib.cgh_point_cloud_host(self.ctx, xyz_host.data_ptr(), amp_host.data_ptr(), n,
                                             out_host.data_ptr()), "cgh_point_cloud_host")
        return out_host

    def factors(self, xyz, amp, form="gemm_f16", ld=None):
        """The separable factors (P, Q) of the GEMM form, as CUDA tensors [rows][ld] (16-bit)."""
        import torch
        form = FORMS[form] if isinstance(form, str) else int(form)
        n = int(amp.numel())
        if ld is None:
            ld = max(64, (2 * n + 63) // 64 * 64)
        planes = 2 if form == CGH_GEMM_SPLIT16 else 1
        dt = torch.bfloat16 if form == CGH_GEMM_BF16 else torch.float16
        P = torch.empty((planes, self.height, ld), dtype=dt, device=self.device)
        Q = torch.empty((planes, self.width, ld), dtype=dt, device=self.device)
        _lib.check(_lib.cgh_factors(self.ctx, xyz.data_ptr() if n else 0, amp.data_ptr() if n else 0, n, form,
                                    P.data_ptr(), Q.data_ptr(), ld), "cgh_factors")
        return (P[0], Q[0]) if planes == 1 else (P, Q)

    def quantize8(self, field, out=None):
        """Min/max 8-bit quantisation of a float32 CUDA tensor."""
        import torch
        _need_cuda_tensor(field, "field", torch.float32)
        if out is None:
            out = torch.empty(field.shape, dtype=torch.uint8, device=field.device)
        _need_cuda_tensor(out, "out", torch.uint8)
        _lib.check(_lib.cgh_quantize8(self.ctx, field.data_ptr(), field.numel(), CGH_Q_AMPLITUDE_MINMAX,
                                      out.data_ptr()), "cgh_quantize8")
        return out

    def profile(self, on: bool = True) -> None:
        _lib.cgh_set_option(self.ctx, _lib.CGH_OPT_PROFILE, 1 if on else 0)

    def profile_read(self, reset: bool = True) -> dict:
        return _lib.cgh_profile_read(self.ctx, reset)

    def sync(self) -> None:
        _lib.check(_lib.cgh_sync(self.ctx), "cgh_sync")

    def close(self) -> None:
        if getattr(self, "ctx", None):
            _lib.cgh_destroy(self.ctx)
            self.ctx = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def __enter__(self):
        return self

    def __exit__(self, *exc):
        self.close()


def batch(ctx_holder: Hologram, clouds_dev, outs):
    """Runs cgh_batch over (xyz, amp, width, height, pitch, lambda) device tuples."""
    insts = []
    for (xyz, amp, w, h, p, lam), out in zip(clouds_dev, outs):
        n = int(amp.numel())
        insts.append(_lib.cgh_instance(int(w), int(h), float(p), float(lam),
                                       xyz.data_ptr() if n else None, amp.data_ptr() if n else None, n,
                                       out.data_ptr()))
    _lib.check(_lib.cgh_batch(ctx_holder.ctx, insts), "cgh_batch")
    return outs
