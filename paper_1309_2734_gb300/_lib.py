"""ctypes binding of libcgh.so (include/cgh.h).  Argument marshalling only.

Every function here has the name of the C entry point it calls and passes
plain pointers and sizes; all hologram arithmetic runs in the CUDA kernels
behind the C ABI.  If the library is missing, loading raises: there is no
CPU fallback.
"""
from __future__ import annotations

import ctypes
import os
import threading

HERE = os.path.dirname(os.path.abspath(__file__))
# CGH_LIB_VARIANT=debug loads the debug build (device-side bounds checks, python -m paper_1309_2734_gb300.build
# --debug) instead of the release library
LIB_PATH = os.path.join(HERE, "libcgh_debug.so" if os.environ.get("CGH_LIB_VARIANT") == "debug" else "libcgh.so")

# status codes
CGH_OK, CGH_EINVAL, CGH_ENOMEM, CGH_ECUDA, CGH_ETIMEOUT, CGH_EINPUT, CGH_ENOTSUP, CGH_EBOUNDS = range(8)
# forms
CGH_FORM_AUTO, CGH_DIRECT_SFU, CGH_DIRECT_ACCURATE, CGH_GEMM_F16, CGH_GEMM_BF16, CGH_GEMM_SPLIT16 = range(6)
FORMS = {"auto": 0, "direct_sfu": 1, "direct_accurate": 2, "gemm_f16": 3, "gemm_bf16": 4, "gemm_split16": 5}
# quantiser modes
CGH_Q_AMPLITUDE_MINMAX = 0
CGH_Q_PHASE = 1
# options
CGH_OPT_TIMEOUT_MS, CGH_OPT_POINT_SPLIT, CGH_OPT_GEMM_SPLITK, CGH_OPT_GEMM_BN, CGH_OPT_TOLERANCE_E9 = 1, 2, 3, 4, 5
CGH_OPT_PROFILE = 6
CGH_OPT_GEMM_CHUNK = 7
CGH_OPT_TEST_DROP_TILE = 8
CGH_OPT_FACTOR_BUDGET_MB = 9
CGH_OPT_GEMM_PIPELINE = 10
CGH_OPT_GEMM_TRANSPOSE = 11
CGH_OPT_GEMM_GROUP = 12
CGH_OPT_PHASE_MODEL = 13
CGH_OPT_DIRECT_CTAS = 14
CGH_OPT_BATCH_MODE = 15
CGH_OPT_BATCH_OVERLAP = 16
CGH_OPT_TEST_ALLOC_FAIL = 17
CGH_OPT_DIRECT_SHAPE = 18
CGH_OPT_GEMM_PERSISTENT = 19
CGH_OPT_GEMM_PAIR = 20
CGH_OPT_BATCH_CHUNK_MB = 21
CGH_OPT_BATCH_PREMADE_PCT = 22
CGH_PHASE_FRESNEL, CGH_PHASE_FRESNEL_PISTON, CGH_PHASE_SPHERICAL = 0, 1, 2

EXPORTS = ("cgh_abi_version", "cgh_status_string", "cgh_create", "cgh_destroy", "cgh_set_stream",
           "cgh_set_form", "cgh_set_option", "cgh_point_cloud", "cgh_point_cloud_host", "cgh_factors",
           "cgh_batch", "cgh_quantize8", "cgh_profile_read", "cgh_sync", "cgh_point_cloud_noalloc",
           "cgh_autotune", "cgh_wave", "cgh_set_reference", "cgh_fresnel", "cgh_wrp_record", "cgh_wrp",
           "cgh_measure_mufu", "cgh_batch_forms", "cgh_tune_cache_check", "cgh_gemm_layout")
CGH_NOALLOC_MAX_POINTS = 131072


class cgh_instance(ctypes.Structure):
    _fields_ = [("width", ctypes.c_int), ("height", ctypes.c_int),
                ("pitch_m", ctypes.c_double), ("lambda_m", ctypes.c_double),
                ("d_xyz", ctypes.c_void_p), ("d_amp", ctypes.c_void_p),
                ("n_points", ctypes.c_int64), ("d_out", ctypes.c_void_p)]


class cgh_kernel_time(ctypes.Structure):
    _fields_ = [("name", ctypes.c_char * 32), ("launches", ctypes.c_int64), ("total_ms", ctypes.c_double)]


class CghError(RuntimeError):
    def __init__(self, code: int, where: str):
        self.code = code
        super().__init__(f"{where}: {status_string(code)} (status {code})")


_lib = None
_lock = threading.Lock()


def load(path: str = LIB_PATH) -> ctypes.CDLL:
    """Loads libcgh.so once; raises if it has not been built."""
    global _lib
    with _lock:
        if _lib is not None:
            return _lib
        if not os.path.exists(path):
            raise RuntimeError(f"{os.path.basename(path)} not found at {path}; build it with "
                               "`python -m paper_1309_2734_gb300.build` (no CPU fallback exists)")
        lib = ctypes.CDLL(path)
        vp, i64, ci, cd = ctypes.c_void_p, ctypes.c_int64, ctypes.c_int, ctypes.c_double
        sig = {
            "cgh_abi_version": ([], ci),
            "cgh_status_string": ([ci], ctypes.c_char_p),
            "cgh_create": ([ci, ci, cd, cd, ctypes.POINTER(vp)], ci),
            "cgh_destroy": ([vp], ci),
            "cgh_set_stream": ([vp, vp], ci),
            "cgh_set_form": ([vp, ci], ci),
            "cgh_set_option": ([vp, ci, i64], ci),
            "cgh_point_cloud": ([vp, vp, vp, i64, vp], ci),
            "cgh_point_cloud_host": ([vp, vp, vp, i64, vp], ci),
            "cgh_factors": ([vp, vp, vp, i64, ci, vp, vp, i64], ci),
            "cgh_batch": ([vp, ctypes.POINTER(cgh_instance), ci], ci),
            "cgh_batch_forms": ([vp, ctypes.POINTER(ci), ci, ctypes.POINTER(ci)], ci),
            "cgh_tune_cache_check": ([ctypes.c_char_p, ctypes.c_char_p, ctypes.POINTER(ci)], ci),
            "cgh_gemm_layout": ([ci, ci, i64, ci, ci, ctypes.POINTER(ci)], ci),
            "cgh_quantize8": ([vp, vp, i64, ci, vp], ci),
            "cgh_profile_read": ([vp, ctypes.POINTER(cgh_kernel_time), ci, ctypes.POINTER(ci), ci], ci),
            "cgh_sync": ([vp], ci),
            "cgh_point_cloud_noalloc": ([ci, ci, cd, cd, vp, vp, i64, vp, vp], ci),
            "cgh_autotune": ([vp, ci], ci),
            "cgh_wave": ([vp, vp, vp, i64, vp], ci),
            "cgh_set_reference": ([vp, cd, cd, cd], ci),
            "cgh_fresnel": ([vp, vp, cd, vp], ci),
            "cgh_wrp_record": ([vp, vp, vp, i64, cd, vp], ci),
            "cgh_wrp": ([vp, vp, vp, i64, cd, vp], ci),
            "cgh_measure_mufu": ([vp, ctypes.POINTER(cd)], ci),
        }
        for name, (args, res) in sig.items():
            fn = getattr(lib, name)
            fn.argtypes = args
            fn.restype = res
        _lib = lib
        return lib


def status_string(code: int) -> str:
    try:
        return load().cgh_status_string(int(code)).decode()
    except RuntimeError:
        return f"status {code}"


def check(code: int, where: str) -> None:
    if code != CGH_OK:
        raise CghError(code, where)


# --- thin wrappers with the C names -------------------------------------------------

def cgh_create(width: int, height: int, pitch_m: float, lambda_m: float) -> int:
    h = ctypes.c_void_p()
    check(load().cgh_create(int(width), int(height), float(pitch_m), float(lambda_m), ctypes.byref(h)),
          "cgh_create")
    return h.value


def cgh_destroy(ctx: int) -> int:
    return load().cgh_destroy(ctx)


def cgh_set_stream(ctx: int, stream_handle: int) -> None:
    check(load().cgh_set_stream(ctx, stream_handle), "cgh_set_stream")


def cgh_set_form(ctx: int, form) -> None:
    form = FORMS[form] if isinstance(form, str) else int(form)
    check(load().cgh_set_form(ctx, form), "cgh_set_form")


def cgh_set_option(ctx: int, key: int, value: int) -> None:
    check(load().cgh_set_option(ctx, int(key), int(value)), "cgh_set_option")


def cgh_set_reference(ctx: int, sin_x: float, sin_y: float, phase0_rad: float) -> None:
    check(load().cgh_set_reference(ctx, float(sin_x), float(sin_y), float(phase0_rad)), "cgh_set_reference")


def cgh_point_cloud(ctx: int, d_xyz: int, d_amp: int, n_points: int, d_out: int) -> int:
    return load().cgh_point_cloud(ctx, d_xyz, d_amp, int(n_points), d_out)


def cgh_point_cloud_host(ctx: int, h_xyz: int, h_amp: int, n_points: int, h_out: int) -> int:
    return load().cgh_point_cloud_host(ctx, h_xyz, h_amp, int(n_points), h_out)


def cgh_factors(ctx: int, d_xyz: int, d_amp: int, n_points: int, dtype_form: int, d_p: int, d_q: int,
                ld: int) -> int:
    return load().cgh_factors(ctx, d_xyz, d_amp, int(n_points), int(dtype_form), d_p, d_q, int(ld))


def cgh_batch(ctx: int, instances) -> int:
    arr = (cgh_instance * len(instances))(*instances)
    return load().cgh_batch(ctx, arr, len(instances))


def cgh_batch_forms(ctx: int, max_entries: int = 4096) -> list:
    """The forms the last cgh_batch plan chose, one per instance."""
    buf = (ctypes.c_int * max(1, max_entries))()
    n = ctypes.c_int(0)
    check(load().cgh_batch_forms(ctx, buf, max_entries, ctypes.byref(n)), "cgh_batch_forms")
    return [int(buf[i]) for i in range(min(n.value, max_entries))]


def cgh_tune_cache_check(path: str, device_name: str) -> bool:
    """Whether the autotuner would accept the cache file at path for the device (no GPU needed)."""
    ok = ctypes.c_int(0)
    check(load().cgh_tune_cache_check(path.encode(), device_name.encode(), ctypes.byref(ok)),
          "cgh_tune_cache_check")
    return ok.value == 1


def cgh_gemm_layout(width: int, height: int, n_points: int, form: int, num_sms: int) -> dict:
    """The GEMM launch shape cgh_point_cloud takes at default options (no GPU needed)."""
    out = (ctypes.c_int * 4)()
    check(load().cgh_gemm_layout(int(width), int(height), int(n_points), int(form), int(num_sms), out),
          "cgh_gemm_layout")
    return {"transposed": bool(out[0]), "bn": int(out[1]), "splits": int(out[2]), "pair": bool(out[3])}


def cgh_quantize8(ctx: int, d_field: int, n: int, mode: int, d_out: int) -> int:
    return load().cgh_quantize8(ctx, d_field, int(n), int(mode), d_out)


def cgh_profile_read(ctx: int, reset: bool = True) -> dict:
    """{kernel name: (launches, total device ms)} recorded while CGH_OPT_PROFILE was on."""
    buf = (cgh_kernel_time * 64)()
    n = ctypes.c_int(0)
    check(load().cgh_profile_read(ctx, buf, 64, ctypes.byref(n), 1 if reset else 0), "cgh_profile_read")
    return {buf[i].name.decode(): (int(buf[i].launches), float(buf[i].total_ms)) for i in range(min(n.value, 64))}


def cgh_wave(ctx: int, d_xyz: int, d_amp: int, n_points: int, d_out: int) -> int:
    return load().cgh_wave(ctx, d_xyz, d_amp, int(n_points), d_out)


def cgh_measure_mufu(ctx: int) -> float:
    """Measured hardware-sine results per second of the whole GPU."""
    v = ctypes.c_double(0.0)
    check(load().cgh_measure_mufu(ctx, ctypes.byref(v)), "cgh_measure_mufu")
    return float(v.value)


def cgh_fresnel(ctx: int, d_in: int, z_m: float, d_out: int) -> int:
    return load().cgh_fresnel(ctx, d_in, float(z_m), d_out)


def cgh_wrp_record(ctx: int, d_xyz: int, d_amp: int, n_points: int, z_wrp_m: float, d_plane: int) -> int:
    return load().cgh_wrp_record(ctx, d_xyz, d_amp, int(n_points), float(z_wrp_m), d_plane)


def cgh_wrp(ctx: int, d_xyz: int, d_amp: int, n_points: int, z_wrp_m: float, d_out: int) -> int:
    return load().cgh_wrp(ctx, d_xyz, d_amp, int(n_points), float(z_wrp_m), d_out)


def cgh_autotune(ctx: int, force: bool = False) -> int:
    return load().cgh_autotune(ctx, 1 if force else 0)


def cgh_sync(ctx: int) -> int:
    return load().cgh_sync(ctx)


def cgh_point_cloud_noalloc(width: int, height: int, pitch_m: float, lambda_m: float, d_xyz: int, d_amp: int,
                            n_points: int, d_out: int, stream_handle: int = 0) -> int:
    """The context-free, allocation-free direct hologram (see include/cgh.h)."""
    return load().cgh_point_cloud_noalloc(int(width), int(height), float(pitch_m), float(lambda_m), d_xyz, d_amp,
                                          int(n_points), d_out, stream_handle)
