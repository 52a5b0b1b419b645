"""Seeded synthetic point clouds shaped like the paper's CGH workloads.

This module only draws inputs.  It holds none of the hologram arithmetic, so
both the CUDA path and the FP64 oracle can consume the very same arrays.

Workload shapes follow the paper's direct-calculation experiments (Section 5,
Tables 3-4: a 1920x1080 hologram, 10^3 to 10^5 object points, 8 um pitch) and
the object model of Section 2.1 (N point light sources at (x_j, y_j, z_j) with
amplitude A_j).  Coordinates x_j, y_j are integers on the pixel grid (origin at
pixel (0, 0), m = column, n = row); z_j is in metres.  The paper's Fig. 3
object (11,646 points) is not available, so these seeded clouds stand in for
it.

Draw order per cloud is x, y, z, A from numpy's PCG64 ``default_rng(seed)``.
"""
from __future__ import annotations

import dataclasses
import math
from typing import List, Optional

import numpy as np

LAMBDA_M = 532e-9       # wavelength used by every workload (m)
PITCH_M = 8e-6          # hologram sampling pitch (m), as in the paper's listings


@dataclasses.dataclass
class Cloud:
    """One hologram problem: a point cloud and the hologram it is recorded on."""
    width: int
    height: int
    pitch_m: float
    lambda_m: float
    xyz: np.ndarray         # float32 [n][3]: x, y in pixel units (integers), z in metres
    amp: np.ndarray         # float32 [n]
    name: str = ""

    @property
    def n_points(self) -> int:
        return int(self.amp.shape[0])

    @property
    def evals(self) -> int:
        """Point-pixel evaluations W*H*N of one hologram."""
        return self.width * self.height * self.n_points


def _draw(rng: np.random.Generator, width: int, height: int, n: int,
          z_lo: float, z_hi: float, a_lo: float, a_hi: float,
          z_planes: Optional[np.ndarray] = None) -> tuple:
    x = rng.integers(0, width, size=n)
    y = rng.integers(0, height, size=n)
    if z_planes is None:
        z = rng.uniform(z_lo, z_hi, size=n)
    else:
        z = z_planes[rng.integers(0, len(z_planes), size=n)]
    a = rng.uniform(a_lo, a_hi, size=n)
    xyz = np.empty((n, 3), dtype=np.float32)
    xyz[:, 0] = x
    xyz[:, 1] = y
    xyz[:, 2] = z
    return xyz, a.astype(np.float32)


def random_cloud(seed: int, width: int, height: int, n: int,
                 z_range=(0.3, 1.0), a_range=(0.5, 1.0), name: str = "") -> Cloud:
    """A cloud with x ~ U{0..W-1}, y ~ U{0..H-1}, z ~ U[z_range], A ~ U[a_range]."""
    rng = np.random.default_rng(seed)
    xyz, amp = _draw(rng, width, height, n, z_range[0], z_range[1], a_range[0], a_range[1])
    return Cloud(width, height, PITCH_M, LAMBDA_M, xyz, amp, name or f"rand{width}x{height}n{n}")


def small_direct() -> Cloud:
    """256x256 hologram, 1,024 points, z ~ U[0.5, 1.0] m, A ~ U[0.5, 1.0]."""
    return random_cloud(13092734001, 256, 256, 1024, (0.5, 1.0), (0.5, 1.0), "direct-256x256-n1024")


def display_direct() -> Cloud:
    """1920x1080 hologram, 10,000 points, z ~ U[0.3, 1.0] m, A ~ U[0.5, 1.0]."""
    return random_cloud(13092734002, 1920, 1080, 10000, (0.3, 1.0), (0.5, 1.0), "direct-1920x1080-n10000")


def display_gemm() -> Cloud:
    """1920x1080 hologram, 50,000 points (same distributions as the display case)."""
    return random_cloud(13092734003, 1920, 1080, 50000, (0.3, 1.0), (0.5, 1.0), "gemm-1920x1080-n50000")


BATCH_SIZES = ((1024, 1024), (1920, 1080), (3840, 2160))


def video_batch(n_instances: int = 64, seed: int = 13092734004,
                n_lo: int = 1000, n_hi: int = 200000) -> List[Cloud]:
    """Frames of a holographic video: uneven point counts and hologram shapes.

    N_i = round(exp(U[ln n_lo, ln n_hi])); the hologram size is uniform over
    1024x1024, 1920x1080 and 3840x2160; otherwise as the display case.  Per
    instance the draw order is N_i, size_i, then x, y, z, A.
    """
    rng = np.random.default_rng(seed)
    out = []
    for i in range(n_instances):
        n = int(round(math.exp(rng.uniform(math.log(n_lo), math.log(n_hi)))))
        w, h = BATCH_SIZES[int(rng.integers(0, len(BATCH_SIZES)))]
        xyz, amp = _draw(rng, w, h, n, 0.3, 1.0, 0.5, 1.0)
        out.append(Cloud(w, h, PITCH_M, LAMBDA_M, xyz, amp, f"frame{i:02d}-{w}x{h}-n{n}"))
    return out


def depth_planes() -> np.ndarray:
    """Sixteen depth planes z_k = 0.2 + 0.8 k / 15 m, k = 0..15."""
    return 0.2 + 0.8 * np.arange(16) / 15.0


def large_layered(n: int = 1_000_000, size: int = 4096, seed: int = 13092734005) -> Cloud:
    """4096x4096 hologram, 10^6 points on 16 depth planes in [0.2, 1.0] m, A ~ U[0.1, 1.0]."""
    rng = np.random.default_rng(seed)
    xyz, amp = _draw(rng, size, size, n, 0.0, 0.0, 0.1, 1.0, z_planes=depth_planes())
    return Cloud(size, size, PITCH_M, LAMBDA_M, xyz, amp, f"layered-{size}x{size}-n{n}")


def layered_cloud(seed: int, width: int, height: int, n: int, n_planes: int,
                  x_range: Optional[tuple] = None, a_range=(0.1, 1.0)) -> Cloud:
    """A cloud on n_planes depth planes z_k = 0.2 + 0.8 k / max(n_planes - 1, 1) m.

    x ~ U{x_range[0] .. x_range[1] - 1} (default the hologram's columns), y ~ U{0..H-1},
    plane ~ U{0..n_planes-1}, A ~ U[a_range]: small stand-ins for the depth-layered case.
    """
    rng = np.random.default_rng(seed)
    planes = 0.2 + 0.8 * np.arange(n_planes) / max(n_planes - 1, 1)
    xyz, amp = _draw(rng, width, height, n, 0.0, 0.0, a_range[0], a_range[1], z_planes=planes)
    if x_range is not None:
        xyz[:, 0] = rng.integers(x_range[0], x_range[1], size=n)
    return Cloud(width, height, PITCH_M, LAMBDA_M, xyz, amp, f"layered{n_planes}-{width}x{height}-n{n}")


def wrp_cloud(seed: int, width: int, height: int, n: int, z_wrp: float = 0.5,
              d_range=(0.002, 0.010), a_range=(0.5, 1.0)) -> Cloud:
    """A cloud for the wavefront-recording method: x ~ U{0..W-1}, y ~ U{0..H-1}, z = z_wrp + U[d_range]
    (the object just behind the virtual plane), A ~ U[a_range]."""
    rng = np.random.default_rng(seed)
    xyz, amp = _draw(rng, width, height, n, z_wrp + d_range[0], z_wrp + d_range[1], a_range[0], a_range[1])
    return Cloud(width, height, PITCH_M, LAMBDA_M, xyz, amp, f"wrp-{width}x{height}-n{n}")


def complex_plane(seed: int, width: int, height: int) -> np.ndarray:
    """A random complex input plane [2][H][W] float32 (real, imaginary ~ N(0, 1)) for Fresnel diffraction."""
    rng = np.random.default_rng(seed)
    return rng.standard_normal((2, height, width)).astype(np.float32)


def large_crop(size: int = 4096, crop: int = 512) -> tuple:
    """(row0, col0, rows, cols) of the central crop compared for the large case."""
    r0 = (size - crop) // 2
    return r0, r0, crop, crop


WORKLOADS = {
    "direct-256x256-n1024": small_direct,
    "direct-1920x1080-n10000": display_direct,
    "gemm-1920x1080-n50000": display_gemm,
    "layered-4096x4096-n1000000": large_layered,
}
