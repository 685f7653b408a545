"""Seeded synthetic inputs shared by the tests, the benchmark and the oracle checks.

This module only *generates* inputs: direction sets, phantom volumes, noise and
random line data.  It holds none of the NUFFT arithmetic (no scaling factors,
no interpolation coefficients, no transforms), so both the CUDA path and the
FP64 oracle can consume the identical arrays it produces.

Workload recipes follow the paper's experiments: an N^3 volume (128^3 in
Sec. 3.2), 2N radial samples per line (Sec. 1, Eqs. 1.3-1.6 and the 2N rule
of Sec. 3.1), radial lines through the origin of 3D Fourier/Radon space whose
direction is given by an azimuth phi and an elevation theta (Eq. 2.1).  The
paper's Shepp-Logan and real-CT images are not available; seeded random
ellipsoid phantoms (plus Gaussian noise) stand in for them.
"""
from __future__ import annotations

import dataclasses
import math
from typing import List, Optional

import numpy as np

__all__ = [
    "umbrella_directions",
    "random_directions",
    "axis_directions",
    "Ellipsoid",
    "random_ellipsoids",
    "ellipsoid_volume",
    "gaussian_blob_volume",
    "random_volume",
    "random_lines",
    "Workload",
    "workload",
    "batched_workloads",
    "WORKLOADS",
]


# ----------------------------------------------------------------------------
# direction sets
# ----------------------------------------------------------------------------
def umbrella_directions(n_az: int, n_pol: int, cone_half_angle_deg: float = 15.0) -> np.ndarray:
    """Unit direction vectors of the radial lines, azimuth-major.

    Line l = a * n_pol + p has azimuth phi_a = 2*pi*a/n_az (the projection angle
    of the circular trajectory) and elevation
    theta_p = g + (pi - 2g) (p + 1/2) / n_pol with g the cone half-angle, so that
    theta stays inside [g, pi - g]: planes whose normal lies in the missing cone
    around the rotation axis are not sampled.  The Cartesian direction is
    (cos phi sin theta, sin phi sin theta, cos theta) (Eq. 2.1 with rho = 1).

    Returns a float64 array of shape (n_az * n_pol, 3) with columns (x, y, z).
    """
    if n_az <= 0 or n_pol <= 0:
        raise ValueError("n_az and n_pol must be positive")
    g = math.radians(cone_half_angle_deg)
    a = np.arange(n_az, dtype=np.float64)
    p = np.arange(n_pol, dtype=np.float64)
    phi = 2.0 * np.pi * a / n_az
    theta = g + (np.pi - 2.0 * g) * (p + 0.5) / n_pol
    ph, th = np.meshgrid(phi, theta, indexing="ij")  # [a][p]
    d = np.stack([np.cos(ph) * np.sin(th), np.sin(ph) * np.sin(th), np.cos(th)], axis=-1)
    return np.ascontiguousarray(d.reshape(-1, 3))


def random_directions(n: int, seed: int) -> np.ndarray:
    """n seeded directions uniform on the unit sphere (float64, (n, 3))."""
    rng = np.random.default_rng(seed)
    v = rng.normal(size=(n, 3))
    v /= np.linalg.norm(v, axis=1, keepdims=True)
    return np.ascontiguousarray(v)


def axis_directions() -> np.ndarray:
    """The three coordinate axes e_x, e_y, e_z (float64, (3, 3))."""
    return np.eye(3, dtype=np.float64)


# ----------------------------------------------------------------------------
# phantoms
# ----------------------------------------------------------------------------
@dataclasses.dataclass
class Ellipsoid:
    """A constant-density ellipsoid in field-of-view units ([-1/2, 1/2)^3).

    center: (3,) position (x, y, z); axes: (3,) semi-axes along the body frame;
    rot: (3, 3) rotation whose columns are the body axes in the lab frame;
    density: additive density (overlaps add).
    """

    center: np.ndarray
    axes: np.ndarray
    rot: np.ndarray
    density: float


def _quat_to_rot(q: np.ndarray) -> np.ndarray:
    w, x, y, z = q / np.linalg.norm(q)
    return np.array(
        [
            [1 - 2 * (y * y + z * z), 2 * (x * y - w * z), 2 * (x * z + w * y)],
            [2 * (x * y + w * z), 1 - 2 * (x * x + z * z), 2 * (y * z - w * x)],
            [2 * (x * z - w * y), 2 * (y * z + w * x), 1 - 2 * (x * x + y * y)],
        ]
    )


def random_ellipsoids(n_ell: int, seed: int, center_range: float = 0.4,
                      axes_range=(0.05, 0.3), density_range=(-0.5, 1.0)) -> List[Ellipsoid]:
    """Seeded random ellipsoids: centres U[-0.4, 0.4]^3, semi-axes U[0.05, 0.3],
    densities U[-0.5, 1], orientation from a uniformly random unit quaternion."""
    rng = np.random.default_rng(seed)
    out = []
    for _ in range(n_ell):
        c = rng.uniform(-center_range, center_range, size=3)
        a = rng.uniform(axes_range[0], axes_range[1], size=3)
        rho = float(rng.uniform(density_range[0], density_range[1]))
        q = rng.normal(size=4)
        out.append(Ellipsoid(center=c, axes=a, rot=_quat_to_rot(q), density=rho))
    return out


def ellipsoid_volume(n: int, ellipsoids: List[Ellipsoid], dtype=np.float32) -> np.ndarray:
    """Point-sample the ellipsoids at the voxel centres r = (j - n/2) / n.

    The array is C-ordered [z][y][x] (x fastest), shape (n, n, n).
    """
    coords = (np.arange(n, dtype=np.float64) - n // 2) / n
    vol = np.zeros((n, n, n), dtype=np.float64)
    zz, yy = np.meshgrid(coords, coords, indexing="ij")
    for e in ellipsoids:
        # body-frame coordinates: b = R^T (r - c); inside if sum (b_i / a_i)^2 <= 1
        rt = e.rot.T
        for ix in range(n):
            rx = coords[ix] - e.center[0]
            ry = yy - e.center[1]
            rz = zz - e.center[2]
            b0 = rt[0, 0] * rx + rt[0, 1] * ry + rt[0, 2] * rz
            b1 = rt[1, 0] * rx + rt[1, 1] * ry + rt[1, 2] * rz
            b2 = rt[2, 0] * rx + rt[2, 1] * ry + rt[2, 2] * rz
            inside = (b0 / e.axes[0]) ** 2 + (b1 / e.axes[1]) ** 2 + (b2 / e.axes[2]) ** 2 <= 1.0
            vol[:, :, ix] += e.density * inside
    return vol.astype(dtype)


def gaussian_blob_volume(n: int, center_vox, sigma_vox: float, amplitude: float = 1.0,
                         dtype=np.float64) -> np.ndarray:
    """amplitude * exp(-|m - c|^2 / (2 sigma^2)) sampled at the centred voxel
    indices m = j - n/2 (voxel units), C-ordered [z][y][x]."""
    m = np.arange(n, dtype=np.float64) - n // 2
    cx, cy, cz = (float(v) for v in center_vox)
    gx = np.exp(-((m - cx) ** 2) / (2 * sigma_vox ** 2))
    gy = np.exp(-((m - cy) ** 2) / (2 * sigma_vox ** 2))
    gz = np.exp(-((m - cz) ** 2) / (2 * sigma_vox ** 2))
    vol = amplitude * gz[:, None, None] * gy[None, :, None] * gx[None, None, :]
    return vol.astype(dtype)


def random_volume(n: int, seed: int, complex_values: bool = False, dtype=None) -> np.ndarray:
    """Seeded N(0, 1) volume (complex: independent real and imaginary parts)."""
    rng = np.random.default_rng(seed)
    if complex_values:
        v = rng.normal(size=(n, n, n)) + 1j * rng.normal(size=(n, n, n))
        return v.astype(dtype or np.complex128)
    return rng.normal(size=(n, n, n)).astype(dtype or np.float64)


def random_lines(n_dirs: int, m: int, seed: int, dtype=np.complex128) -> np.ndarray:
    """Seeded complex N(0, 1) line data of shape (n_dirs, m)."""
    rng = np.random.default_rng(seed)
    return (rng.normal(size=(n_dirs, m)) + 1j * rng.normal(size=(n_dirs, m))).astype(dtype)


# ----------------------------------------------------------------------------
# workload recipes
# ----------------------------------------------------------------------------
@dataclasses.dataclass
class Workload:
    """One projector problem: volume edge n, grid edge k, taps j, table
    oversampling table_oversamp, n_az x n_pol umbrella directions, m radial
    samples per line, phantom recipe and seed."""

    name: str
    n: int
    k: int
    j: int
    table_oversamp: int
    n_az: int
    n_pol: int
    m: int
    n_ellipsoids: int
    noise_sigma: float
    seed: int

    @property
    def n_dirs(self) -> int:
        return self.n_az * self.n_pol

    @property
    def n_points(self) -> int:
        return self.n_dirs * self.m

    def directions(self) -> np.ndarray:
        return umbrella_directions(self.n_az, self.n_pol, 15.0)

    def volume(self, dtype=np.float32) -> np.ndarray:
        ell = random_ellipsoids(self.n_ellipsoids, self.seed)
        vol = ellipsoid_volume(self.n, ell, dtype=np.float64)
        if self.noise_sigma > 0:
            rng = np.random.default_rng(self.seed + 1000)
            vol = vol + rng.normal(0.0, self.noise_sigma, size=vol.shape)
        return vol.astype(dtype)

    def ellipsoids(self) -> List[Ellipsoid]:
        return random_ellipsoids(self.n_ellipsoids, self.seed)


WORKLOADS = {
    # 32^3, 10 ellipsoids, K = 64, J = 6, L = 1024, 64 x 32 directions, M = 64
    "tiny32": Workload("tiny32", 32, 64, 6, 1024, 64, 32, 64, 10, 0.0, 0),
    # 128^3, K = 256, 180 x 128 directions, M = 256 (5.9M points)
    "mid128": Workload("mid128", 128, 256, 6, 1024, 180, 128, 256, 10, 0.0, 1),
    # 256^3 plus N(0, 0.01^2) noise, K = 512, 360 x 256 directions, M = 512 (47M points)
    "full256": Workload("full256", 256, 512, 6, 1024, 360, 256, 512, 10, 0.01, 2),
}


def workload(name: str) -> Workload:
    return WORKLOADS[name]


def batched_workloads(seed: int = 4) -> List[Workload]:
    """24 mixed problems: 8 each at 64^3, 128^3 and 192^3 (K = 2N, M = 2N),
    azimuth count drawn from {90, 180, 360} and polar count from {64, 128}."""
    rng = np.random.default_rng(seed)
    out = []
    idx = 0
    for n in (64, 128, 192):
        for _ in range(8):
            n_az = int(rng.choice([90, 180, 360]))
            n_pol = int(rng.choice([64, 128]))
            out.append(Workload(f"batch{idx}_{n}", n, 2 * n, 6, 1024, n_az, n_pol, 2 * n,
                                10, 0.0, seed + idx))
            idx += 1
    return out


def shifted_polar_targets(shape, shift, device=None):
    """Targets (u_s, u_theta, u_phi), in grid-index units, of every cell of a
    polar grid of shape (n_phi, n_theta, n_s) moved by shift = (ds, dtheta, dphi)
    cells: a resampling onto a shifted polar grid.  Rows in grid order (phi
    slowest, s fastest).  float32; a torch tensor on `device` if one is given
    (the 47 M targets of the 256^3 grid are made on the GPU), else NumPy."""
    n_phi, n_theta, n_s = (int(v) for v in shape)
    if device is not None:
        import torch

        p = torch.arange(n_phi, device=device, dtype=torch.float32) + float(shift[2])
        t = torch.arange(n_theta, device=device, dtype=torch.float32) + float(shift[1])
        s = torch.arange(n_s, device=device, dtype=torch.float32) + float(shift[0])
        P, Tt, Ss = torch.meshgrid(p, t, s, indexing="ij")
        return torch.stack([Ss.reshape(-1), Tt.reshape(-1), P.reshape(-1)], dim=1).contiguous()
    p = np.arange(n_phi, dtype=np.float32) + np.float32(shift[2])
    t = np.arange(n_theta, dtype=np.float32) + np.float32(shift[1])
    s = np.arange(n_s, dtype=np.float32) + np.float32(shift[0])
    P, Tt, Ss = np.meshgrid(p, t, s, indexing="ij")
    return np.stack([Ss.ravel(), Tt.ravel(), P.ravel()], axis=1)
