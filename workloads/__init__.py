"""Seeded synthetic inputs shared by the oracle, the tests and the benchmark.

This module holds input *data* only: the scatterer descriptions (a list of
voxels with their relative permittivity, or a general tetrahedral mesh given by
its vertices and tets), seeded random block vectors and plane-wave sets.  It contains none of the method's arithmetic (no mesh
splitting, no basis functions, no matrix entries, no compression): the
oracle and the CUDA library each build those from these inputs on their own.

Units: lambda0 = 1, so k0 = 2*pi.  Time convention exp(+j*omega*t) as in the
paper (Sec. II), so a lossy permittivity has a negative imaginary part.

Voxel rule (the scatterers of the workloads): a cubic grid of pitch h whose
cells have centres ((i+1/2)h, (j+1/2)h, (k+1/2)h); a voxel is kept when its
centre lies inside the body.  Voxels are listed in lexicographic (i, j, k)
order, i slowest.
"""
from __future__ import annotations

import dataclasses
import math
from typing import Callable

import numpy as np

K0 = 2.0 * math.pi  # lambda0 = 1


@dataclasses.dataclass(frozen=True)
class VoxelBody:
    """A scatterer on the voxel lattice: integer voxel indices, pitch, eps_r per voxel."""

    name: str
    h: float
    ijk: np.ndarray  # (nvox, 3) int32
    eps: np.ndarray  # (nvox,) complex128, relative permittivity per voxel

    @property
    def nvox(self) -> int:
        return int(self.ijk.shape[0])


def _select(h: float, extent: float, inside: Callable[[np.ndarray, np.ndarray, np.ndarray], np.ndarray]):
    m = int(math.ceil(extent / h)) + 1
    idx = np.arange(-m, m, dtype=np.int64)
    c = (idx + 0.5) * h
    x, y, z = np.meshgrid(c, c, c, indexing="ij")
    keep = inside(x, y, z)
    ii, jj, kk = np.meshgrid(idx, idx, idx, indexing="ij")
    ijk = np.stack([ii[keep], jj[keep], kk[keep]], axis=1).astype(np.int32)
    return ijk  # meshgrid 'ij' + boolean mask keeps lexicographic (i, j, k) order


def sphere(radius: float, eps: complex, h: float, name: str = "sphere") -> VoxelBody:
    ijk = _select(h, radius, lambda x, y, z: x * x + y * y + z * z < radius * radius)
    return VoxelBody(name, h, ijk, np.full(len(ijk), complex(eps), dtype=np.complex128))


def shell(r_out: float, r_in: float, eps: complex, h: float, name: str = "shell") -> VoxelBody:
    """Spherical shell; the core (eps_r = 1, zero contrast) is not meshed."""

    def inside(x, y, z):
        r2 = x * x + y * y + z * z
        return (r2 < r_out * r_out) & (r2 >= r_in * r_in)

    ijk = _select(h, r_out, inside)
    return VoxelBody(name, h, ijk, np.full(len(ijk), complex(eps), dtype=np.complex128))


def cube_grf(side: float, h: float, corr: float = 0.5, seed: int = 20211101,
             eps_lo: float = 1.0, eps_span: float = 49.0, name: str = "cube_grf") -> VoxelBody:
    """Cube of the given side with eps_r = eps_lo + eps_span * u per voxel.

    u = Phi(z) where z is a standardized stationary Gaussian random field with
    squared-exponential covariance exp(-|d|^2 / (2 corr^2)), synthesized by FFT
    on the voxel centres (seeded), and Phi is the standard normal CDF.
    """
    n = int(round(side / h))
    half = n // 2
    idx = np.arange(-half, n - half, dtype=np.int64)
    ii, jj, kk = np.meshgrid(idx, idx, idx, indexing="ij")
    ijk = np.stack([ii.ravel(), jj.ravel(), kk.ravel()], axis=1).astype(np.int32)
    rng = np.random.default_rng(seed)
    m = 2 * n  # padded periodic grid to limit wrap-around correlation
    f = np.fft.fftfreq(m, d=h)
    fx, fy, fz = np.meshgrid(f, f, f, indexing="ij")
    k2 = (2 * np.pi) ** 2 * (fx * fx + fy * fy + fz * fz)
    spec = np.exp(-0.5 * k2 * corr * corr)  # PSD of the squared-exponential covariance (up to scale)
    white = rng.standard_normal((m, m, m))
    field = np.fft.ifftn(np.fft.fftn(white) * np.sqrt(spec)).real[:n, :n, :n]
    z = (field - field.mean()) / field.std()
    from scipy.special import ndtr

    u = ndtr(z).ravel()
    eps = (eps_lo + eps_span * u).astype(np.complex128)
    return VoxelBody(name, h, ijk, eps)


@dataclasses.dataclass(frozen=True)
class TetMesh:
    """A general tetrahedral mesh given as data: vertex coordinates, 4 vertex ids per tet
    (any orientation) and eps_r per tet."""

    name: str
    verts: np.ndarray  # (nv, 3) float64
    tets: np.ndarray   # (nt, 4) int32
    eps: np.ndarray    # (nt,) complex128


# the five tetrahedra of a unit cube (corner bits x, y, z), by cube parity: for even cubes
# the tet of the four even corners plus one tet per odd corner, for odd cubes the mirror;
# neighbouring cubes have opposite parity and share their face diagonals
_CUBE5 = {
    0: [[0b000, 0b110, 0b101, 0b011], [0b100, 0b000, 0b110, 0b101], [0b010, 0b000, 0b110, 0b011],
        [0b001, 0b000, 0b101, 0b011], [0b111, 0b110, 0b101, 0b011]],
    1: [[0b100, 0b010, 0b001, 0b111], [0b000, 0b100, 0b010, 0b001], [0b110, 0b100, 0b010, 0b111],
        [0b101, 0b100, 0b001, 0b111], [0b011, 0b010, 0b001, 0b111]],
}


def tet_body(body: VoxelBody, jitter: float = 0.08, seed: int = 5, name: str | None = None) -> TetMesh:
    """The voxels of ``body`` cut into five tetrahedra each (alternating cube parity, a
    conforming mesh unlike the Kuhn split), with every vertex moved by a seeded uniform
    offset of up to ``jitter`` * h per coordinate, so the elements are off any lattice.
    Vertices are the distinct lattice corners in lexicographic order; tets are
    voxel-major, five per voxel; eps_r of a tet is that of its voxel."""
    ijk = np.asarray(body.ijk, dtype=np.int64)
    corners = []
    for v in ijk:
        par = int(v.sum()) % 2
        for t in _CUBE5[par]:
            corners.append([[v[0] + (c >> 2 & 1), v[1] + (c >> 1 & 1), v[2] + (c & 1)] for c in t])
    lat = np.asarray(corners, dtype=np.int64)  # (nt, 4, 3)
    uniq, inv = np.unique(lat.reshape(-1, 3), axis=0, return_inverse=True)
    rng = np.random.default_rng(seed)
    verts = (uniq.astype(np.float64) + rng.uniform(-jitter, jitter, size=uniq.shape)) * body.h
    tets = inv.reshape(-1, 4).astype(np.int32)
    eps = np.repeat(np.asarray(body.eps, dtype=np.complex128), 5)
    return TetMesh(name or body.name + "_tet5", verts, tets, eps)


# --------------------------------------------------------------------------------------
# Named workloads (sizes follow the voxel rule; N = 12 * nvox + exposed voxel faces)
# --------------------------------------------------------------------------------------

def sphere_small_fp64(h: float = 1.0 / 20) -> VoxelBody:
    """Homogeneous lossless sphere r = 0.3, eps_r = 4, pitch lambda_d/10 = 1/20 (N = 11,616)."""
    return sphere(0.3, 4.0, h, name="sphere_r0.3_eps4")


def sphere_large_c32(h: float = 1.0 / 10) -> VoxelBody:
    """Homogeneous lossy sphere r = 2, eps_r = 4 - 0.1j, pitch 1/10 (N = 410,208)."""
    return sphere(2.0, 4.0 - 0.1j, h, name="sphere_r2_eps4-0.1j")


def drude_eps(wp_over_w: float = 1.8, nu_over_w: float = 0.05) -> complex:
    """Drude permittivity 1 - wp^2 / (w (w - j nu)) in the exp(+j w t) convention."""
    return 1.0 - wp_over_w ** 2 / (1.0 * (1.0 - 1j * nu_over_w))


def plasma_shell(h: float = 1.0 / 20) -> VoxelBody:
    """Plasma shell 1.5 / 1.2, Drude eps_r ~ -2.23 - 0.16j, vacuum core (N = 690,768)."""
    return shell(1.5, 1.2, drude_eps(), h, name="plasma_shell")


def tiny_block(nx: int = 2, ny: int = 1, nz: int = 1, h: float = 0.1, eps: complex = 4.0) -> VoxelBody:
    """A small box of voxels (for brute-force and unit tests)."""
    ii, jj, kk = np.meshgrid(np.arange(nx), np.arange(ny), np.arange(nz), indexing="ij")
    ijk = np.stack([ii.ravel(), jj.ravel(), kk.ravel()], axis=1).astype(np.int32)
    return VoxelBody(f"block{nx}x{ny}x{nz}", h, ijk, np.full(len(ijk), complex(eps), dtype=np.complex128))


def layered_eps(body: VoxelBody, radii, eps_values) -> VoxelBody:
    """Assign eps per voxel by the radius of its centre: eps_values[i] for radii[i+1] <= r < radii[i]."""
    c = (body.ijk.astype(np.float64) + 0.5) * body.h
    r = np.sqrt((c * c).sum(1))
    eps = body.eps.copy()
    for i, e in enumerate(eps_values):
        lo = radii[i + 1] if i + 1 < len(radii) else -1.0
        eps[(r < radii[i]) & (r >= lo)] = e
    return VoxelBody(body.name + "_layered", body.h, body.ijk, eps)


def five_layer_sphere(h: float = 1.0 / 20) -> VoxelBody:
    """Five concentric layers of thickness 0.1 lambda0 (outer radius 0.5), eps_r 2, 3, 4, 5, 6
    from the outside in: the layered-sphere geometry of Sec. IV-A at a GPU-test size."""
    radii = [0.5, 0.4, 0.3, 0.2, 0.1]
    return layered_eps(sphere(radii[0], 2.0, h, name="five_layer_sphere"), radii, [2.0, 3.0, 4.0, 5.0, 6.0])


def two_shell_sphere(h: float = 1.0 / 20) -> VoxelBody:
    """Hollow sphere of two 0.1 lambda0 shells (outer radius 0.5, vacuum core of radius 0.3, not
    meshed), eps_r 4 inside and 2 outside: the two-shell geometry of Sec. IV-A at a GPU-test size."""
    body = shell(0.5, 0.3, 2.0, h, name="two_shell_sphere")
    return layered_eps(body, [0.5, 0.4], [2.0, 4.0])


def equal_volume_layers(h: float, radii):
    """Radii of the spheres with the volume of the grid voxels (pitch h, centres (i + 1/2) h)
    whose centres lie inside each radius: the staircase's equal-volume layer radii."""
    out = []
    for R in radii:
        n = int(math.ceil(R / h)) + 1
        c = (np.arange(-n, n, dtype=np.float64) + 0.5) * h
        x, y, z = np.meshgrid(c, c, c, indexing="ij")
        cnt = np.count_nonzero(x * x + y * y + z * z < R * R)
        out.append((3.0 * cnt * h ** 3 / (4.0 * math.pi)) ** (1.0 / 3.0))
    return out


# --------------------------------------------------------------------------------------
# Seeded vectors and excitations
# --------------------------------------------------------------------------------------

def random_block(n: int, nrhs: int, seed: int, dtype=np.complex128) -> np.ndarray:
    """Column-major-friendly (n, nrhs) complex Gaussian block, seeded."""
    rng = np.random.default_rng(seed)
    x = rng.standard_normal((n, nrhs)) + 1j * rng.standard_normal((n, nrhs))
    return (x / math.sqrt(2.0)).astype(dtype)


def planewave_x_along_z():
    """x-polarized plane wave travelling along +z: (khat, pol)."""
    return np.array([[0.0, 0.0, 1.0]]), np.array([[1.0, 0.0, 0.0]])


def planewave_grid(ntheta: int = 8, nphi: int = 16):
    """Plane waves on a (theta, phi) grid with both polarizations (theta-hat, phi-hat).

    theta_i = (i + 1/2) pi / ntheta, phi_j = 2 pi j / nphi; returns (khat, pol) arrays
    of shape (2 * ntheta * nphi, 3).  The wave travels along khat.
    """
    th = (np.arange(ntheta) + 0.5) * np.pi / ntheta
    ph = 2 * np.pi * np.arange(nphi) / nphi
    T, P = np.meshgrid(th, ph, indexing="ij")
    T, P = T.ravel(), P.ravel()
    k = np.stack([np.sin(T) * np.cos(P), np.sin(T) * np.sin(P), np.cos(T)], 1)
    et = np.stack([np.cos(T) * np.cos(P), np.cos(T) * np.sin(P), -np.sin(T)], 1)
    ep = np.stack([-np.sin(P), np.cos(P), np.zeros_like(P)], 1)
    return np.concatenate([k, k]), np.concatenate([et, ep])


def planewave_random(nrhs: int, seed: int):
    """Random incidence directions uniform on the sphere, random unit polarization orthogonal to khat."""
    rng = np.random.default_rng(seed)
    k = rng.standard_normal((nrhs, 3))
    k /= np.linalg.norm(k, axis=1, keepdims=True)
    a = rng.standard_normal((nrhs, 3))
    a -= (a * k).sum(1, keepdims=True) * k
    a /= np.linalg.norm(a, axis=1, keepdims=True)
    return k, a
