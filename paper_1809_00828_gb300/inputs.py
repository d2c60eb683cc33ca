"""Seeded synthetic inputs shared by the CUDA path, the oracle tests and the bench.

This module holds no arithmetic of the finite cell method: it only draws
geometries (sphere lists, half-spaces, voxel images) and random vectors from
seeds, and names the workload families.  Both the CPU oracle and the GPU
library consume the arrays it returns.

Random numbers come from SplitMix64 (G. Steele, D. Lea, C. Flood, "Fast
splittable pseudorandom number generators", OOPSLA 2014), mapped to doubles in
[0, 1) by taking the top 53 bits.

The paper's own workloads are CT scans (a lumbar vertebra, Sec. 5.2, and a
gearbox housing, Sec. 5.3) that are not available; the families below stand in
for them: a unit cube with one or many spherical voids (the cube with a
spherical cavity of Sec. 5.1 and its porous generalisation) and a thresholded
Gaussian random field for trabecular-like bone.
"""
from __future__ import annotations

import dataclasses
import math

import numpy as np

_MASK64 = (1 << 64) - 1


class SplitMix64:
    """SplitMix64 stream (Steele, Lea, Flood 2014)."""

    def __init__(self, seed: int):
        self.state = seed & _MASK64

    def next_u64(self) -> int:
        self.state = (self.state + 0x9E3779B97F4A7C15) & _MASK64
        z = self.state
        z = ((z ^ (z >> 30)) * 0xBF58476D1CE4E5B9) & _MASK64
        z = ((z ^ (z >> 27)) * 0x94D049BB133111EB) & _MASK64
        return z ^ (z >> 31)

    def uniform(self) -> float:
        """Double in [0, 1) from the top 53 bits."""
        return (self.next_u64() >> 11) * (1.0 / (1 << 53))

    def uniform_range(self, a: float, b: float) -> float:
        return a + (b - a) * self.uniform()


# Geometry kinds understood by both the oracle and the library.
GEOM_SPHERE_VOIDS = 0  # solid = box minus the union of open balls
GEOM_VOXELS = 1        # solid = voxels with value != 0 on a regular image over the box
GEOM_HALFSPACE = 2     # solid = {x : a.x < d}


@dataclasses.dataclass
class Geometry:
    kind: int
    spheres: np.ndarray | None = None    # (m, 4) float64: cx, cy, cz, r
    voxels: np.ndarray | None = None     # (nz, ny, nx) uint8, x fastest in memory
    plane: tuple = (0.0, 0.0, 1.0, 2.0)  # a, b, c, d: solid iff a x + b y + c z < d
    octree_depth: int = 3

    def sphere_array(self) -> np.ndarray:
        if self.spheres is None:
            return np.zeros((0, 4), dtype=np.float64)
        return np.ascontiguousarray(self.spheres, dtype=np.float64)


def single_sphere_void(seed: int, radius: float = 0.3, jitter: float = 0.05,
                       octree_depth: int = 3) -> Geometry:
    """One spherical void of fixed radius, centre 0.5 + U(-jitter, jitter) per axis."""
    g = SplitMix64(seed)
    c = [0.5 + g.uniform_range(-jitter, jitter) for _ in range(3)]
    sph = np.array([[c[0], c[1], c[2], radius]], dtype=np.float64)
    return Geometry(GEOM_SPHERE_VOIDS, spheres=sph, octree_depth=octree_depth)


def random_sphere_voids(seed: int, count: int, rmin: float, rmax: float,
                        octree_depth: int = 3) -> Geometry:
    """`count` spherical voids, centres U[0,1)^3, radii U(rmin, rmax).

    Per sphere the draws are cx, cy, cz, r in that order.  Overlaps and
    crossings of the cube boundary are allowed.
    """
    g = SplitMix64(seed)
    out = np.empty((count, 4), dtype=np.float64)
    for i in range(count):
        cx, cy, cz = g.uniform(), g.uniform(), g.uniform()
        r = g.uniform_range(rmin, rmax)
        out[i] = (cx, cy, cz, r)
    return Geometry(GEOM_SPHERE_VOIDS, spheres=out, octree_depth=octree_depth)


def halfspace(a: float, b: float, c: float, d: float, octree_depth: int = 3) -> Geometry:
    return Geometry(GEOM_HALFSPACE, plane=(a, b, c, d), octree_depth=octree_depth)


def uncut() -> Geometry:
    """The whole box is solid (no voids)."""
    return Geometry(GEOM_SPHERE_VOIDS, spheres=np.zeros((0, 4)), octree_depth=0)


def splitmix_uniforms(seed: int, n: int) -> np.ndarray:
    """n doubles in [0, 1) from the SplitMix64 stream of `seed` (vectorised, same stream as `uniform`)."""
    k = np.arange(1, n + 1, dtype=np.uint64)
    with np.errstate(over="ignore"):
        z = np.uint64(seed & _MASK64) + k * np.uint64(0x9E3779B97F4A7C15)
        z = (z ^ (z >> np.uint64(30))) * np.uint64(0xBF58476D1CE4E5B9)
        z = (z ^ (z >> np.uint64(27))) * np.uint64(0x94D049BB133111EB)
        z = z ^ (z >> np.uint64(31))
    return (z >> np.uint64(11)).astype(np.float64) * (1.0 / (1 << 53))


def gaussian_random_field_voxels(seed: int, m: int = 128, corr_len: float = 0.05, solid_fraction: float = 0.25,
                                 octree_depth: int = 3) -> Geometry:
    """Trabecular-like voxel image on the unit cube (a synthetic stand-in for a bone micro-CT).

    White noise N(0,1) on m^3 voxels (Box-Muller on SplitMix64 uniforms), smoothed
    periodically with a Gaussian of standard deviation corr_len / sqrt(2) (so the
    field's covariance is exp(-d^2 / (2 corr_len^2))), thresholded so that the top
    `solid_fraction` of the values is solid, and restricted to the solid voxels that
    are 6-connected to the face z = 0 (floating islands would only carry the
    fictitious stiffness).  Array layout [z][y][x].
    """
    u = splitmix_uniforms(seed, m ** 3 + (m ** 3) % 2)
    u1, u2 = u[0::2], u[1::2]
    rad = np.sqrt(-2.0 * np.log(1.0 - u1))
    noise = np.concatenate([rad * np.cos(2 * np.pi * u2), rad * np.sin(2 * np.pi * u2)])[: m ** 3].reshape(m, m, m)
    sigma_vox = corr_len / np.sqrt(2.0) * m
    k = np.fft.fftfreq(m)
    g1 = np.exp(-2.0 * (np.pi * k * sigma_vox) ** 2)
    kern = g1[:, None, None] * g1[None, :, None] * g1[None, None, :]
    field = np.real(np.fft.ifftn(np.fft.fftn(noise) * kern))
    thr = np.quantile(field, 1.0 - solid_fraction)
    solid = field > thr
    # keep the solid voxels 6-connected to z = 0 (breadth-first flood fill)
    keep = np.zeros_like(solid)
    frontier = np.zeros_like(solid)
    frontier[0] = solid[0]
    keep |= frontier
    while frontier.any():
        nxt = np.zeros_like(solid)
        nxt[1:] |= frontier[:-1]
        nxt[:-1] |= frontier[1:]
        nxt[:, 1:] |= frontier[:, :-1]
        nxt[:, :-1] |= frontier[:, 1:]
        nxt[:, :, 1:] |= frontier[:, :, :-1]
        nxt[:, :, :-1] |= frontier[:, :, 1:]
        frontier = nxt & solid & ~keep
        keep |= frontier
    return Geometry(GEOM_VOXELS, voxels=keep.astype(np.uint8), octree_depth=octree_depth)


def random_vector(seed: int, n: int) -> np.ndarray:
    """n doubles uniform in [-1, 1) from SplitMix64, vectorised (same stream as `uniform`)."""
    # Vectorised SplitMix64: state_k = seed + k * gamma (mod 2^64), k = 1..n.
    k = np.arange(1, n + 1, dtype=np.uint64)
    with np.errstate(over="ignore"):
        z = np.uint64(seed & _MASK64) + k * np.uint64(0x9E3779B97F4A7C15)
        z = (z ^ (z >> np.uint64(30))) * np.uint64(0xBF58476D1CE4E5B9)
        z = (z ^ (z >> np.uint64(27))) * np.uint64(0x94D049BB133111EB)
        z = z ^ (z >> np.uint64(31))
    u = (z >> np.uint64(11)).astype(np.float64) * (1.0 / (1 << 53))
    return 2.0 * u - 1.0


@dataclasses.dataclass
class Workload:
    """One synthetic finite cell problem: grid, order, fictitious stiffness, geometry, solver tol."""
    name: str
    n: tuple
    p: int
    alpha: float
    geometry: Geometry
    tol: float
    E: float = 1.0
    nu: float = 0.3
    traction: tuple = (0.0, 0.0, -1.0)
    bc: int = 0           # 0: clamp every component on z = 0; 1: rollers on x=0, y=0, z=0
    lo: tuple = (0.0, 0.0, 0.0)
    hi: tuple = (1.0, 1.0, 1.0)

    @property
    def lattice_dofs(self) -> int:
        m = [self.p * k + 1 for k in self.n]
        return 3 * m[0] * m[1] * m[2]


def workload_single_void(seed: int = 0) -> Workload:
    """Unit cube minus one sphere r=0.3 (centre jittered), 4^3 cells, p=2, alpha=1e-8, depth 3, tol 1e-10."""
    return Workload("cube_1void_4x4x4_p2", (4, 4, 4), 2, 1e-8,
                    single_sphere_void(seed, 0.3, 0.05, octree_depth=3), 1e-10)


def workload_porous(seed: int = 11, n: int = 32, p: int = 3, count: int = 40,
                    alpha: float = 1e-10, depth: int = 4, tol: float = 1e-8) -> Workload:
    """Unit cube with `count` seeded spherical voids, radii U(0.02, 0.08)."""
    geo = random_sphere_voids(seed, count, 0.02, 0.08, octree_depth=depth)
    return Workload(f"porous{count}_{n}^3_p{p}", (n, n, n), p, alpha, geo, tol)


WORKLOADS = {
    # ~2k DOFs: one spherical void
    "single_void_4": lambda: workload_single_void(0),
    # ~2.7M DOFs: 40 voids, 32^3 cells, p=3
    "porous40_32_p3": lambda: workload_porous(11, 32, 3, 40, 1e-10, 4, 1e-8),
    # ~6.4M DOFs: 40 voids, 64^3 cells, p=2 (mixed precision family)
    "porous40_64_p2": lambda: workload_porous(12, 64, 2, 40, 1e-10, 3, 1e-8),
    # ~0.35M DOFs: the 32^3 family at 16^3 cells (profiling-sized: ~1.5 GB of block factors)
    "porous40_16_p3": lambda: workload_porous(11, 16, 3, 40, 1e-10, 4, 1e-8),
    # ~0.8M DOFs: 40 voids, 32^3 cells, p=2 (the size of the learned correction's training cubes;
    # profiling-sized for the coarse operator: 74 MB of K_H, ~1 GB of FP32 block factors)
    "porous40_32_p2": lambda: workload_porous(7, 32, 2, 40, 1e-10, 3, 1e-8),
    # ~12.4M DOFs: 300 voids, 80^3 cells, p=2 (the learned correction's evaluation cube)
    "porous300_80_p2": lambda: workload_porous(21, 80, 2, 300, 1e-10, 3, 1e-8),
    # trabecular-like voxel domain (Gaussian random field, volume fraction 0.25), 48^3 cells, p=3, 6 strain loads
    "trabecular_48_p3": lambda: workload_trabecular(13, 48, 3),
    # the same family at 24^3 cells (test-sized)
    "trabecular_24_p3": lambda: workload_trabecular(13, 24, 3),
}


def workload_trabecular(seed: int = 13, n: int = 48, p: int = 3, alpha: float = 1e-10, depth: int = 3,
                        tol: float = 1e-8) -> Workload:
    """Gaussian-random-field voxel domain (128^3 voxels, correlation length 0.05, solid fraction 0.25)."""
    geo = gaussian_random_field_voxels(seed, 128, 0.05, 0.25, octree_depth=depth)
    return Workload(f"trabecular_{n}^3_p{p}", (n, n, n), p, alpha, geo, tol)
