"""The five synthetic workloads, seeded, plus the tetrahedralised ball.

Seeds are 1000 + workload number; the 4096 sample nodes of the 64^3 workload
use seed 2003.  Every interior node is jittered by U(+-0.1 h) per coordinate.
"""
from __future__ import annotations

from dataclasses import dataclass, field

import numpy as np

from .fields import constant_plus_noise, fourier_curl_field, gaussian_blob, gaussian_ring, two_rings
from .mesh import cube_to_ball, jitter_interior, kuhn_grid, orient_positive, tet_volumes6

JITTER = 0.1


@dataclass
class Mesh:
    name: str
    nodes: np.ndarray  # [n, 3] float64
    tets: np.ndarray  # [m, 4] int32
    omega: np.ndarray  # [n, 3] float64
    n_side: int = 0
    meta: dict = field(default_factory=dict)

    @property
    def n_nodes(self) -> int:
        return int(self.nodes.shape[0])

    @property
    def n_tets(self) -> int:
        return int(self.tets.shape[0])


def jittered_grid(n: int, lo: float, hi: float, rng: np.random.Generator, frac: float = JITTER):
    nodes, tets = kuhn_grid(n, lo, hi)
    nodes = jitter_interior(nodes, n, frac, rng)
    tets = orient_positive(nodes, tets)
    assert np.all(tet_volumes6(nodes, tets) > 0)
    return nodes, tets


def config1_plain(n: int = 9) -> Mesh:
    """Unit cube, 8 cells per side (729 nodes, 3072 tets); omega = (0,0,1) + 0.1 N(0,1)."""
    rng = np.random.default_rng(1001)
    nodes, tets = jittered_grid(n, 0.0, 1.0, rng)
    omega = constant_plus_noise(len(nodes), rng)
    return Mesh("plain-cube-9^3", nodes, tets, omega, n)


def config2_ring(n: int = 32) -> Mesh:
    """Gaussian ring (radius 1, sigma 0.2, circulation 1) on a 32^3 grid of [-1.5, 1.5]^3."""
    rng = np.random.default_rng(1002)
    nodes, tets = jittered_grid(n, -1.5, 1.5, rng)
    omega = gaussian_ring(nodes, 1.0, 0.2, 1.0)
    return Mesh(f"gaussian-ring-{n}^3", nodes, tets, omega, n)


def config3_fourier(n: int = 64) -> Mesh:
    """Divergence-free 8-mode Fourier field on a 64^3 grid of [-1, 1]^3."""
    rng = np.random.default_rng(1003)
    nodes, tets = jittered_grid(n, -1.0, 1.0, rng)
    omega = fourier_curl_field(nodes, rng)
    return Mesh(f"fourier-{n}^3", nodes, tets, omega, n)


def config3_samples(n_nodes: int, count: int = 4096) -> np.ndarray:
    """Seeded sample of node indices (without replacement), sorted ascending."""
    rng = np.random.default_rng(2003)
    return np.sort(rng.choice(n_nodes, size=min(count, n_nodes), replace=False)).astype(np.int64)


def config4_batch(count: int = 256, nmin: int = 8, nmax: int = 24) -> list[Mesh]:
    """``count`` independent meshes n^3 (n ~ U{nmin..nmax}) on [-1,1]^3, each with a Gaussian blob."""
    rng = np.random.default_rng(1004)
    out = []
    for i in range(count):
        n = int(rng.integers(nmin, nmax + 1))
        nodes, tets = jittered_grid(n, -1.0, 1.0, rng)
        c = rng.uniform(-0.5, 0.5, size=3)
        sigma = float(rng.uniform(0.1, 0.3))
        axis = rng.standard_normal(3)
        axis /= np.linalg.norm(axis)
        omega = gaussian_blob(nodes, c, sigma, axis)
        out.append(Mesh(f"blob-{i}-{n}^3", nodes, tets, omega, n, {"center": c, "sigma": sigma, "axis": axis}))
    return out


def config5_rings(n: int = 80) -> Mesh:
    """Two coaxial colliding rings (radius 1, sigma 0.15, separation 1.5) on an n^3 grid of [-1.5,1.5]^3."""
    rng = np.random.default_rng(1005)
    nodes, tets = jittered_grid(n, -1.5, 1.5, rng)
    omega = two_rings(nodes, 1.0, 0.15, 1.5)
    return Mesh(f"two-rings-{n}^3", nodes, tets, omega, n)


def ball_mesh(n: int, omega_fn=None, seed: int = 77, jitter: float = 0.0) -> Mesh:
    """Kuhn grid of [-1,1]^3 (n nodes/side) mapped onto the unit ball by y = x |x|_inf / |x|_2.

    Interior nodes are jittered by U(+-jitter h) per coordinate in the cube.  The ball map is not smooth at
    the origin and would turn some jittered tets inside out (a folded mesh) or into slivers; the jitter of the
    nodes of a tet is halved until it keeps at least a quarter of its volume in the unjittered ball mesh.
    """
    rng = np.random.default_rng(seed)
    base, tets = kuhn_grid(n, -1.0, 1.0)
    tets = orient_positive(base, tets)
    disp = jitter_interior(base, n, jitter, rng) - base if jitter > 0 else np.zeros_like(base)
    vol_min = 0.25 * tet_volumes6(cube_to_ball(base), tets)
    for _ in range(40):
        nodes = cube_to_ball(base + disp)
        bad = tet_volumes6(nodes, tets) < vol_min
        if not bad.any():
            break
        disp[np.unique(tets[bad])] *= 0.5
    vol6 = tet_volumes6(nodes, tets)
    assert np.all(vol6 > 0), "ball map produced a degenerate tet"
    omega = omega_fn(nodes) if omega_fn is not None else np.zeros_like(nodes)
    return Mesh(f"ball-{n}^3", nodes, tets, omega, n)
