"""Kuhn-split structured tetrahedral meshes.

A grid of ``n`` nodes per side is cut into (n-1)^3 cubes and every cube into
the six Kuhn tetrahedra that share its main diagonal.  Node index
``i + n*(j + n*k)`` sits at (x_i, y_j, z_k).  These meshes stand in for the
TETGEN meshes of random control points used in the paper (Section 3): the
paper's point sets are not published, the method itself only needs a
conforming tetrahedralisation with nodal vorticity.
"""
from __future__ import annotations

import itertools

import numpy as np


def kuhn_grid(n: int, lo: float, hi: float):
    """Nodes [n^3, 3] (float64) and tets [6(n-1)^3, 4] (int32) of a Kuhn grid on [lo, hi]^3."""
    if n < 2:
        raise ValueError("need at least 2 nodes per side")
    g = np.linspace(lo, hi, n, dtype=np.float64)
    # x fastest
    zz, yy, xx = np.meshgrid(g, g, g, indexing="ij")
    nodes = np.stack([xx.ravel(), yy.ravel(), zz.ravel()], axis=1)

    c = np.arange(n - 1)
    ck, cj, ci = np.meshgrid(c, c, c, indexing="ij")
    ci, cj, ck = ci.ravel(), cj.ravel(), ck.ravel()

    def nid(di, dj, dk):
        return (ci + di) + n * ((cj + dj) + n * (ck + dk))

    unit = np.eye(3, dtype=np.int64)
    tets = []
    for perm in itertools.permutations(range(3)):
        p = np.zeros(3, dtype=np.int64)
        verts = [nid(*p)]
        for ax in perm:
            p = p + unit[ax]
            verts.append(nid(*p))
        tets.append(np.stack(verts, axis=1))
    # interleave so the six tets of a cube are adjacent in memory
    tets = np.stack(tets, axis=1).reshape(-1, 4).astype(np.int32)
    return nodes, orient_positive(nodes, tets)


def tet_volumes6(nodes: np.ndarray, tets: np.ndarray) -> np.ndarray:
    """Six times the signed volume of every tet."""
    v = nodes[tets]
    e1, e2, e3 = v[:, 1] - v[:, 0], v[:, 2] - v[:, 0], v[:, 3] - v[:, 0]
    return np.einsum("ij,ij->i", e1, np.cross(e2, e3))


def orient_positive(nodes: np.ndarray, tets: np.ndarray) -> np.ndarray:
    """Swap the last two vertices of every negatively oriented tet."""
    tets = np.array(tets, dtype=np.int32, copy=True)
    neg = tet_volumes6(nodes, tets) < 0
    tets[neg, 2], tets[neg, 3] = tets[neg, 3].copy(), tets[neg, 2].copy()
    return tets


def boundary_mask(n: int) -> np.ndarray:
    """True for nodes on the boundary of the n^3 grid."""
    i = np.arange(n)
    on = (i == 0) | (i == n - 1)
    ok, oj, oi = np.meshgrid(on, on, on, indexing="ij")
    return (oi | oj | ok).ravel()


def jitter_interior(nodes: np.ndarray, n: int, frac: float, rng: np.random.Generator) -> np.ndarray:
    """Move every interior node by U(-frac*h, +frac*h) per coordinate; boundary nodes stay put."""
    lo, hi = nodes[:, 0].min(), nodes[:, 0].max()
    h = (hi - lo) / (n - 1)
    out = nodes.copy()
    interior = ~boundary_mask(n)
    out[interior] += rng.uniform(-frac * h, frac * h, size=(int(interior.sum()), 3))
    return out


def cube_to_ball(nodes: np.ndarray) -> np.ndarray:
    """Map the cube [-1,1]^3 onto the unit ball by y = x * |x|_inf / |x|_2."""
    linf = np.abs(nodes).max(axis=1)
    l2 = np.linalg.norm(nodes, axis=1)
    scale = np.where(l2 > 0, linf / np.where(l2 > 0, l2, 1.0), 0.0)
    return nodes * scale[:, None]
