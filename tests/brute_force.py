"""Ray-free reference integrals used to pin the oracle.

``tet_integral`` evaluates Eq. 1 over one tetrahedron with linear nodal
vorticity without any angular quadrature: the tet is split into four signed
cones with apex x (one per face), and each cone is integrated in collapsed
(Duffy) coordinates y = x + s (P(u, v) - x), P(u, v) = a + u (b - a) + u v (c - b),
dV = s^2 u D ds du dv with D = (a - x) . ((b - a) x (c - a)).  The s^2 cancels
the 1/R^2 singularity, the s integral of the linear vorticity is its value at
the midpoint, and (u, v) are integrated with a tensor Gauss-Legendre rule from
numpy (an independent library routine).
"""
from __future__ import annotations

import numpy as np

FACES = ((1, 2, 3), (0, 2, 3), (0, 1, 3), (0, 1, 2))


def barycentric(verts: np.ndarray, y: np.ndarray) -> np.ndarray:
    """Barycentric coordinates of points y [..., 3] in the tet verts [4, 3] (np.linalg.solve)."""
    A = np.vstack([verts.T, np.ones(4)])  # 4x4
    rhs = np.concatenate([y.reshape(-1, 3).T, np.ones((1, y.reshape(-1, 3).shape[0]))], axis=0)
    lam = np.linalg.solve(A, rhs).T
    return lam.reshape(y.shape[:-1] + (4,))


def _gl01(n: int):
    t, w = np.polynomial.legendre.leggauss(n)
    return 0.5 * (t + 1.0), 0.5 * w


def tet_integral(x, verts, om, n: int = 48) -> np.ndarray:
    """-(1/4pi) int_T (x - y) x omega(y) / |x - y|^3 dV(y) for linear nodal omega [4, 3]."""
    x = np.asarray(x, dtype=np.float64)
    verts = np.asarray(verts, dtype=np.float64)
    om = np.asarray(om, dtype=np.float64)
    h = max(np.linalg.norm(verts[i] - verts[j]) for i in range(4) for j in range(i + 1, 4))
    u, wu = _gl01(n)
    U, V = np.meshgrid(u, u, indexing="ij")
    W = np.outer(wu, wu)
    total = np.zeros(3)
    for f, opp in zip(FACES, range(4)):
        a, b, c = (verts[i] for i in f)
        nrm = np.cross(b - a, c - a)
        if np.dot(nrm, a - verts[opp]) < 0:  # orient the face outwards
            b, c = c, b
            nrm = -nrm
        D = np.dot(a - x, nrm)
        if abs(D) <= 1e-12 * h**3:
            continue  # x lies in this face's plane: the cone has no volume
        P = a[None, None, :] + U[..., None] * (b - a) + (U * V)[..., None] * (c - b)
        d = P - x[None, None, :]
        R = np.linalg.norm(d, axis=-1)
        mid = 0.5 * (P + x[None, None, :])
        lam = barycentric(verts, mid)
        w = lam @ om
        integrand = np.cross(d, w) / R[..., None] ** 3 * (U * D)[..., None]
        total += np.einsum("ij,ijk->k", W, integrand)
    return total / (4.0 * np.pi)


def chord_by_sampling(x, s, verts, span: float, n: int = 20001):
    """Chord [R0, R1] of the line x + R s through the tet, by dense sampling then bisection.

    Membership of a point is decided by its barycentric coordinates from
    ``barycentric`` (a linear solve), not by any face test.  Returns None when
    no sample lies inside.
    """
    x = np.asarray(x, dtype=np.float64)
    s = np.asarray(s, dtype=np.float64)
    R = np.linspace(-span, span, n)
    lam = barycentric(verts, x[None, :] + R[:, None] * s[None, :])
    inside = np.all(lam >= 0.0, axis=1)
    if not inside.any():
        return None
    idx = np.nonzero(inside)[0]
    i0, i1 = idx[0], idx[-1]

    def is_in(r):
        return bool(np.all(barycentric(verts, (x + r * s)[None, :]) >= 0.0))

    def bisect(lo_out, hi_in):
        for _ in range(200):
            mid = 0.5 * (lo_out + hi_in)
            if mid == lo_out or mid == hi_in:
                break
            if is_in(mid):
                hi_in = mid
            else:
                lo_out = mid
        return hi_in

    R0 = bisect(R[i0 - 1], R[i0]) if i0 > 0 else R[0]
    R1 = bisect(R[i1 + 1], R[i1]) if i1 + 1 < n else R[-1]
    return R0, R1


def signed_chord_integral(x, s, verts, om, R0, R1, n: int = 8) -> np.ndarray:
    """int_{R0}^{R1} sign(R) omega(x + R s) dR by Gauss-Legendre on each side of R = 0."""
    x = np.asarray(x, dtype=np.float64)
    s = np.asarray(s, dtype=np.float64)
    pieces = [(R0, R1)] if (R0 >= 0 or R1 <= 0) else [(R0, 0.0), (0.0, R1)]
    t, w = np.polynomial.legendre.leggauss(n)
    J = np.zeros(3)
    for a, b in pieces:
        r = 0.5 * (a + b) + 0.5 * (b - a) * t
        lam = barycentric(verts, x[None, :] + r[:, None] * s[None, :])
        vals = lam @ om
        sign = 1.0 if (a + b) > 0 else -1.0
        J += sign * 0.5 * (b - a) * (w @ vals)
    return J
