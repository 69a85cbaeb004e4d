"""Pin measurements of the oracle against results that do not come from it.

Each function runs one family of checks on an oracle object (the shipped
``oracle`` module, or a compiled copy of ``bs_oracle.c`` with a planted
mistake) and returns the numbers the tests compare with their bounds.

  single_tet   Eq. 1 on one tet / the star of a node, exact values from the
               ray-free Duffy-cone integrator in ``brute_force.py``.
  ball         uniform omega in a tetrahedralised unit ball: closed form
               omega x (x - c)/3 inside, a^3 omega x (x - c) / (3|x - c|^3)
               outside; convergence in h at 64 x 64 directions (Section 3.2
               reports eps ~ h^2.15 for its ring).
  hill         Hill's spherical vortex (Section 3.1), with the velocity
               re-derived from the Stokes stream function (the printed
               formula is garbled, see ``hill_velocity``).
  dderiv       derivative of the all-ray velocity along a direction (the
               stretching term): central differences of the oracle's own
               velocity at interior points and nodes, and the uniform ball's
               exact derivative omega x e / 3.
  analytic     the exact single-tet integral (the analytic near-field
               evaluation of Section 1): the Duffy-cone integral at points
               inside, outside, on a vertex, an edge, a face and an edge's
               line; additivity when a tet is cut into sub-tets (the faces
               inside cancel); zero divergence by central differences; the ray
               rule converging onto it as the angular order grows; and the
               uniform ball, where only the polyhedral error O(h^2) is left.
"""
from __future__ import annotations

import numpy as np
from brute_force import tet_integral

from workloads import ball_mesh, hill_velocity, hill_vorticity
from workloads.configs import jittered_grid


def _rel(a, b):
    return float(np.linalg.norm(np.asarray(a) - np.asarray(b)) / np.linalg.norm(b))


def single_tet_fixture():
    rng = np.random.default_rng(5)
    V = np.array([[0, 0, 0], [1, 0.1, 0], [0.2, 1, 0.1], [0.1, 0.2, 1.0]])
    om = rng.standard_normal((4, 3))
    return V, om


def single_tet(orc, Ns=(32, 64, 128), qs=(1, 4, 27, 64)):
    V, om = single_tet_fixture()
    tets = np.array([[0, 1, 2, 3]], dtype=np.int32)
    points = {
        "inside": V.mean(axis=0) + 0.05,
        "outside": np.array([1.2, 0.9, 0.8]),
        "vertex": V[2].copy(),
        "far": np.array([3.0, 2.0, 1.0]),
    }
    out = {}
    for name, x in points.items():
        exact = tet_integral(x, V, om, 48)
        out[name] = {
            "ray": [_rel(orc.velocity(V, tets, om, x[None], far_ratio=np.inf, n_theta=N, n_phi=N)[0], exact)
                    for N in Ns],
            "gauss": [_rel(orc.velocity(V, tets, om, x[None], far_ratio=0.0, tet_order=q)[0], exact) for q in qs],
        }
    return out


def star_fixture():
    rng = np.random.default_rng(11)
    nodes, tets = jittered_grid(4, 0.0, 1.0, rng)
    om = rng.standard_normal(nodes.shape)
    c = 1 + 4 * (1 + 4 * 1)  # interior node (1, 1, 1)
    star = tets[np.any(tets == c, axis=1)]
    return nodes, star, om, c


def star(orc, Ns=(16, 32, 64, 128)):
    """Pure-ray velocity at an interior node from the 24 tets around it, against the Duffy sum."""
    nodes, st, om, c = star_fixture()
    x = nodes[c]
    exact = sum(tet_integral(x, nodes[t], om[t], 48) for t in st)
    return [_rel(orc.velocity(nodes, st, om, x[None], far_ratio=np.inf, n_theta=N, n_phi=N)[0], exact)
            for N in Ns]


BALL_OMEGA = np.array([0.3, -0.5, 0.8])


def _ball_points(mesh, count, rmax, seed=0):
    r = np.linalg.norm(mesh.nodes, axis=1)
    idx = np.nonzero(r < rmax)[0]
    rng = np.random.default_rng(seed)
    return mesh.nodes[rng.choice(idx, size=min(count, len(idx)), replace=False)]


def ball(orc, ns=(5, 9, 17), N=64, count=8):
    """RMS error / |omega|_max at interior nodes for the pure-ray rule, and the fitted slope in h."""
    errs = []
    hs = []
    for n in ns:
        b = ball_mesh(n, lambda X: np.tile(BALL_OMEGA, (len(X), 1)))
        X = _ball_points(b, count, 0.55)
        v = orc.velocity(b.nodes, b.tets, b.omega, X, far_ratio=np.inf, n_theta=N, n_phi=N)
        exact = np.cross(BALL_OMEGA, X) / 3.0
        errs.append(float(np.sqrt(np.mean(np.sum((v - exact) ** 2, axis=1))) / np.abs(BALL_OMEGA).max()))
        hs.append(2.0 / (n - 1))
    slope = float(np.polyfit(np.log(hs), np.log(errs), 1)[0])
    return errs, slope


def ball_outside(orc, n=9, params=None):
    params = params or dict(far_ratio=2.0, tet_order=4, n_theta=16, n_phi=16)
    b = ball_mesh(n, lambda X: np.tile(BALL_OMEGA, (len(X), 1)))
    X = np.array([[0.0, 0.0, 1.5], [1.3, 0.4, -0.2], [-0.9, -1.1, 0.7], [2.5, -1.0, 0.5]])
    v = orc.velocity(b.nodes, b.tets, b.omega, X, **params)
    R = np.linalg.norm(X, axis=1)
    exact = np.cross(BALL_OMEGA, X) / (3.0 * R[:, None] ** 3)
    return float(np.abs(v - exact).max() / np.abs(exact).max())


def hill(orc, ns=(5, 9, 17), params=None, count=12):
    params = params or dict(far_ratio=2.0, tet_order=4, n_theta=16, n_phi=16)
    errs = []
    for n in ns:
        b = ball_mesh(n, hill_vorticity)
        X = _ball_points(b, count, 0.6)
        v = orc.velocity(b.nodes, b.tets, b.omega, X, **params)
        ex = hill_velocity(X)
        errs.append(float(np.sqrt(np.mean(np.sum((v - ex) ** 2, axis=1))) / np.abs(ex).max()))
    return errs


def divergence(orc, N=64, far_ratio=np.inf, count=4, seed=3):
    """max |div v| / max |grad v| by central differences at off-node points of the unit-cube mesh."""
    from workloads import config1_plain

    m = config1_plain()
    rng = np.random.default_rng(seed)
    X = rng.uniform(0.3, 0.7, size=(count, 3))
    d = 1e-3 / 8
    pts = []
    for x in X:
        for j in range(3):
            e = np.zeros(3)
            e[j] = d
            pts += [x + e, x - e]
    v = orc.velocity(m.nodes, m.tets, m.omega, np.array(pts), far_ratio=far_ratio, n_theta=N, n_phi=N)
    v = v.reshape(count, 3, 2, 3)
    grad = (v[:, :, 0, :] - v[:, :, 1, :]) / (2 * d)  # [pt, j (d/dx_j), component]
    div = np.einsum("pjj->p", grad)
    return float(np.abs(div).max() / np.abs(grad).max())


def dderiv(orc, n=5, count=20, ball_n=7):
    """Largest errors (relative to the largest derivative) of orc.velocity_dderiv against central differences
    of orc.velocity (all-ray, 8 x 16 directions) at interior off-node points (step 1e-5) and interior nodes
    (step 1e-6), and against the uniform ball's exact derivative omega x e / 3 inside (16 x 32 directions)."""
    rng = np.random.default_rng(23)
    nodes, tets = jittered_grid(n, 0.0, 1.0, rng)
    om = np.array([0.0, 0.0, 1.0]) + 0.3 * rng.standard_normal(nodes.shape)
    P = dict(n_theta=8, n_phi=16)
    inner = np.all((nodes > 1e-9) & (nodes < 1 - 1e-9), axis=1)
    out = {}
    for name, pts, d in (("points", rng.uniform(0.15, 0.85, (count, 3)), 1e-5),
                         ("nodes", nodes[inner][:count], 1e-6)):
        e = rng.standard_normal(pts.shape)
        _, dv = orc.velocity_dderiv(nodes, tets, om, pts, e, **P)
        vp = orc.velocity(nodes, tets, om, pts + d * e, far_ratio=np.inf, **P)
        vm = orc.velocity(nodes, tets, om, pts - d * e, far_ratio=np.inf, **P)
        out[name] = float(np.abs((vp - vm) / (2 * d) - dv).max() / np.abs(dv).max())
    m = ball_mesh(ball_n)
    w0 = np.array([0.3, -0.2, 1.0])
    pts = rng.uniform(-0.4, 0.4, (count, 3))
    e = rng.standard_normal((count, 3))
    _, dv = orc.velocity_dderiv(m.nodes, m.tets, np.tile(w0, (len(m.nodes), 1)), pts, e, n_theta=16, n_phi=32)
    ex = np.cross(w0, e) / 3.0
    out["ball"] = float(np.abs(dv - ex).max() / np.abs(ex).max())
    return out


def analytic(orc, quick=False):
    """Measurements of orc.tet_analytic / near_rule 1 against results that do not come from it."""
    V, om = single_tet_fixture()
    out = {}
    pts = {"inside": V.mean(axis=0) + 0.05, "outside": np.array([1.2, 0.9, 0.8]), "vertex": V[2].copy(),
           "edge": 0.5 * (V[0] + V[1]), "face": (V[1] + V[2] + V[3]) / 3, "edge line": V[0] + 1.7 * (V[1] - V[0]),
           "far": np.array([3.0, 2.0, 1.0])}
    if quick:
        pts = {k: pts[k] for k in ("inside", "outside", "vertex")}
    out["single"] = {k: _rel(orc.tet_analytic(x, V, om), tet_integral(x, V, om, 96)) for k, x in pts.items()}
    # cut the tet at a point q of edge 0-1 and at an interior point c: omega interpolates linearly
    lam = np.array([0.3, 0.7, 0.0, 0.0])
    q, wq = lam @ V, lam @ om
    c, wc = np.array([0.1, 0.2, 0.3, 0.4]) @ V, np.array([0.1, 0.2, 0.3, 0.4]) @ om
    parts = [(np.array([V[0], q, V[2], V[3]]), np.array([om[0], wq, om[2], om[3]])),
             (np.array([q, V[1], V[2], V[3]]), np.array([wq, om[1], om[2], om[3]]))]
    cones = []
    for f in ((1, 2, 3), (0, 2, 3), (0, 1, 3), (0, 1, 2)):
        cones.append((np.array([c, *V[list(f)]]), np.array([wc, *om[list(f)]])))
    split = 0.0
    for x in (V[0], V.mean(axis=0) + 0.03, np.array([0.9, -0.4, 0.6]), q):
        full = orc.tet_analytic(x, V, om)
        for pieces in (parts, cones):
            split = max(split, _rel(sum(orc.tet_analytic(x, a, b) for a, b in pieces), full))
    out["split"] = split
    # divergence of the exact integral vanishes (central differences, step 1e-4)
    rng = np.random.default_rng(41)
    worst = 0.0
    d = 1e-4
    for x in (V.mean(axis=0) + 0.02, np.array([1.1, 0.8, 0.6]), 0.5 * (V[1] + V[2]) + 0.01):
        grad = np.zeros((3, 3))
        for j in range(3):
            e = np.zeros(3)
            e[j] = d
            grad[j] = (orc.tet_analytic(x + e, V, om) - orc.tet_analytic(x - e, V, om)) / (2 * d)
        worst = max(worst, abs(np.trace(grad)) / np.abs(grad).max())
    out["div"] = worst
    # the ray rule converges onto the exact integral as the angular order grows
    tets = np.array([[0, 1, 2, 3]], dtype=np.int32)
    x = V.mean(axis=0) + 0.05
    ex = orc.tet_analytic(x, V, om)
    Ns = (16, 64) if quick else (16, 32, 64, 128)
    out["ray"] = [_rel(orc.velocity(V, tets, om, x[None], far_ratio=np.inf, n_theta=N, n_phi=N)[0], ex)
                  for N in Ns]
    if not quick:
        # uniform ball, every tet exact: the error left is the polyhedral one, O(h^2)
        errs, hs = [], []
        for n in (5, 9, 17):
            b = ball_mesh(n, lambda X: np.tile(BALL_OMEGA, (len(X), 1)))
            X = _ball_points(b, 8, 0.55)
            v = orc.velocity(b.nodes, b.tets, b.omega, X, far_ratio=np.inf, near_rule=1)
            exact = np.cross(BALL_OMEGA, X) / 3.0
            errs.append(float(np.sqrt(np.mean(np.sum((v - exact) ** 2, axis=1))) / np.abs(BALL_OMEGA).max()))
            hs.append(2.0 / (n - 1))
        out["ball"] = errs
        out["ball_slope"] = float(np.polyfit(np.log(hs), np.log(errs), 1)[0])
    return out
