"""The oracle's derivative of the all-ray velocity along a direction (the stretching term), no GPU.

The paper gives no vorticity update; the library's stretching term
(omega . grad) v is the exact derivative of the all-ray rule, and the oracle
computes it from its definition (chord lengths times the tet's vorticity
gradient, plus the jump of omega to zero where a line leaves the mesh).  Pinned
here by central differences of the oracle's own velocity (a different
computation: three velocity evaluations, no derivative formula) at interior
points and interior nodes, and by the uniform ball's exact derivative
omega x e / 3, which converges with the mesh size.
"""
import numpy as np

import pins
from workloads import ball_mesh
from workloads.configs import jittered_grid


def test_matches_central_differences(orc):
    d = pins.dderiv(orc)
    assert d["points"] <= 1e-4, d
    assert d["nodes"] <= 2e-3, d


def test_uniform_ball_converges(orc):
    """RMS error (over 40 interior points, relative to the largest exact value) against omega x e / 3
    decreases as the ball mesh is refined (16 x 32 directions; the maximum is dominated by the
    angular quadrature and is not monotone point by point)."""
    rng = np.random.default_rng(8)
    w0 = np.array([0.3, -0.2, 1.0])
    pts = rng.uniform(-0.4, 0.4, (40, 3))
    e = rng.standard_normal((40, 3))
    ex = np.cross(w0, e) / 3.0
    errs = []
    for n in (7, 11, 15):
        m = ball_mesh(n)
        _, dv = orc.velocity_dderiv(m.nodes, m.tets, np.tile(w0, (len(m.nodes), 1)), pts, e, n_theta=16, n_phi=32)
        errs.append(np.sqrt(np.mean((dv - ex) ** 2)) / np.abs(ex).max())
    assert errs[0] > errs[1] > errs[2] and errs[2] <= 3e-3, errs


def test_velocity_output_is_the_all_ray_velocity(orc):
    rng = np.random.default_rng(9)
    nodes, tets = jittered_grid(5, 0.0, 1.0, rng)
    om = rng.standard_normal(nodes.shape)
    pts = rng.uniform(0.0, 1.0, (12, 3))
    v, _ = orc.velocity_dderiv(nodes, tets, om, pts, rng.standard_normal((12, 3)))
    assert np.array_equal(v, orc.velocity(nodes, tets, om, pts, far_ratio=np.inf))


def test_linear_in_the_direction(orc):
    rng = np.random.default_rng(10)
    nodes, tets = jittered_grid(5, 0.0, 1.0, rng)
    om = rng.standard_normal(nodes.shape)
    pts = rng.uniform(0.1, 0.9, (10, 3))
    e1, e2 = rng.standard_normal((10, 3)), rng.standard_normal((10, 3))
    _, d1 = orc.velocity_dderiv(nodes, tets, om, pts, e1)
    _, d2 = orc.velocity_dderiv(nodes, tets, om, pts, e2)
    _, d12 = orc.velocity_dderiv(nodes, tets, om, pts, e1 - 2.5 * e2)
    assert np.abs(d12 - (d1 - 2.5 * d2)).max() <= 1e-12 * np.abs(d12).max()
