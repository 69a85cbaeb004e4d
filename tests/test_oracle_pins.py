"""The oracle against results it does not compute itself (no GPU).

P1 single tet / star of a node vs the Duffy-cone integral, P2 uniform ball
closed form and its h-convergence, P5 Hill's spherical vortex, P4 divergence.
Bounds were set from the converged behaviour of the method (angular
quadrature error for the ray rule, degree of the tet rule for the far rule)
and are far tighter than the error any of the planted mistakes in
``test_oracle_mutants.py`` produces.
"""
import json
import os

import numpy as np
import pins

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")


def _monotone(seq, factor=1.0):
    return all(b < a * factor for a, b in zip(seq, seq[1:]))


def test_single_tet_ray_rule_converges(orc):
    r = pins.single_tet(orc, Ns=(32, 64, 128))
    # x strictly inside: the ray integrand is smooth in direction
    assert _monotone(r["inside"]["ray"], 1.0) and r["inside"]["ray"][-1] < 1e-4
    # x outside: kinks at the silhouette, second order in 1/N
    assert _monotone(r["outside"]["ray"]) and r["outside"]["ray"][-1] < 1.5e-3
    # x at a vertex: the integrand jumps at the three faces through x (first order)
    assert _monotone(r["vertex"]["ray"]) and r["vertex"]["ray"][-1] < 0.15


def test_single_tet_gauss_rule_converges(orc):
    r = pins.single_tet(orc, Ns=(8,))
    far = r["far"]["gauss"]  # orders 1, 4, 27, 64
    assert _monotone(far) and far[-1] < 1e-7 and far[1] < 5e-3
    assert _monotone(r["outside"]["gauss"]) and r["outside"]["gauss"][-1] < 1e-4


def test_star_of_node_converges(orc):
    errs = pins.star(orc, Ns=(16, 32, 64, 128))
    assert _monotone(errs) and errs[-1] < 5e-4


def test_uniform_ball_second_order(orc):
    with open(os.path.join(GOLDEN, "paper_convergence.json")) as f:
        paper = json.load(f)
    errs, slope = pins.ball(orc, ns=(5, 9, 17), N=64)
    assert _monotone(errs)
    assert errs[-1] < 1e-4
    lo, hi = paper["slope_accept"]
    assert lo <= slope <= hi, (errs, slope, paper["exponent"])


def test_uniform_ball_outside(orc):
    # outside, the error is the volume the inscribed polyhedron misses: O(h^2)
    e9 = pins.ball_outside(orc, n=9)
    e17 = pins.ball_outside(orc, n=17)
    assert e9 < 3e-2 and e17 < 7e-3 and e17 < e9 / 3


def test_hill_vortex_second_order(orc):
    errs = pins.hill(orc, ns=(5, 9, 17))
    assert _monotone(errs, 0.4)  # each halving of h cuts the error by more than 2.5x
    assert errs[-1] < 5e-3


def test_divergence_small_and_decreasing(orc):
    d16 = pins.divergence(orc, N=16)
    d64 = pins.divergence(orc, N=64)
    assert d64 < 0.05 and d64 < d16


def test_heun_step_against_rigid_rotation(orc):
    """Uniform omega in a ball turns it rigidly: v = A x, A = [omega]x / 3.  Heun's method on v = A x
    gives exactly x1 = (I + dt A + dt^2 A^2 / 2) x0; the oracle's step must match it within the
    discretisation error (about 1% on the boundary nodes that the first stage moves, which the second
    stage feels inside), and at least four times better than a one-stage (Euler) step (15% here)."""
    import oracle as orc_mod

    from workloads import ball_mesh

    w = np.array([0.0, 0.0, 3.0])  # A = rotation about z at unit rate
    b = ball_mesh(9, lambda X: np.tile(w, (len(X), 1)))
    A = np.array([[0.0, -w[2], w[1]], [w[2], 0.0, -w[0]], [-w[1], w[0], 0.0]]) / 3.0
    dt = 0.3
    x1 = orc_mod.heun_step(orc, b.nodes, b.tets, b.omega, dt, far_ratio=np.inf, tet_order=4, n_theta=32, n_phi=32)
    inner = np.linalg.norm(b.nodes, axis=1) < 0.5
    x0 = b.nodes[inner]
    exact = x0 + dt * x0 @ A.T + 0.5 * dt**2 * x0 @ (A @ A).T
    euler = x0 + dt * x0 @ A.T
    err = np.linalg.norm(x1[inner] - exact) / np.linalg.norm(exact - x0)
    err_euler = np.linalg.norm(euler - exact) / np.linalg.norm(exact - x0)
    assert err < 3e-2 and err < err_euler / 4


def test_near_far_counts_against_numpy_classification(orc):
    """Near count = tets with |x - centroid| <= far_ratio * circumradius, the circumcentre found by
    numpy's linear solve (not the oracle's Cramer rule)."""
    from workloads import config1_plain

    m = config1_plain()
    V = m.nodes[m.tets]  # [t, 4, 3]
    c = V.mean(axis=1)
    A = 2.0 * (V[:, 1:] - V[:, :1])
    rhs = np.sum(V[:, 1:] ** 2, axis=2) - np.sum(V[:, :1] ** 2, axis=2)
    p = np.linalg.solve(A, rhs[..., None])[..., 0]
    rho = np.linalg.norm(p - V[:, 0], axis=1)
    pts = m.nodes[::9]
    _, cnt = orc.velocity(m.nodes, m.tets, m.omega, pts, far_ratio=2.0, counts=True)
    d = np.linalg.norm(pts[:, None, :] - c[None, :, :], axis=2)
    near = (d <= 2.0 * rho[None, :]).sum(axis=1)
    assert np.array_equal(cnt[:, 0], near)
    assert np.array_equal(cnt[:, 1], len(m.tets) - near)
