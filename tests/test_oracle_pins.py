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
