"""The oracle's exact single-tet integral (near_rule 1: the analytic near-field evaluation that Section 1 sets
the ray rule against), pinned by results that do not come from it (no GPU)."""
import numpy as np
import pytest

import pins


@pytest.fixture(scope="module")
def res(orc):
    return pins.analytic(orc)


def test_single_tet_matches_the_duffy_cone_integral(res):
    """Inside, outside, on a vertex, an edge, a face, on an edge's line and far away."""
    for name, err in res["single"].items():
        assert err <= 5e-12, (name, err)


def test_additive_over_a_cut_tet(res):
    """The tet cut in two at a point of an edge, and into four cones from an interior point: the faces inside
    cancel, so the pieces sum to the whole (points at a vertex, inside, outside and on the cut)."""
    assert res["split"] <= 1e-12


def test_divergence_free(res):
    """v is the curl of the vector potential, so div v = 0 (central differences, step 1e-4)."""
    assert res["div"] <= 5e-6


def test_ray_rule_converges_onto_it(res):
    """The ray rule (N x N directions, N = 16..128) approaches the exact integral monotonically."""
    r = res["ray"]
    assert all(b < a for a, b in zip(r, r[1:]))
    assert r[-1] <= 2e-4


def test_uniform_ball_error_is_the_polyhedral_one(res):
    """Every tet exact: the error against omega x x / 3 comes from the faceted boundary alone, O(h^2)."""
    assert res["ball"][-1] <= 1e-4
    assert 1.7 <= res["ball_slope"] <= 2.5


def test_far_rule_and_exact_integral_agree_far_away(orc):
    """Far from the tet, the 64-point conical rule (degree 7) and the exact integral agree."""
    V, om = pins.single_tet_fixture()
    tets = np.array([[0, 1, 2, 3]], dtype=np.int32)
    x = np.array([6.0, -4.0, 5.0])
    g = orc.velocity(V, tets, om, x[None], far_ratio=0.0, tet_order=64)[0]
    a = orc.tet_analytic(x, V, om)
    assert np.linalg.norm(g - a) / np.linalg.norm(a) <= 1e-9


def test_near_rule_switch(orc):
    """near_rule 1 in orc.velocity sums tet_analytic over the near tets; far tets keep the Gauss rule; no ray
    hits are counted."""
    from workloads import config1_plain

    m = config1_plain()
    x = m.nodes[[40, 333]]
    v, c = orc.velocity(m.nodes, m.tets, m.omega, x, far_ratio=2.0, near_rule=1, counts=True)
    vf, cf = orc.velocity(m.nodes, m.tets, m.omega, x, far_ratio=2.0, counts=True)
    assert np.array_equal(c[:, :2], cf[:, :2]) and np.all(c[:, 2] == 0)
    assert np.linalg.norm(v - vf) / np.linalg.norm(vf) <= 1e-2  # the 8 x 16 ray rule's own error
    # every tet near: the sum of the single-tet integrals
    sub = m.tets[:50]
    va = orc.velocity(m.nodes, sub, m.omega, x, far_ratio=np.inf, near_rule=1)
    ref = np.array([sum(orc.tet_analytic(xx, m.nodes[t], m.omega[t]) for t in sub) for xx in x])
    assert np.abs(va - ref).max() <= 1e-14 * np.abs(ref).max()
    with pytest.raises(ValueError):
        orc.velocity(m.nodes, m.tets, m.omega, x, near_rule=2)
