"""Pins of the oracle's per-line step (Section 2.1, Eq. 5) against a face-test-free chord finder.

For random tets and lines, the chord [R0, R1] found by the oracle's
Moller-Trumbore face tests must match the one found by dense sampling plus
bisection on barycentric coordinates (a linear solve), and the chord integral
with the sign of R kept must match Gauss-Legendre quadrature of
sign(R) omega(x + R s) along it.  The pre-check may reject only lines that
miss the tet.
"""
import numpy as np
import pytest
from brute_force import chord_by_sampling, signed_chord_integral


def _random_tet(rng):
    while True:
        v = rng.uniform(-1, 1, size=(4, 3))
        vol6 = np.linalg.det(np.stack([v[1] - v[0], v[2] - v[0], v[3] - v[0]]))
        if abs(vol6) > 0.3:
            return v


def _unit(rng):
    s = rng.standard_normal(3)
    return s / np.linalg.norm(s)


@pytest.mark.parametrize("seed", range(6))
def test_chord_matches_sampling(orc, seed):
    rng = np.random.default_rng(100 + seed)
    checked = 0
    while checked < 8:
        v = _random_tet(rng)
        om = rng.standard_normal((4, 3))
        # aim the line near the tet so that about half the lines hit
        x = v.mean(axis=0) + rng.uniform(-1.5, 1.5, size=3)
        target = v.mean(axis=0) + 0.3 * rng.standard_normal(3)
        s = target - x
        s /= np.linalg.norm(s)
        hit, R0, R1, J = orc.line_tet(x, s, v, om)
        ref = chord_by_sampling(x, s, v, span=6.0)
        if ref is None:
            assert not hit
            continue
        r0, r1 = ref
        if r1 - r0 < 1e-6:
            continue  # grazing line: not a pin
        assert hit
        assert abs(R0 - r0) < 1e-12 and abs(R1 - r1) < 1e-12
        Jref = signed_chord_integral(x, s, v, om, R0, R1)
        assert np.allclose(J, Jref, atol=1e-13, rtol=0)
        checked += 1


def test_chord_through_evaluation_point(orc):
    """x inside the tet: the chord straddles R = 0 and the two halves enter with opposite signs."""
    rng = np.random.default_rng(7)
    v = _random_tet(rng)
    om = rng.standard_normal((4, 3))
    x = v.mean(axis=0)
    for _ in range(10):
        s = _unit(rng)
        hit, R0, R1, J = orc.line_tet(x, s, v, om)
        assert hit and R0 < 0 < R1
        Jref = signed_chord_integral(x, s, v, om, R0, R1)
        assert np.allclose(J, Jref, atol=1e-13)
    # uniform omega: J = (R1 + R0) omega (the sign of R weights the two halves)
    omu = np.tile([0.3, -0.2, 0.9], (4, 1))
    s = _unit(rng)
    hit, R0, R1, J = orc.line_tet(x, s, v, omu)
    assert np.allclose(J, (R1 + R0) * omu[0], atol=1e-14)


def test_chord_from_vertex(orc):
    """x at a vertex: one end of every chord is R = 0 exactly, omega there is the nodal value."""
    rng = np.random.default_rng(8)
    v = _random_tet(rng)
    om = rng.standard_normal((4, 3))
    hits = 0
    for _ in range(400):
        s = _unit(rng)
        hit, R0, R1, J = orc.line_tet(v[2], s, v, om)
        if not hit:
            continue
        hits += 1
        assert R0 == 0.0 or R1 == 0.0
        Jref = signed_chord_integral(v[2], s, v, om, R0, R1)
        assert np.allclose(J, Jref, atol=1e-13)
    assert hits > 20


def test_precheck_only_rejects_misses(orc):
    rng = np.random.default_rng(9)
    n_rejected = 0
    for _ in range(3000):
        v = _random_tet(rng) * 0.2
        om = rng.standard_normal((4, 3))
        x = rng.uniform(-1.5, 1.5, size=3)
        s = _unit(rng)
        a = orc.line_tet(x, s, v, om, use_precheck=False)
        b = orc.line_tet(x, s, v, om, use_precheck=True)
        assert a[0] == b[0]
        if a[0]:
            assert a[1:3] == b[1:3] and np.array_equal(a[3], b[3])
        # count the rejections that the pre-check makes on its own
        r = v[0] - x
        if np.dot(r, s) ** 2 < np.dot(r, r) - 2 * max(
                np.sum((v[i] - v[j]) ** 2) for i in range(4) for j in range(i + 1, 4)):
            n_rejected += 1
            assert not a[0]
    assert n_rejected > 1000
