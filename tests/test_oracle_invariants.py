"""Exact properties of the discrete rule (no GPU).

P3: linearity in omega, invariance to tet order, to vertex order inside a tet
and to translation, covariance under the rotation by pi about z (which maps
the direction set of Eq. 3 onto itself).  P6: the pre-check of Section 2.1
never changes a result.  Counts: near + far = number of tets.
"""
import numpy as np
import pytest

from workloads import config1_plain

PARAMS = dict(far_ratio=2.0, tet_order=4, n_theta=8, n_phi=16)


@pytest.fixture(scope="module")
def mesh():
    return config1_plain()


@pytest.fixture(scope="module")
def pts(mesh):
    rng = np.random.default_rng(21)
    idx = rng.choice(mesh.n_nodes, size=48, replace=False)
    off = rng.uniform(0.05, 0.95, size=(16, 3))
    return np.concatenate([mesh.nodes[idx], off])


def _rel(a, b):
    return np.linalg.norm(a - b) / np.linalg.norm(b)


def test_linearity_in_omega(orc, mesh, pts):
    rng = np.random.default_rng(3)
    w1 = rng.standard_normal(mesh.omega.shape)
    w2 = rng.standard_normal(mesh.omega.shape)
    a, b = 0.7, -1.9
    v1 = orc.velocity(mesh.nodes, mesh.tets, w1, pts, **PARAMS)
    v2 = orc.velocity(mesh.nodes, mesh.tets, w2, pts, **PARAMS)
    v12 = orc.velocity(mesh.nodes, mesh.tets, a * w1 + b * w2, pts, **PARAMS)
    assert _rel(v12, a * v1 + b * v2) < 1e-13


def test_tet_order_and_vertex_order_invariance(orc, mesh, pts):
    rng = np.random.default_rng(4)
    v = orc.velocity(mesh.nodes, mesh.tets, mesh.omega, pts, **PARAMS)
    perm = rng.permutation(mesh.n_tets)
    tets = mesh.tets[perm]
    # random vertex permutation inside every tet (flips orientation for odd ones)
    vp = np.array([rng.permutation(4) for _ in range(len(tets))])
    tets = np.take_along_axis(tets, vp, axis=1)
    v2 = orc.velocity(mesh.nodes, tets, mesh.omega, pts, **PARAMS)
    assert _rel(v2, v) < 1e-13


def test_translation_invariance(orc, mesh, pts):
    shift = np.array([0.25, -0.5, 0.125])  # exact in binary: node coordinates shift without rounding
    v = orc.velocity(mesh.nodes, mesh.tets, mesh.omega, pts, **PARAMS)
    v2 = orc.velocity(mesh.nodes + shift, mesh.tets, mesh.omega, pts + shift, **PARAMS)
    assert _rel(v2, v) < 1e-12


def test_rotation_by_pi_about_z(orc, mesh, pts):
    Rz = np.diag([-1.0, -1.0, 1.0])
    v = orc.velocity(mesh.nodes, mesh.tets, mesh.omega, pts, **PARAMS)
    v2 = orc.velocity(mesh.nodes @ Rz.T, mesh.tets, mesh.omega @ Rz.T, pts @ Rz.T, **PARAMS)
    assert _rel(v2, v @ Rz.T) < 1e-12


def test_precheck_never_changes_results(orc, mesh, pts):
    for fr in (2.0, np.inf):
        p = dict(PARAMS, far_ratio=fr)
        a, ca = orc.velocity(mesh.nodes, mesh.tets, mesh.omega, pts, use_precheck=True, counts=True, **p)
        b, cb = orc.velocity(mesh.nodes, mesh.tets, mesh.omega, pts, use_precheck=False, counts=True, **p)
        assert np.array_equal(a, b) and np.array_equal(ca, cb)


def test_counts_consistent(orc, mesh, pts):
    v, c = orc.velocity(mesh.nodes, mesh.tets, mesh.omega, pts, counts=True, **PARAMS)
    assert np.all(c[:, 0] + c[:, 1] == mesh.n_tets)
    assert np.all(c[:, 2] <= c[:, 0] * 128)
    # every node is a vertex of at least one tet, which is near, and some line enters it
    assert np.all(c[:48, 0] >= 1) and np.all(c[:, 2] > 0)
    vi, ci = orc.velocity(mesh.nodes, mesh.tets, mesh.omega, pts, counts=True, **dict(PARAMS, far_ratio=np.inf))
    assert np.all(ci[:, 0] == mesh.n_tets) and np.all(ci[:, 1] == 0)


def test_thread_count_independent(orc, mesh, pts):
    """Each point's sum is sequential: the result is bit-identical for any OpenMP thread count."""
    import subprocess
    import sys
    import os

    code = (
        "import sys, numpy as np; sys.path[:0] = [%r, %r];"
        "import oracle; from workloads import config1_plain; m = config1_plain();"
        "v = oracle.velocity(m.nodes, m.tets, m.omega, m.nodes[:64]); sys.stdout.write(v.tobytes().hex())"
    ) % (os.path.dirname(os.path.dirname(os.path.abspath(__file__))), os.path.dirname(os.path.abspath(__file__)))
    outs = []
    for nt in ("1", "3"):
        env = dict(os.environ, OMP_NUM_THREADS=nt)
        outs.append(subprocess.run([sys.executable, "-c", code], env=env, capture_output=True, text=True,
                                   check=True).stdout)
    assert outs[0] == outs[1] and len(outs[0]) == 64 * 3 * 16
