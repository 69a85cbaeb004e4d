"""Input generators: sizes, orientation, conformity and seeding (no GPU)."""
import numpy as np

from workloads import config1_plain, config2_ring, config3_samples, kuhn_grid
from workloads.configs import ball_mesh, config4_batch
from workloads.mesh import tet_volumes6


def test_kuhn_grid_counts_and_volume():
    for n in (2, 3, 5):
        nodes, tets = kuhn_grid(n, -1.0, 1.0)
        assert nodes.shape == (n**3, 3) and tets.shape == (6 * (n - 1) ** 3, 4)
        vol = tet_volumes6(nodes, tets) / 6
        assert np.all(vol > 0)
        assert abs(vol.sum() - 8.0) < 1e-12


def test_kuhn_grid_is_conforming():
    """Every interior face is shared by exactly two tets, boundary faces by one."""
    n = 4
    nodes, tets = kuhn_grid(n, 0.0, 1.0)
    faces = {}
    for t in tets:
        for f in ((1, 2, 3), (0, 2, 3), (0, 1, 3), (0, 1, 2)):
            key = tuple(sorted(t[list(f)]))
            faces[key] = faces.get(key, 0) + 1
    counts = np.array(list(faces.values()))
    assert set(counts) <= {1, 2}
    assert (counts == 1).sum() == 6 * 2 * (n - 1) ** 2  # two triangles per boundary square


def test_config_sizes_and_seeds():
    a, b = config1_plain(), config1_plain()
    assert a.n_nodes == 729 and a.n_tets == 3072
    assert np.array_equal(a.nodes, b.nodes) and np.array_equal(a.omega, b.omega)
    assert np.all(tet_volumes6(a.nodes, a.tets) > 0)
    c2 = config2_ring()
    assert c2.n_nodes == 32768 and c2.n_tets == 178746
    s = config3_samples(64**3)
    assert len(s) == 4096 and len(np.unique(s)) == 4096


def test_ball_and_batch():
    b = ball_mesh(9)
    assert np.all(tet_volumes6(b.nodes, b.tets) > 0)
    assert np.linalg.norm(b.nodes, axis=1).max() <= 1.0 + 1e-15
    batch = config4_batch(count=4)
    assert len(batch) == 4 and all(8 <= m.n_side <= 24 for m in batch)


def test_jittered_ball_is_not_folded():
    """The jittered ball keeps every tet at >= 1/4 of its unjittered volume and positive, and no two tets that share
    a face lie on the same side of it (the ball map alone would fold tets near the origin)."""
    for n in (8, 11, 16):
        b = ball_mesh(n, jitter=0.1)
        b0 = ball_mesh(n)
        v, v0 = tet_volumes6(b.nodes, b.tets), tet_volumes6(b0.nodes, b0.tets)
        assert np.all(v > 0) and np.all(v >= 0.25 * v0 - 1e-15)
        assert np.abs(b.nodes - b0.nodes).max() > 0  # the jitter moved the interior
        # every interior face: the two opposite vertices on opposite sides of its plane
        faces = {}
        for t, tet in enumerate(b.tets):
            for k in range(4):
                key = tuple(sorted(np.delete(tet, k)))
                faces.setdefault(key, []).append((t, tet[k]))
        for key, owners in faces.items():
            if len(owners) != 2:
                continue
            p0, p1, p2 = b.nodes[list(key)]
            nrm = np.cross(p1 - p0, p2 - p0)
            s = [np.dot(nrm, b.nodes[o] - p0) for _, o in owners]
            assert s[0] * s[1] < 0
