"""bs_velocity_nodes: the all-ray velocity at the mesh nodes by walking each line through face neighbours.

On a convex conforming mesh every half-line from a node crosses the tets it
meets one after the other; the sum of their chords is the ray rule's sum over
all tets.  The walk must match the CPU oracle's all-ray velocity at the nodes
(float64: relative L2 <= 1e-12, counts bit-exact on stable nodes; float32: RMS
error over max speed <= 1e-5) and the all-ray kernel.  On a non-convex domain
(an L-shaped block) lines leave and come back; the walk finds the re-entries
through a grid of the boundary faces.  The Heun step uses the same path.
"""
import os

import numpy as np
import pytest
from gpu_helpers import TOL_FP32_RMS_MAX, TOL_FP64_REL_L2, oracle_with_stability, rel_l2, rms_over_max

from workloads import config1_plain, config2_ring
from workloads.mesh import kuhn_grid, orient_positive

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")
if not torch.cuda.is_available():
    pytest.skip("no CUDA device", allow_module_level=True)

import oracle  # noqa: E402
import paper_0712_1695_gb300 as bs  # noqa: E402

ALLRAY = dict(far_ratio=np.inf, tet_gauss_order=4, n_theta=8, n_phi=16)


def _op(p):
    return dict(far_ratio=p["far_ratio"], tet_order=p["tet_gauss_order"], n_theta=p["n_theta"], n_phi=p["n_phi"])


@pytest.fixture(scope="module", autouse=True)
def built():
    bs.build()
    bs.load()


def nodes_velocity(h, n, precision, walk=True, **p):
    cnt = torch.zeros((n, 3), dtype=torch.int32, device="cuda")
    old = os.environ.get("BS_WALK")
    os.environ["BS_WALK"] = "1" if walk else "0"
    try:
        out = h.bs_velocity_nodes(counts_dev=cnt, precision=precision, **p)
        h.bs_status()
    finally:
        if old is None:
            del os.environ["BS_WALK"]
        else:
            os.environ["BS_WALK"] = old
    return out.cpu().numpy(), cnt.cpu().numpy()


@pytest.fixture(scope="module")
def c1():
    m = config1_plain()
    return m, bs.Mesh(m.nodes, m.tets, m.omega)


def test_plain_cube_against_oracle(orc, c1):
    m, h = c1
    vo, co, stable = oracle_with_stability(orc, m, m.nodes, rel=1e-5, **_op(ALLRAY))
    v, c = nodes_velocity(h, m.n_nodes, bs.BS_FP64, **ALLRAY)
    assert rel_l2(v, vo) <= TOL_FP64_REL_L2
    assert stable.mean() >= 0.99
    assert np.array_equal(c[stable], co[stable])
    v32, c32 = nodes_velocity(h, m.n_nodes, bs.BS_FP32, **ALLRAY)
    assert rms_over_max(v32, vo) <= TOL_FP32_RMS_MAX
    assert np.array_equal(c32[:, :2], co[:, :2])
    assert np.abs(c32[:, 2] - co[:, 2]).sum() <= 1e-3 * co[:, 2].sum()


def test_walk_equals_the_all_ray_kernel(c1):
    m, h = c1
    for prec, tol in ((bs.BS_FP64, 1e-13), (bs.BS_FP32, 2e-6)):
        v, c = nodes_velocity(h, m.n_nodes, prec, **ALLRAY)
        vr, cr = nodes_velocity(h, m.n_nodes, prec, walk=False, **ALLRAY)
        if prec == bs.BS_FP64:
            assert np.array_equal(c, cr) and rel_l2(v, vr) <= tol
        else:
            assert np.array_equal(c[:, :2], cr[:, :2]) and rms_over_max(v, vr) <= tol


@pytest.mark.parametrize("n_phi,n_theta", [(4, 4), (32, 16)])
def test_other_direction_tables(orc, c1, n_phi, n_theta):
    m, h = c1
    p = dict(ALLRAY, n_phi=n_phi, n_theta=n_theta)
    vo = orc.velocity(m.nodes, m.tets, m.omega, m.nodes, **_op(p))
    v, _ = nodes_velocity(h, m.n_nodes, bs.BS_FP64, **p)
    assert rel_l2(v, vo) <= TOL_FP64_REL_L2


def test_after_moving_the_nodes(orc):
    """bs_update moves the nodes (the domain stays convex): the walk uses the new positions."""
    m = config1_plain()
    h = bs.Mesh(m.nodes, m.tets, m.omega)
    nodes_velocity(h, m.n_nodes, bs.BS_FP64, **ALLRAY)
    rng = np.random.default_rng(5)
    interior = np.all((m.nodes > 1e-9) & (m.nodes < 1 - 1e-9), axis=1)
    nodes2 = m.nodes.copy()
    nodes2[interior] += 0.01 * rng.standard_normal((interior.sum(), 3))
    omega2 = 0.5 * m.omega + 0.1
    h.bs_update(torch.from_numpy(nodes2).cuda(), torch.from_numpy(omega2).cuda())
    v, _ = nodes_velocity(h, m.n_nodes, bs.BS_FP64, **ALLRAY)
    vo = orc.velocity(nodes2, m.tets, omega2, nodes2, **_op(ALLRAY))
    assert rel_l2(v, vo) <= TOL_FP64_REL_L2


def _l_shaped():
    """The plain cube's Kuhn grid without the tets of the corner block x > 0.5, y > 0.5 (non-convex)."""
    nodes, tets = kuhn_grid(9, 0.0, 1.0)
    c = nodes[tets].mean(axis=1)
    keep = ~((c[:, 0] > 0.5) & (c[:, 1] > 0.5))
    tets = tets[keep]
    used = np.unique(tets)
    remap = -np.ones(len(nodes), dtype=np.int64)
    remap[used] = np.arange(len(used))
    nodes = nodes[used]
    tets = orient_positive(nodes, remap[tets].astype(np.int32))
    rng = np.random.default_rng(11)
    omega = np.array([0.0, 0.0, 1.0]) + 0.1 * rng.standard_normal((len(nodes), 3))
    return nodes, tets, omega


def test_non_convex_domain_walks_with_re_entries(orc):
    """An L-shaped block: lines that leave the mesh come back into it; the walk finds the re-entries through a
    grid of boundary faces, and matches the oracle and the all-ray kernel (counts exactly)."""
    nodes, tets, omega = _l_shaped()
    h = bs.Mesh(nodes, tets, omega)
    vo, co, stable = oracle_with_stability(orc, _Mesh(nodes, tets, omega), nodes, **_op(ALLRAY))
    v, c = nodes_velocity(h, len(nodes), bs.BS_FP64, **ALLRAY)
    vr, cr = nodes_velocity(h, len(nodes), bs.BS_FP64, walk=False, **ALLRAY)
    assert rel_l2(v, vo) <= TOL_FP64_REL_L2
    assert rel_l2(v, vr) <= 1e-13
    assert np.array_equal(c, cr)
    assert np.array_equal(c[stable], co[stable])
    v32, _ = nodes_velocity(h, len(nodes), bs.BS_FP32, **ALLRAY)
    assert rms_over_max(v32, vo) <= TOL_FP32_RMS_MAX


class _Mesh:
    def __init__(self, nodes, tets, omega):
        self.nodes, self.tets, self.omega = nodes, tets, omega


def test_ring_mesh_full_size(orc):
    """The 32^3 Gaussian-ring mesh: walk against the all-ray kernel at all 32768 nodes (float32) and
    the oracle on 48 seeded nodes (float64)."""
    m = config2_ring()
    h = bs.Mesh(m.nodes, m.tets, m.omega)
    v, c = nodes_velocity(h, m.n_nodes, bs.BS_FP32, **ALLRAY)
    vr, cr = nodes_velocity(h, m.n_nodes, bs.BS_FP32, walk=False, **ALLRAY)
    assert rms_over_max(v, vr) <= 2e-6
    assert np.array_equal(c[:, :2], cr[:, :2])
    assert np.abs(c[:, 2] - cr[:, 2]).sum() <= 1e-4 * cr[:, 2].sum()
    v64, _ = nodes_velocity(h, m.n_nodes, bs.BS_FP64, **ALLRAY)
    idx = np.random.default_rng(2002).choice(m.n_nodes, size=48, replace=False)
    vo = orc.velocity(m.nodes, m.tets, m.omega, m.nodes[idx], **_op(ALLRAY))
    assert rel_l2(v64[idx], vo) <= TOL_FP64_REL_L2
    assert rms_over_max(v[idx], vo) <= TOL_FP32_RMS_MAX


def test_heun_step_all_ray_uses_the_walk(orc, c1):
    m, _ = c1
    h = bs.Mesh(m.nodes, m.tets, m.omega)
    dt = 0.01
    h.bs_rk2_step(dt, precision=bs.BS_FP64, **ALLRAY)
    h.bs_status()
    x1 = h.bs_nodes().cpu().numpy()
    ref = oracle.heun_step(orc, m.nodes, m.tets, m.omega, dt, **_op(ALLRAY))
    assert np.abs(x1 - ref).max() <= 1e-12 * max(1.0, np.abs(ref).max())


def test_hybrid_rule_at_the_nodes_matches_bs_velocity(c1):
    """With a finite far ratio bs_velocity_nodes computes the rule bs_velocity computes at the nodes (the near
    field by the walk or in the far kernel, whichever variant each path takes): equal to rounding, with the same
    near/far split (the same float test decides it) and, to a few grazing lines, the same ray hits."""
    m, h = c1
    p = dict(far_ratio=2.0, tet_gauss_order=4, n_theta=8, n_phi=16)
    for prec in (bs.BS_FP64, bs.BS_FP32):
        v, c = nodes_velocity(h, m.n_nodes, prec, **p)
        cnt = torch.zeros((m.n_nodes, 3), dtype=torch.int32, device="cuda")
        vr = h.bs_velocity(torch.from_numpy(m.nodes).cuda(), counts_dev=cnt, precision=prec, **p).cpu().numpy()
        h.bs_status()
        cr = cnt.cpu().numpy()
        if prec == bs.BS_FP64:
            assert rel_l2(v, vr) <= TOL_FP64_REL_L2
        else:
            assert rms_over_max(v, vr) <= TOL_FP32_RMS_MAX
        assert np.array_equal(c[:, :2], cr[:, :2])
        assert np.abs(c[:, 2] - cr[:, 2]).sum() <= 1e-3 * cr[:, 2].sum()


def test_box_deformed_by_lagrangian_steps(orc):
    """Three Heun steps with vortex stretching bend the cube's faces (a non-convex domain, lines grazing the
    bent faces leave and re-enter): on the moved mesh the walk matches the all-ray kernel and the oracle."""
    m = config1_plain()
    h = bs.Mesh(m.nodes, m.tets, m.omega)
    for _ in range(3):
        h.bs_rk2_step_stretch(0.02, precision=bs.BS_FP64, **ALLRAY)
    h.bs_status()
    nodes, omega = h.bs_nodes().cpu().numpy(), h.bs_omega().cpu().numpy()
    assert np.abs(nodes - m.nodes).max() > 1e-3
    h2 = bs.Mesh(nodes, m.tets, omega)
    v, c = nodes_velocity(h2, m.n_nodes, bs.BS_FP64, **ALLRAY)
    vr, cr = nodes_velocity(h2, m.n_nodes, bs.BS_FP64, walk=False, **ALLRAY)
    assert rel_l2(v, vr) <= 1e-13
    assert np.array_equal(c, cr)
    vo = orc.velocity(nodes, m.tets, omega, nodes, **_op(ALLRAY))
    assert rel_l2(v, vo) <= TOL_FP64_REL_L2


@pytest.mark.parametrize("n", [8, 11])
def test_ball_mesh(orc, n):
    """A jittered Kuhn grid mapped onto the unit ball (Hill's vortex, Section 3.1): flattened tets near the
    mapped cube's edges and a faceted boundary; the walk matches the all-ray kernel and the oracle."""
    from workloads import ball_mesh, hill_vorticity

    b = ball_mesh(n, hill_vorticity, jitter=0.1)
    h = bs.Mesh(b.nodes, b.tets, b.omega)
    p = dict(ALLRAY, n_theta=16, n_phi=16)
    v, c = nodes_velocity(h, len(b.nodes), bs.BS_FP64, **p)
    vr, cr = nodes_velocity(h, len(b.nodes), bs.BS_FP64, walk=False, **p)
    assert rel_l2(v, vr) <= 1e-13
    assert np.array_equal(c, cr)
    vo = orc.velocity(b.nodes, b.tets, b.omega, b.nodes, **_op(p))
    assert rel_l2(v, vo) <= TOL_FP64_REL_L2
    v32, _ = nodes_velocity(h, len(b.nodes), bs.BS_FP32, **p)
    assert rms_over_max(v32, vo) <= TOL_FP32_RMS_MAX


def test_hill_vortex_error_falls_with_the_mesh():
    """Hill's spherical vortex (Section 3.1, the Table 1 case) by the all-ray walk at 16 x 16 directions on
    jittered balls of 10^3 and 16^3 grid nodes: the r.m.s. error against the closed-form velocity falls, and is
    below 1.5e-3 (largest speed 1/3) on the finer mesh."""
    from workloads import ball_mesh, hill_velocity, hill_vorticity

    p = dict(ALLRAY, n_theta=16, n_phi=16)
    eps = []
    for n in (10, 16):
        b = ball_mesh(n, hill_vorticity, jitter=0.1)
        h = bs.Mesh(b.nodes, b.tets, b.omega)
        v, _ = nodes_velocity(h, len(b.nodes), bs.BS_FP32, **p)
        eps.append(float(np.sqrt(np.mean(np.sum((v - hill_velocity(b.nodes)) ** 2, axis=1)))))
    assert eps[1] < 0.7 * eps[0]
    assert eps[1] < 1.5e-3
