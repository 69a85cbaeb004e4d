"""Derivative of the all-ray velocity along directions at the nodes (bs_velocity_nodes_dderiv) and the Heun
step with vortex stretching (bs_rk2_step_stretch), through the C ABI, against the oracle.

The derivative is computed during the mesh walk; the oracle computes it from
its definition over all tets (chord lengths times the vorticity gradient, plus
the jump of omega at the mesh boundary) and is pinned by central differences
of its own velocity.  float64: velocity relative L2 <= 1e-12; derivative
relative L2 <= 1e-11 (the oracle's per-tet sum cancels the chord-end terms of
neighbouring tets, up to rounding relative to terms ~1/|n.s| larger than the
result; the walk leaves them out).  float32: RMS error over the largest value
<= 1e-5 for the velocity, 1e-4 for the derivative.
"""
import numpy as np
import pytest
from gpu_helpers import TOL_FP32_RMS_MAX, TOL_FP64_REL_L2, rel_l2, rms_over_max

from workloads import config1_plain, config2_ring
from workloads.mesh import kuhn_grid, orient_positive

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")
if not torch.cuda.is_available():
    pytest.skip("no CUDA device", allow_module_level=True)

import oracle  # noqa: E402
import paper_0712_1695_gb300 as bs  # noqa: E402
from paper_0712_1695_gb300.binding import BS_ERR_ARG, BS_ERR_MESH, BSError  # noqa: E402

ALLRAY = dict(far_ratio=np.inf, tet_gauss_order=4, n_theta=8, n_phi=16)
TOL_DERIV_FP64 = 1e-11
TOL_DERIV_FP32 = 1e-4


@pytest.fixture(scope="module", autouse=True)
def built():
    bs.build()
    bs.load()


@pytest.fixture(scope="module")
def c1():
    m = config1_plain()
    return m, bs.Mesh(m.nodes, m.tets, m.omega)


def dderiv(h, precision, dirs=None, **p):
    d = None if dirs is None else torch.from_numpy(np.ascontiguousarray(dirs)).cuda()
    v, dv = h.bs_velocity_nodes_dderiv(dirs_dev=d, precision=precision, **p)
    h.bs_status()
    return v.cpu().numpy(), dv.cpu().numpy()


@pytest.mark.parametrize("which", ["vorticity", "random"])
def test_plain_cube_against_oracle(orc, c1, which):
    m, h = c1
    dirs = m.omega if which == "vorticity" else np.random.default_rng(4).standard_normal(m.nodes.shape)
    vo, do = orc.velocity_dderiv(m.nodes, m.tets, m.omega, m.nodes, dirs, n_theta=8, n_phi=16)
    v, dv = dderiv(h, bs.BS_FP64, None if which == "vorticity" else dirs, **ALLRAY)
    assert rel_l2(v, vo) <= TOL_FP64_REL_L2
    assert rel_l2(dv, do) <= TOL_DERIV_FP64
    v32, dv32 = dderiv(h, bs.BS_FP32, None if which == "vorticity" else dirs, **ALLRAY)
    assert rms_over_max(v32, vo) <= TOL_FP32_RMS_MAX
    assert rms_over_max(dv32, do) <= TOL_DERIV_FP32


def test_heun_step_with_stretching_against_oracle(orc, c1):
    m, _ = c1
    h = bs.Mesh(m.nodes, m.tets, m.omega)
    dt = 0.01
    h.bs_rk2_step_stretch(dt, precision=bs.BS_FP64, **ALLRAY)
    h.bs_status()
    x1, w1 = h.bs_nodes().cpu().numpy(), h.bs_omega().cpu().numpy()
    xr, wr = oracle.heun_step_stretch(orc, m.nodes, m.tets, m.omega, dt)
    assert rel_l2(x1 - m.nodes, xr - m.nodes) <= 1e-10
    assert rel_l2(w1 - m.omega, wr - m.omega) <= 1e-9
    assert np.abs(wr - m.omega).max() > 1e-4  # the vorticity did change


def test_other_parameters_are_rejected(c1):
    m, h = c1
    with pytest.raises(BSError) as ei:
        h.bs_velocity_nodes_dderiv(precision=bs.BS_FP64, far_ratio=2.0, tet_gauss_order=4, n_theta=8, n_phi=16)
    assert ei.value.code == BS_ERR_ARG


def test_non_convex_domain(orc):
    """An L-shaped block: the derivative includes the jumps where lines come back into the mesh."""
    nodes, tets = kuhn_grid(9, 0.0, 1.0)
    c = nodes[tets].mean(axis=1)
    tets = tets[~((c[:, 0] > 0.5) & (c[:, 1] > 0.5))]
    used = np.unique(tets)
    remap = -np.ones(len(nodes), dtype=np.int64)
    remap[used] = np.arange(len(used))
    nodes = nodes[used]
    tets = orient_positive(nodes, remap[tets].astype(np.int32))
    omega = np.array([0.0, 0.0, 1.0]) + 0.2 * np.random.default_rng(13).standard_normal((len(nodes), 3))
    h = bs.Mesh(nodes, tets, omega)
    v, dv = dderiv(h, bs.BS_FP64, **ALLRAY)
    vo, do = orc.velocity_dderiv(nodes, tets, omega, nodes, omega, n_theta=8, n_phi=16)
    assert rel_l2(v, vo) <= TOL_FP64_REL_L2
    assert rel_l2(dv, do) <= TOL_DERIV_FP64


def test_mesh_the_walk_cannot_serve_reports_no_derivative():
    """A node that belongs to no tet: the velocity is computed (all-ray kernel), the derivative is not."""
    m = config1_plain()
    nodes = np.vstack([m.nodes, [[0.5, 0.5, 0.5]]])
    omega = np.vstack([m.omega, [[0.0, 0.0, 1.0]]])
    h = bs.Mesh(nodes, m.tets, omega)
    h.bs_velocity_nodes_dderiv(precision=bs.BS_FP64, **ALLRAY)
    with pytest.raises(BSError) as ei:
        h.bs_status()
    assert ei.value.code == BS_ERR_MESH


def _folded_ball(n=8):
    """Jittered Kuhn grid mapped onto the ball with no guard against the map's kink at the origin: a few
    tets turn inside out and are re-oriented, so neighbours overlap (a folded mesh)."""
    from workloads.mesh import cube_to_ball, jitter_interior, tet_volumes6

    base, tets = kuhn_grid(n, -1.0, 1.0)
    tets = orient_positive(base, tets)
    nodes = cube_to_ball(jitter_interior(base, n, 0.1, np.random.default_rng(77)))
    assert (tet_volumes6(nodes, tets) < 0).sum() > 0
    tets = orient_positive(nodes, tets)
    omega = np.array([0.0, 0.0, 1.0]) + 0.2 * np.random.default_rng(14).standard_normal((len(nodes), 3))
    return nodes, tets, omega


def test_folded_mesh_is_served_by_the_ray_kernel(orc):
    """A folded mesh: the walk is switched off, the node velocities come from the all-ray kernel and still
    match the oracle (which sums every tet as given), and the derivative is refused."""
    nodes, tets, omega = _folded_ball()
    h = bs.Mesh(nodes, tets, omega)
    v = h.bs_velocity_nodes(precision=bs.BS_FP64, **ALLRAY).cpu().numpy()
    h.bs_status()
    vo = orc.velocity(nodes, tets, omega, nodes, tet_order=4, far_ratio=np.inf, n_theta=8, n_phi=16)
    assert rel_l2(v, vo) <= TOL_FP64_REL_L2
    h.bs_velocity_nodes_dderiv(precision=bs.BS_FP64, **ALLRAY)
    with pytest.raises(BSError) as ei:
        h.bs_status()
    assert ei.value.code == BS_ERR_MESH


def test_ring_mesh_full_size(orc):
    """The 32^3 ring mesh: float32 against float64 at all 32768 nodes, 24 seeded nodes against the oracle."""
    m = config2_ring()
    h = bs.Mesh(m.nodes, m.tets, m.omega)
    v64, d64 = dderiv(h, bs.BS_FP64, **ALLRAY)
    v32, d32 = dderiv(h, bs.BS_FP32, **ALLRAY)
    assert rms_over_max(v32, v64) <= TOL_FP32_RMS_MAX
    assert rms_over_max(d32, d64) <= TOL_DERIV_FP32
    idx = np.random.default_rng(2002).choice(m.n_nodes, size=24, replace=False)
    vo, do = orc.velocity_dderiv(m.nodes, m.tets, m.omega, m.nodes[idx], m.omega[idx], n_theta=8, n_phi=16)
    assert rel_l2(v64[idx], vo) <= TOL_FP64_REL_L2
    assert rel_l2(d64[idx], do) <= TOL_DERIV_FP64
