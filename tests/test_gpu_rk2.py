"""The Lagrangian stage driver (Heun / RK2 steps of the node positions) on the GPU.

One float64 step against the oracle's Heun step (velocity at the nodes, move,
velocity on the moved mesh, average); and 20 steps of the colliding-rings
workload on a 24^3 grid, float32 against float64 trajectories.
"""
import numpy as np
import pytest
from gpu_helpers import rel_l2

from workloads import config1_plain, config5_rings

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")
if not torch.cuda.is_available():
    pytest.skip("no CUDA device", allow_module_level=True)

import oracle  # noqa: E402
import paper_0712_1695_gb300 as bs  # noqa: E402

P = dict(far_ratio=2.0, tet_gauss_order=4, n_theta=8, n_phi=16)


def test_one_heun_step_matches_oracle(orc):
    m = config1_plain()
    h = bs.Mesh(m.nodes, m.tets, m.omega)
    dt = 0.02
    h.bs_rk2_step(dt, precision=bs.BS_FP64, **P)
    h.bs_status()
    x1 = h.bs_nodes().cpu().numpy()
    ref = oracle.heun_step(orc, m.nodes, m.tets, m.omega, dt, far_ratio=2.0, tet_order=4, n_theta=8, n_phi=16)
    # compare the displacements (the positions themselves are O(1))
    assert rel_l2(x1 - m.nodes, ref - m.nodes) <= 1e-11
    # and a second step from there
    h.bs_rk2_step(dt, precision=bs.BS_FP64, **P)
    h.bs_status()
    x2 = h.bs_nodes().cpu().numpy()
    ref2 = oracle.heun_step(orc, ref, m.tets, m.omega, dt, far_ratio=2.0, tet_order=4, n_theta=8, n_phi=16)
    assert rel_l2(x2 - ref, ref2 - ref) <= 1e-10


def test_rings_trajectory_fp32_vs_fp64():
    m = config5_rings(n=24)
    traj = {}
    for prec in (bs.BS_FP64, bs.BS_FP32):
        h = bs.Mesh(m.nodes, m.tets, m.omega)
        for _ in range(20):
            h.bs_rk2_step(0.01, precision=prec, **P)
        h.bs_status()
        traj[prec] = h.bs_nodes().cpu().numpy()
    d64, d32 = traj[bs.BS_FP64] - m.nodes, traj[bs.BS_FP32] - m.nodes
    assert np.abs(d64).max() > 1e-3  # the rings did move
    drift = np.linalg.norm(traj[bs.BS_FP32] - traj[bs.BS_FP64], axis=1)
    assert drift.max() <= 1e-5 * np.abs(d64).max() * 100  # <= 1e-3 of the largest displacement
    assert np.sqrt(np.mean(drift**2)) <= 1e-5 * np.abs(d64).max()


@pytest.mark.parametrize("side_stream", [False, True])
def test_graph_steps_equal_eager_steps(side_stream):
    """bs_rk2_steps (first step eager, the rest replayed from a captured CUDA graph) moves the nodes exactly as
    the same number of bs_rk2_step calls, on the default stream and on a side stream."""
    m = config1_plain()
    params = dict(P, precision=bs.BS_FP32)
    eager = bs.Mesh(m.nodes, m.tets, m.omega)
    for _ in range(6):
        eager.bs_rk2_step(0.02, **params)
    eager.bs_status()
    g = bs.Mesh(m.nodes, m.tets, m.omega)
    stream = torch.cuda.Stream() if side_stream else None
    g.bs_rk2_steps(0.02, 6, stream=stream, **params)
    if stream is not None:
        stream.synchronize()
    g.bs_status()
    assert g.bs_graph_steps() == 5
    assert np.array_equal(g.bs_nodes().cpu().numpy(), eager.bs_nodes().cpu().numpy())
    # zero steps change nothing; a negative count is an argument error
    before = g.bs_nodes().cpu().numpy()
    g.bs_rk2_steps(0.02, 0, **params)
    assert np.array_equal(g.bs_nodes().cpu().numpy(), before)
    with pytest.raises(bs.BSError):
        g.bs_rk2_steps(0.02, -1, **params)


def test_graph_steps_with_stretching_equal_eager_steps():
    """The same for the all-ray Heun step with vortex stretching (the mesh walk, nodes and vorticity)."""
    m = config1_plain()
    params = dict(far_ratio=np.inf, tet_gauss_order=4, n_theta=4, n_phi=8, precision=bs.BS_FP32)
    eager = bs.Mesh(m.nodes, m.tets, m.omega)
    for _ in range(4):
        eager.bs_rk2_step_stretch(0.01, **params)
    eager.bs_status()
    g = bs.Mesh(m.nodes, m.tets, m.omega)
    g.bs_rk2_steps(0.01, 4, stretch=True, **params)
    g.bs_status()
    assert g.bs_graph_steps() == 3
    assert np.array_equal(g.bs_nodes().cpu().numpy(), eager.bs_nodes().cpu().numpy())
    assert np.array_equal(g.bs_omega().cpu().numpy(), eager.bs_omega().cpu().numpy())
