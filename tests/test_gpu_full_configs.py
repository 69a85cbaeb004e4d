"""The batch and the Lagrangian workloads at their full stated sizes, against the oracle on sampled nodes.

* 256 independent meshes (n ~ U{8..24} nodes per side, Gaussian blobs) in one
  batched launch, float32: RMS error over max speed <= 1e-5 against the oracle
  on up to 256 seeded nodes of 8 meshes, among them the smallest and the
  largest.
* One Heun step of the two colliding rings on the 80^3 grid (512000 nodes,
  2958234 tets), float32.  The oracle's Heun step needs the velocity at every
  node (the whole mesh moves before the second stage), which is out of reach
  on the host; so the first stage is taken at all nodes from the GPU's own
  float32 evaluation (the one bs_rk2_step runs), the moved mesh is built from
  it, and the oracle evaluates both stages at 256 seeded nodes: the step's
  displacement there must match the GPU's to RMS over max <= 1e-5.
"""
import numpy as np
import pytest
from gpu_helpers import TOL_FP32_RMS_MAX, rms_over_max

from workloads import config4_batch, config5_rings

pytestmark = [pytest.mark.gpu, pytest.mark.slow]

torch = pytest.importorskip("torch")
if not torch.cuda.is_available():
    pytest.skip("no CUDA device", allow_module_level=True)

import paper_0712_1695_gb300 as bs  # noqa: E402

P = dict(far_ratio=2.0, tet_gauss_order=4, n_theta=8, n_phi=16)
OP = dict(far_ratio=2.0, tet_order=4, n_theta=8, n_phi=16)


def test_batch_of_256_meshes_against_oracle(orc):
    bs.build()
    ms = config4_batch()  # the stated size: 256 meshes, n ~ U{8..24}
    assert len(ms) == 256
    hs = [bs.Mesh(m.nodes, m.tets, m.omega) for m in ms]
    batch = bs.Batch(hs)
    stream = torch.cuda.Stream()
    outs = [torch.full((m.n_nodes, 3), float("nan"), dtype=torch.float64, device="cuda") for m in ms]
    with torch.cuda.stream(stream):
        batch.bs_batch_velocity(outs, stream=stream, precision=bs.BS_FP32, **P)
    stream.synchronize()
    sizes = np.array([m.n_tets for m in ms])
    rng = np.random.default_rng(256)
    others = rng.choice(np.setdiff1d(np.arange(256), [sizes.argmin(), sizes.argmax()]), size=6, replace=False)
    chosen = [int(sizes.argmin()), int(sizes.argmax()), *map(int, others)]
    for i in chosen:
        m = ms[i]
        idx = np.sort(rng.choice(m.n_nodes, size=min(256, m.n_nodes), replace=False))
        ref = orc.velocity(m.nodes, m.tets, m.omega, m.nodes[idx], **OP)
        v = outs[i].cpu().numpy()[idx]
        assert rms_over_max(v, ref) <= TOL_FP32_RMS_MAX, f"mesh {i} ({m.n_side}^3)"
    assert all(torch.isfinite(o).all() for o in outs)


def test_rings_80_heun_step_sampled(orc):
    bs.build()
    m = config5_rings(80)
    assert m.n_nodes == 512000
    dt = 0.01
    # the GPU's step
    h = bs.Mesh(m.nodes, m.tets, m.omega)
    h.bs_rk2_step(dt, precision=bs.BS_FP32, **P)
    h.bs_status()
    x1 = h.bs_nodes().cpu().numpy()
    # its first stage at all nodes (the same deterministic float32 evaluation) gives the moved mesh
    h0 = bs.Mesh(m.nodes, m.tets, m.omega)
    v0 = h0.bs_velocity_nodes(precision=bs.BS_FP32, **P).cpu().numpy()
    h0.bs_status()
    xs = m.nodes + dt * v0
    # the oracle's Heun step at seeded nodes: both stages evaluated there
    idx = np.sort(np.random.default_rng(80).choice(m.n_nodes, size=256, replace=False))
    v0o = orc.velocity(m.nodes, m.tets, m.omega, m.nodes[idx], **OP)
    v1o = orc.velocity(xs, m.tets, m.omega, xs[idx], **OP)
    step_o = 0.5 * dt * (v0o + v1o)
    step = x1[idx] - m.nodes[idx]
    assert np.abs(step_o).max() > 1e-4  # the rings move
    assert rms_over_max(step, step_o) <= TOL_FP32_RMS_MAX
