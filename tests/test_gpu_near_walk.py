"""The hybrid rule at the mesh's nodes with the near field taken by the mesh walk.

bs_velocity_nodes with a finite far ratio and a kernel variant that leaves the
near pairs to a pass of their own: the far sweep leaves them out, and the walk
traces each line from the node through the near tets (those the far sweep's
test calls near, decided bit for bit the same way) until every later tet must
be far.  The result is the paper's rule (Gauss far field, ray near field), so
it must match the FP64 oracle: float64 at relative L2 <= 1e-12, float32 at RMS
over max speed <= 1e-5, near/far counts bit-exact on stable nodes and the ray
hits of the near tets (float64: bit-exact on stable nodes).  The same result
must come from the near pass when the walk is switched off, on a deformed
(non-convex) mesh where lines leave and come back, and inside the Heun step.
"""
import numpy as np
import pytest
from gpu_helpers import TOL_FP32_RMS_MAX, TOL_FP64_REL_L2, oracle_with_stability, rel_l2, rms_over_max

from workloads import config1_plain, config5_rings

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")
if not torch.cuda.is_available():
    pytest.skip("no CUDA device", allow_module_level=True)

import paper_0712_1695_gb300 as bs  # noqa: E402

bs.build()
P = dict(far_ratio=2.0, tet_gauss_order=4, n_theta=8, n_phi=16)
OP = dict(far_ratio=2.0, tet_order=4, n_theta=8, n_phi=16)


def near_pass_variants(prec, q=4):
    return [v for v in range(bs.bs_num_variants(prec, q)) if bs.bs_variant_shape(prec, q, 0, v)["near_drain"] == 3]


CASES = [(bs.BS_FP64, v) for v in near_pass_variants(bs.BS_FP64)] + \
        [(bs.BS_FP32, v) for v in near_pass_variants(bs.BS_FP32)]


@pytest.fixture(scope="module")
def rings(orc):
    m = config5_rings(16)
    vo, co, stable = oracle_with_stability(orc, m, m.nodes, rel=1e-5, **OP)
    assert stable.mean() >= 0.99
    return m, bs.Mesh(m.nodes, m.tets, m.omega), vo, co, stable


def _nodes(h, prec, variant, counts=True, **extra):
    params = dict(P, **extra)
    n = h.n_nodes
    cnt = torch.full((n, 3), -1, dtype=torch.int32, device="cuda") if counts else None
    h.bs_set_variant(prec, params["tet_gauss_order"], bs.BS_NEAR_RAY, variant)
    try:
        v = h.bs_velocity_nodes(counts_dev=cnt, precision=prec, **params)
        h.bs_status()
    finally:
        h.bs_set_variant(prec, params["tet_gauss_order"], bs.BS_NEAR_RAY, -1)
    return v.cpu().numpy(), (cnt.cpu().numpy() if counts else None)


@pytest.mark.parametrize("prec,variant", CASES,
                         ids=[f"{'fp64' if p == bs.BS_FP64 else 'fp32'}-v{v}" for p, v in CASES])
def test_near_walk_at_nodes_matches_oracle(rings, prec, variant):
    m, h, vo, co, stable = rings
    v, c = _nodes(h, prec, variant)
    if prec == bs.BS_FP64:
        assert rel_l2(v, vo) <= TOL_FP64_REL_L2
        assert np.array_equal(c[stable], co[stable])
    else:
        assert rms_over_max(v, vo) <= TOL_FP32_RMS_MAX
        assert np.array_equal(c[stable, :2], co[stable, :2])
        assert np.abs(c[:, 2] - co[:, 2]).sum() <= 1e-3 * co[:, 2].sum()


@pytest.mark.parametrize("prec", [bs.BS_FP64, bs.BS_FP32], ids=["fp64", "fp32"])
def test_near_walk_equals_near_pass(rings, prec, monkeypatch):
    m, h, *_ = rings
    variant = near_pass_variants(prec)[0]
    walk, cw = _nodes(h, prec, variant)
    monkeypatch.setenv("BS_WALK", "0")  # the near pass takes the near pairs
    npass, cp = _nodes(h, prec, variant)
    if prec == bs.BS_FP64:
        assert rel_l2(walk, npass) <= TOL_FP64_REL_L2
    else:
        assert rms_over_max(walk, npass) <= TOL_FP32_RMS_MAX
    assert np.array_equal(cw[:, :2], cp[:, :2])


def test_near_walk_on_a_deformed_mesh(orc):
    """Nodes moved by a smooth non-affine map: the box is no longer convex, lines leave and re-enter."""
    m = config1_plain()
    h = bs.Mesh(m.nodes, m.tets, m.omega)
    x = m.nodes
    nodes2 = x + 0.06 * np.stack([np.sin(2 * np.pi * x[:, 1]), np.sin(2 * np.pi * x[:, 2]),
                                  np.sin(2 * np.pi * x[:, 0])], axis=1)
    h.bs_update(torch.from_numpy(nodes2).cuda(), None)
    h.bs_status()
    vo = orc.velocity(nodes2, m.tets, m.omega, nodes2, **OP)
    for prec, variant in ((bs.BS_FP64, near_pass_variants(bs.BS_FP64)[0]), (bs.BS_FP32, near_pass_variants(bs.BS_FP32)[0])):
        v, _ = _nodes(h, prec, variant, counts=False)
        if prec == bs.BS_FP64:
            assert rel_l2(v, vo) <= TOL_FP64_REL_L2
        else:
            assert rms_over_max(v, vo) <= TOL_FP32_RMS_MAX


def test_heun_step_with_the_near_walk(orc):
    """bs_rk2_step evaluates through bs_velocity_nodes: with a near-pass variant the walk takes the near field."""
    from oracle import heun_step

    m = config1_plain()
    h = bs.Mesh(m.nodes, m.tets, m.omega)
    h.bs_set_variant(bs.BS_FP64, 4, bs.BS_NEAR_RAY, near_pass_variants(bs.BS_FP64)[0])
    h.bs_rk2_step(0.02, precision=bs.BS_FP64, **P)
    h.bs_status()
    x1 = h.bs_nodes().cpu().numpy()
    ref = heun_step(orc, m.nodes, m.tets, m.omega, 0.02, **OP)
    assert rel_l2(x1 - m.nodes, ref - m.nodes) <= 1e-11
