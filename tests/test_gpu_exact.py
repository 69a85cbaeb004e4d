"""The exact near-field rule (near_rule = BS_NEAR_EXACT: the analytic evaluation that Section 1 compares the
ray rule against) through the C ABI.

Near pairs take the exact single-tet integral in float64 under both precisions; far pairs keep the Gauss
rule.  The GPU must match the CPU oracle's near_rule 1 (float64: relative L2 <= 1e-12, near/far counts
bit-exact on stable points, no ray hits; float32: RMS error over max speed <= 1e-5) at nodes, at points
inside tets, on faces and edges, and outside the mesh, with every tet exact (far_ratio = +inf), in the
batched launch, and on the 32^3 ring mesh at full size.
"""
import numpy as np
import pytest
from gpu_helpers import TOL_FP32_RMS_MAX, TOL_FP64_REL_L2, oracle_with_stability, rel_l2, rms_over_max

from workloads import config1_plain, config2_ring, config4_batch

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")
if not torch.cuda.is_available():
    pytest.skip("no CUDA device", allow_module_level=True)

import paper_0712_1695_gb300 as bs  # noqa: E402
from paper_0712_1695_gb300.binding import BS_ERR_ARG, BSError  # noqa: E402

EXACT = dict(far_ratio=2.0, tet_gauss_order=4, n_theta=8, n_phi=16, near_rule=bs.BS_NEAR_EXACT)


def _op(p):
    return dict(far_ratio=p["far_ratio"], tet_order=p["tet_gauss_order"], n_theta=p["n_theta"], n_phi=p["n_phi"],
                near_rule=p.get("near_rule", 0))


@pytest.fixture(scope="module", autouse=True)
def built():
    bs.build()
    bs.load()


@pytest.fixture(scope="module")
def c1():
    m = config1_plain()
    return m, bs.Mesh(m.nodes, m.tets, m.omega)


def gpu(h, pts, precision, **p):
    cnt = torch.zeros((len(pts), 3), dtype=torch.int32, device="cuda")
    out = h.bs_velocity(torch.from_numpy(np.ascontiguousarray(pts)).cuda(), counts_dev=cnt, precision=precision, **p)
    h.bs_status()
    return out.cpu().numpy(), cnt.cpu().numpy()


@pytest.mark.parametrize("precision", ["fp64", "fp32"])
def test_plain_cube_nodes_against_oracle(orc, c1, precision):
    m, h = c1
    vo, co, stable = oracle_with_stability(orc, m, m.nodes, **_op(EXACT))
    assert np.all(co[:, 2] == 0)
    prec = bs.BS_FP64 if precision == "fp64" else bs.BS_FP32
    v, c = gpu(h, m.nodes, prec, **EXACT)
    if prec == bs.BS_FP64:
        assert rel_l2(v, vo) <= TOL_FP64_REL_L2
    else:
        assert rms_over_max(v, vo) <= TOL_FP32_RMS_MAX
    assert stable.mean() >= 0.99
    assert np.array_equal(c[stable], co[stable])


def test_off_node_points_against_oracle(orc, c1):
    """Points inside tets, on faces and on edges (the singular cases of the closed form), and outside."""
    m, h = c1
    rng = np.random.default_rng(33)
    t = m.tets[rng.choice(len(m.tets), 60, replace=False)]
    face = (m.nodes[t[:, 0]] + m.nodes[t[:, 1]] + m.nodes[t[:, 2]]) / 3
    edge = 0.3 * m.nodes[t[:, 0]] + 0.7 * m.nodes[t[:, 3]]
    pts = np.concatenate([rng.uniform(0.02, 0.98, size=(120, 3)), rng.uniform(-0.5, 1.5, size=(60, 3)), face, edge])
    vo = orc.velocity(m.nodes, m.tets, m.omega, pts, **_op(EXACT))
    v, _ = gpu(h, pts, bs.BS_FP64, **EXACT)
    assert rel_l2(v, vo) <= TOL_FP64_REL_L2
    v32, _ = gpu(h, pts, bs.BS_FP32, **EXACT)
    assert rms_over_max(v32, vo) <= TOL_FP32_RMS_MAX


def test_every_tet_exact(orc, c1):
    """far_ratio = +inf: every pair takes the exact integral (the velocity kernel, not the all-ray kernel)."""
    m, h = c1
    p = dict(EXACT, far_ratio=np.inf)
    pts = m.nodes[::5]
    vo, co = orc.velocity(m.nodes, m.tets, m.omega, pts, counts=True, **_op(p))
    v, c = gpu(h, pts, bs.BS_FP64, **p)
    assert rel_l2(v, vo) <= TOL_FP64_REL_L2
    assert np.array_equal(c, co)
    v32, _ = gpu(h, pts, bs.BS_FP32, **p)
    assert rms_over_max(v32, vo) <= TOL_FP32_RMS_MAX
    # the nodes entry point takes the same path (no mesh walk for the exact rule)
    vn = h.bs_velocity_nodes(precision=bs.BS_FP64, **p).cpu().numpy()
    h.bs_status()
    assert rel_l2(vn[::5], v) <= 1e-14


def test_ray_rule_approaches_the_exact_rule(c1):
    """The ray rule's near field at 8x16, 32x32 and 64x64 directions moves towards the exact one."""
    m, h = c1
    ve, _ = gpu(h, m.nodes, bs.BS_FP64, **EXACT)
    errs = []
    for nt, npf in ((8, 16), (32, 32), (64, 64)):
        vr, _ = gpu(h, m.nodes, bs.BS_FP64, **dict(EXACT, near_rule=bs.BS_NEAR_RAY, n_theta=nt, n_phi=npf))
        errs.append(rel_l2(vr, ve))
    assert errs[0] > errs[1] > errs[2]


def test_batch_with_the_exact_rule(orc):
    ms = config4_batch(count=6, nmin=6, nmax=12)
    hs = [bs.Mesh(m.nodes, m.tets, m.omega) for m in ms]
    batch = bs.Batch(hs)
    outs = [torch.empty((m.n_nodes, 3), dtype=torch.float64, device="cuda") for m in ms]
    batch.bs_batch_velocity(outs, precision=bs.BS_FP64, **EXACT)
    torch.cuda.synchronize()
    for m, o in zip(ms[:3], outs[:3]):
        idx = np.random.default_rng(m.n_nodes).choice(m.n_nodes, size=min(40, m.n_nodes), replace=False)
        vo = orc.velocity(m.nodes, m.tets, m.omega, m.nodes[idx], **_op(EXACT))
        assert rel_l2(o.cpu().numpy()[idx], vo) <= TOL_FP64_REL_L2


def test_ring_mesh_full_size_sampled(orc):
    """The 32^3 ring mesh, all 32768 nodes in one launch (float32); 32 seeded nodes against the oracle."""
    m = config2_ring()
    h = bs.Mesh(m.nodes, m.tets, m.omega)
    v, c = gpu(h, m.nodes, bs.BS_FP32, **EXACT)
    idx = np.random.default_rng(2012).choice(m.n_nodes, size=32, replace=False)
    vo, co = orc.velocity(m.nodes, m.tets, m.omega, m.nodes[idx], counts=True, **_op(EXACT))
    assert rms_over_max(v[idx], vo) <= TOL_FP32_RMS_MAX
    assert np.array_equal(c[idx, :2], co[:, :2]) and np.all(c[:, 2] == 0)


def test_argument_errors(c1):
    m, h = c1
    with pytest.raises(BSError) as ei:
        h.bs_velocity(torch.from_numpy(m.nodes).cuda(), precision=bs.BS_FP64, **dict(EXACT, near_rule=2))
    assert ei.value.code == BS_ERR_ARG
    with pytest.raises(BSError) as ei:
        h.bs_velocity_nodes_dderiv(precision=bs.BS_FP64, **dict(EXACT, far_ratio=np.inf))
    assert ei.value.code == BS_ERR_ARG
