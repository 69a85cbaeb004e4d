"""CUDA path (through the C ABI) against the FP64 CPU oracle, element by element.

float64 path: relative L2 <= 1e-12 and counts bit-exact on points whose
counts are stable under perturbed thresholds.  float32 path: RMS error over
the largest speed <= 1e-5 and near/far counts bit-exact on stable points.
Sizes span many tiles and point blocks with ragged tails; the 64^3 workload
runs at full size in the launch configuration the benchmark times and is
checked on sampled nodes.
"""
import numpy as np
import pytest
from gpu_helpers import TOL_FP32_RMS_MAX, TOL_FP64_REL_L2, oracle_with_stability, rel_l2, rms_over_max

from workloads import config1_plain, config2_ring, config3_fourier, config3_samples

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")
if not torch.cuda.is_available():
    pytest.skip("no CUDA device", allow_module_level=True)

import paper_0712_1695_gb300 as bs  # noqa: E402
from paper_0712_1695_gb300.binding import BS_ERR_ARG, BS_ERR_MESH, BS_ERR_ORDER, BSError  # noqa: E402

DEFAULT = dict(far_ratio=2.0, tet_gauss_order=4, n_theta=8, n_phi=16)


def _oracle_params(p):
    return dict(far_ratio=p["far_ratio"], tet_order=p["tet_gauss_order"], n_theta=p["n_theta"], n_phi=p["n_phi"])


@pytest.fixture(scope="module", autouse=True)
def built():
    bs.build()
    bs.load()


@pytest.fixture(scope="module")
def c1():
    m = config1_plain()
    return m, bs.Mesh(m.nodes, m.tets, m.omega)


def gpu_velocity(handle, pts, precision, counts=False, **p):
    dev = torch.from_numpy(np.ascontiguousarray(pts)).cuda()
    cnt = torch.zeros((len(pts), 3), dtype=torch.int32, device="cuda") if counts else None
    out = handle.bs_velocity(dev, counts_dev=cnt, precision=precision, **p)
    handle.bs_status()
    return out.cpu().numpy(), (cnt.cpu().numpy() if counts else None)


# ---------------------------------------------------------------- tables
@pytest.mark.parametrize("n_phi,n_theta", [(16, 8), (4, 4), (64, 64), (1, 3), (256, 255)])
def test_direction_table_matches_oracle(orc, n_phi, n_theta):
    s, k = bs.bs_direction_table(n_phi, n_theta)
    so, ko = orc.directions(n_phi, n_theta)
    assert np.abs(s - so).max() < 4e-15 and np.abs(k - ko).max() < 1e-16


@pytest.mark.parametrize("order", [1, 4, 8, 27, 64])
def test_tet_rule_matches_oracle(orc, order):
    b, w = bs.bs_tet_rule(order)
    bo, wo = orc.tet_rule(order)
    # the same set of points (the two sides enumerate the conical product in different orders)
    i = np.lexsort(np.round(b, 12).T[::-1])
    io = np.lexsort(np.round(bo, 12).T[::-1])
    assert np.abs(b[i] - bo[io]).max() < 5e-15 and np.abs(w[i] - wo[io]).max() < 5e-15


# ---------------------------------------------------------------- plain cube, all nodes
@pytest.mark.parametrize("params", [
    DEFAULT,
    dict(DEFAULT, far_ratio=np.inf, n_theta=4, n_phi=4),
    dict(DEFAULT, far_ratio=3.0, tet_gauss_order=1),
    dict(DEFAULT, far_ratio=2.5, tet_gauss_order=8, n_theta=6, n_phi=10),
    dict(DEFAULT, tet_gauss_order=27, n_theta=16, n_phi=16),
    dict(DEFAULT, tet_gauss_order=64, n_theta=3, n_phi=5),
], ids=["default", "all-ray-4x4", "q1", "q8", "q27", "q64-odd-orders"])
def test_plain_cube_fp64(orc, c1, params):
    m, h = c1
    vo, co, stable = oracle_with_stability(orc, m, m.nodes, **_oracle_params(params))
    v, c = gpu_velocity(h, m.nodes, bs.BS_FP64, counts=True, **params)
    assert rel_l2(v, vo) <= TOL_FP64_REL_L2
    # odd orders put theta or phi at pi/2: lines then lie in the axis-aligned boundary faces and the
    # hit decisions sit exactly on a threshold (unstable by construction); even orders avoid that
    if params["n_theta"] % 2 == 0 and params["n_phi"] % 2 == 0:
        assert stable.mean() >= 0.99
    assert np.array_equal(c[stable], co[stable])


@pytest.mark.parametrize("params", [DEFAULT, dict(DEFAULT, far_ratio=np.inf, n_theta=4, n_phi=4),
                                    dict(DEFAULT, tet_gauss_order=8)], ids=["default", "all-ray-4x4", "q8"])
def test_plain_cube_fp32(orc, c1, params):
    m, h = c1
    vo, co, stable = oracle_with_stability(orc, m, m.nodes, rel=1e-5, **_oracle_params(params))
    v, c = gpu_velocity(h, m.nodes, bs.BS_FP32, counts=True, **params)
    assert rms_over_max(v, vo) <= TOL_FP32_RMS_MAX
    assert np.array_equal(c[stable, :2], co[stable, :2])
    # ray hits: float32 may flip a line that grazes an edge; allow a handful per thousand
    assert np.abs(c[:, 2] - co[:, 2]).sum() <= 1e-3 * co[:, 2].sum()


def test_off_node_points_fp64_and_fp32(orc, c1):
    """Points inside tets (chords straddling R = 0), on the boundary and outside the mesh."""
    m, h = c1
    rng = np.random.default_rng(12)
    pts = np.concatenate([rng.uniform(0.02, 0.98, size=(300, 3)), rng.uniform(-0.5, 1.5, size=(200, 3)),
                          0.5 * (m.nodes[m.tets[:50, 0]] + m.nodes[m.tets[:50, 1]])])  # edge midpoints
    p = DEFAULT
    vo, co, stable = oracle_with_stability(orc, m, pts, **_oracle_params(p))
    v, c = gpu_velocity(h, pts, bs.BS_FP64, counts=True, **p)
    assert rel_l2(v, vo) <= TOL_FP64_REL_L2
    assert np.array_equal(c[stable], co[stable])
    v32, _ = gpu_velocity(h, pts, bs.BS_FP32, **p)
    assert rms_over_max(v32, vo) <= TOL_FP32_RMS_MAX


@pytest.mark.parametrize("k", [1, 2, 31, 255, 256, 257, 513])
def test_ragged_point_counts(orc, c1, k):
    m, h = c1
    rng = np.random.default_rng(k)
    pts = m.nodes[rng.choice(m.n_nodes, size=k, replace=k > m.n_nodes)]
    vo = orc.velocity(m.nodes, m.tets, m.omega, pts, **_oracle_params(DEFAULT))
    v, _ = gpu_velocity(h, pts, bs.BS_FP64, **DEFAULT)
    assert rel_l2(v, vo) <= TOL_FP64_REL_L2


@pytest.mark.parametrize("n_tets", [1, 5, 63, 64, 65, 200])
def test_ragged_tet_counts(orc, n_tets):
    m = config1_plain()
    tets = m.tets[:n_tets]
    h = bs.Mesh(m.nodes, tets, m.omega)
    pts = m.nodes[::7]
    for prec in (bs.BS_FP64, bs.BS_FP32):
        vo, co = orc.velocity(m.nodes, tets, m.omega, pts, counts=True, **_oracle_params(DEFAULT))
        v, c = gpu_velocity(h, pts, prec, counts=True, **DEFAULT)
        if prec == bs.BS_FP64:
            assert rel_l2(v, vo) <= TOL_FP64_REL_L2
        else:
            assert rms_over_max(v, vo) <= TOL_FP32_RMS_MAX
        assert np.array_equal(c[:, :2], co[:, :2])


def test_empty_inputs(c1):
    m, h = c1
    # no points: a no-op
    out = torch.full((0, 3), 7.0, dtype=torch.float64, device="cuda")
    h.bs_velocity(torch.zeros((0, 3), dtype=torch.float64, device="cuda"), out_dev=out, **DEFAULT)
    # no tets: zero velocity
    e = bs.Mesh(m.nodes, np.zeros((0, 4), dtype=np.int32), m.omega)
    v, c = gpu_velocity(e, m.nodes[:10], bs.BS_FP32, counts=True, **DEFAULT)
    assert np.all(v == 0) and np.all(c == 0)


def test_deterministic_and_host_path(c1):
    m, h = c1
    a, _ = gpu_velocity(h, m.nodes, bs.BS_FP32, **DEFAULT)
    b, _ = gpu_velocity(h, m.nodes, bs.BS_FP32, **DEFAULT)
    assert np.array_equal(a, b)
    c = h.bs_velocity_host(m.nodes, precision=bs.BS_FP32, **DEFAULT)
    assert np.array_equal(a, c)


def test_update_matches_fresh_mesh(orc):
    m = config1_plain()
    h = bs.Mesh(m.nodes, m.tets, m.omega)
    rng = np.random.default_rng(5)
    nodes2 = m.nodes + 0.01 * rng.standard_normal(m.nodes.shape) * (1.0 / 8)
    omega2 = m.omega[::-1].copy()
    h.bs_update(torch.from_numpy(nodes2).cuda(), torch.from_numpy(omega2).cuda())
    h.bs_status()
    v, _ = gpu_velocity(h, nodes2, bs.BS_FP64, **DEFAULT)
    vo = orc.velocity(nodes2, m.tets, omega2, nodes2, **_oracle_params(DEFAULT))
    assert rel_l2(v, vo) <= TOL_FP64_REL_L2


def test_argument_and_mesh_errors(c1):
    m, h = c1
    pts = torch.from_numpy(m.nodes[:4].copy()).cuda()
    for bad, code in [(dict(DEFAULT, far_ratio=1.5), BS_ERR_ARG), (dict(DEFAULT, n_theta=0), BS_ERR_ARG),
                      (dict(DEFAULT, n_phi=300), BS_ERR_ARG), (dict(DEFAULT, tet_gauss_order=5), BS_ERR_ORDER),
                      (dict(DEFAULT, far_ratio=float("nan")), BS_ERR_ARG)]:
        with pytest.raises(BSError) as ei:
            h.bs_velocity(pts, **bad)
        assert ei.value.code == code
    bad_tets = m.tets.copy()
    bad_tets[17, 2] = m.n_nodes + 3
    with pytest.raises(BSError) as ei:
        bs.Mesh(m.nodes, bad_tets, m.omega)
    assert ei.value.code == BS_ERR_MESH and "tet 17" in str(ei.value)
    flat = m.tets.copy()
    flat[9] = [flat[9, 0], flat[9, 1], flat[9, 1], flat[9, 2]]
    with pytest.raises(BSError) as ei:
        bs.Mesh(m.nodes, flat, m.omega)
    assert ei.value.code == BS_ERR_MESH and "tet 9" in str(ei.value)


# ---------------------------------------------------------------- larger workloads
def test_gaussian_ring_sampled(orc):
    m = config2_ring()
    h = bs.Mesh(m.nodes, m.tets, m.omega)
    dev = torch.from_numpy(m.nodes).cuda()
    v64 = h.bs_velocity(dev, precision=bs.BS_FP64, **DEFAULT).cpu().numpy()
    v32 = h.bs_velocity(dev, precision=bs.BS_FP32, **DEFAULT).cpu().numpy()
    h.bs_status()
    idx = np.random.default_rng(2002).choice(m.n_nodes, size=1024, replace=False)
    vo, co, stable = oracle_with_stability(orc, m, m.nodes[idx], **_oracle_params(DEFAULT))
    assert rel_l2(v64[idx], vo) <= TOL_FP64_REL_L2
    assert rms_over_max(v32[idx], vo) <= TOL_FP32_RMS_MAX
    # the whole float32 field against the whole float64 field
    assert rms_over_max(v32, v64) <= TOL_FP32_RMS_MAX


@pytest.mark.slow
def test_fourier_64_full_size_sampled(orc):
    """The benchmark's workload at full size (float32, bench launch configuration), sampled nodes vs oracle."""
    m = config3_fourier()
    h = bs.Mesh(m.nodes, m.tets, m.omega)
    dev = torch.from_numpy(m.nodes).cuda()
    cnt = torch.zeros((m.n_nodes, 3), dtype=torch.int32, device="cuda")
    v32 = h.bs_velocity(dev, counts_dev=cnt, precision=bs.BS_FP32, **DEFAULT).cpu().numpy()
    h.bs_status()
    c = cnt.cpu().numpy()
    assert np.all(c[:, 0] + c[:, 1] == m.n_tets)
    idx = config3_samples(m.n_nodes, 4096)[::16]  # 256 of the 4096 seeded samples
    vo, co, stable = oracle_with_stability(orc, m, m.nodes[idx], rel=1e-5, **_oracle_params(DEFAULT))
    assert rms_over_max(v32[idx], vo) <= TOL_FP32_RMS_MAX
    assert np.array_equal(c[idx][stable, :2], co[stable, :2])
    # float64 path on the same sampled nodes
    v64 = h.bs_velocity(torch.from_numpy(m.nodes[idx].copy()).cuda(), precision=bs.BS_FP64, **DEFAULT).cpu().numpy()
    assert rel_l2(v64, vo) <= TOL_FP64_REL_L2


def test_point_order_does_not_change_results(c1):
    """Points are visited in a spatial order; each point's result must not depend on it (bitwise)."""
    m, h = c1
    rng = np.random.default_rng(99)
    pts = np.concatenate([m.nodes, rng.uniform(0, 1, size=(300, 3))])
    perm = rng.permutation(len(pts))
    for prec in (bs.BS_FP32, bs.BS_FP64):
        a, _ = gpu_velocity(h, pts, prec, **DEFAULT)
        b, _ = gpu_velocity(h, pts[perm], prec, **DEFAULT)
        assert np.array_equal(a[perm], b)
