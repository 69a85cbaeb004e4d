"""The all-ray kernel (far_ratio = +inf: the ray rule of Section 2 for every pair) through the C ABI.

Every pair takes the ray rule; the kernel visits, per pair, only the rings of
directions whose polar angle can bring the line within the tet's bounding
sphere.  It must match the CPU oracle (float64: relative L2 <= 1e-12, counts
bit-exact on stable points; float32: RMS error over max speed <= 1e-5), and it
must find exactly the line hits of the dense loop over all directions (the
velocity kernel's all-ray path, BS_ALLRAY_GENERIC=1), which shows that the
direction window drops no line: one tet seen from every direction (poles, the
theta = 0 / pi seam) and every distance.
"""
import os

import numpy as np
import pytest
from gpu_helpers import TOL_FP32_RMS_MAX, TOL_FP64_REL_L2, oracle_with_stability, rel_l2, rms_over_max

from workloads import config1_plain, config2_ring

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")
if not torch.cuda.is_available():
    pytest.skip("no CUDA device", allow_module_level=True)

import paper_0712_1695_gb300 as bs  # noqa: E402

ALLRAY = dict(far_ratio=np.inf, tet_gauss_order=4, n_theta=8, n_phi=16)


def _op(p):
    return dict(far_ratio=p["far_ratio"], tet_order=p["tet_gauss_order"], n_theta=p["n_theta"], n_phi=p["n_phi"])


@pytest.fixture(scope="module", autouse=True)
def built():
    bs.build()
    bs.load()


def gpu_velocity(handle, pts, precision, generic=False, **p):
    dev = torch.from_numpy(np.ascontiguousarray(pts)).cuda()
    cnt = torch.zeros((len(pts), 3), dtype=torch.int32, device="cuda")
    old = os.environ.get("BS_ALLRAY_GENERIC")
    os.environ["BS_ALLRAY_GENERIC"] = "1" if generic else "0"
    try:
        out = handle.bs_velocity(dev, counts_dev=cnt, precision=precision, **p)
        handle.bs_status()
    finally:
        if old is None:
            del os.environ["BS_ALLRAY_GENERIC"]
        else:
            os.environ["BS_ALLRAY_GENERIC"] = old
    return out.cpu().numpy(), cnt.cpu().numpy()


@pytest.fixture(scope="module")
def c1():
    m = config1_plain()
    return m, bs.Mesh(m.nodes, m.tets, m.omega)


@pytest.mark.parametrize("precision", ["fp64", "fp32"])
def test_plain_cube_all_nodes_against_oracle(orc, c1, precision):
    m, h = c1
    vo, co, stable = oracle_with_stability(orc, m, m.nodes, rel=1e-5, **_op(ALLRAY))
    if precision == "fp64":
        v, c = gpu_velocity(h, m.nodes, bs.BS_FP64, **ALLRAY)
        assert rel_l2(v, vo) <= TOL_FP64_REL_L2
        assert stable.mean() >= 0.99
        assert np.array_equal(c[stable], co[stable])
    else:
        v, c = gpu_velocity(h, m.nodes, bs.BS_FP32, **ALLRAY)
        assert rms_over_max(v, vo) <= TOL_FP32_RMS_MAX
        assert np.array_equal(c[:, :2], co[:, :2])  # every pair near, none far
        assert np.abs(c[:, 2] - co[:, 2]).sum() <= 1e-3 * co[:, 2].sum()


def test_off_node_points_against_oracle(orc, c1):
    """Points inside tets, on edges and outside the mesh (the float64 steps of the float32 path)."""
    m, h = c1
    rng = np.random.default_rng(21)
    pts = np.concatenate([rng.uniform(0.02, 0.98, size=(150, 3)), rng.uniform(-0.5, 1.5, size=(100, 3)),
                          0.5 * (m.nodes[m.tets[:40, 0]] + m.nodes[m.tets[:40, 2]])])
    vo, co, stable = oracle_with_stability(orc, m, pts, **_op(ALLRAY))
    v, c = gpu_velocity(h, pts, bs.BS_FP64, **ALLRAY)
    assert rel_l2(v, vo) <= TOL_FP64_REL_L2
    assert np.array_equal(c[stable], co[stable])
    v32, _ = gpu_velocity(h, pts, bs.BS_FP32, **ALLRAY)
    assert rms_over_max(v32, vo) <= TOL_FP32_RMS_MAX


def _sphere_directions(n):
    """Fibonacci directions plus the poles and directions in the y = 0 plane (the theta seam)."""
    i = np.arange(n) + 0.5
    phi = np.arccos(1 - 2 * i / n)
    th = np.pi * (1 + 5 ** 0.5) * i
    d = np.stack([np.sin(phi) * np.cos(th), np.sin(phi) * np.sin(th), np.cos(phi)], axis=1)
    a = np.linspace(0, 2 * np.pi, 24, endpoint=False)
    seam = np.stack([np.cos(a), np.zeros_like(a), np.sin(a)], axis=1)
    poles = np.array([[0, 0, 1.0], [0, 0, -1.0], [1e-7, 0, 1.0], [0, -1e-7, -1.0]])
    d = np.concatenate([d, seam, poles])
    return d / np.linalg.norm(d, axis=1, keepdims=True)


@pytest.mark.parametrize("n_phi,n_theta", [(16, 8), (64, 32), (7, 5)])
def test_window_keeps_every_line_of_the_dense_loop(orc, n_phi, n_theta):
    """One tet, seen from every direction at distances 0.3 to 5000 tet sizes: the ray kernel's line hits
    equal the dense loop's exactly (float64), and both match the oracle."""
    nodes = np.array([[0.0, 0.0, 0.0], [0.011, 0.001, -0.002], [0.002, 0.012, 0.001], [0.001, -0.001, 0.013]])
    nodes += np.array([0.3, -0.2, 0.1])
    tets = np.array([[0, 1, 2, 3]], dtype=np.int32)
    omega = np.array([[0.0, 0.0, 1.0], [0.2, -0.1, 1.0], [-0.3, 0.1, 0.7], [0.1, 0.4, 1.2]])
    c = nodes.mean(axis=0)
    d = _sphere_directions(400)
    dist = np.geomspace(0.004, 60.0, 9)
    pts = (c + d[:, None, :] * dist[None, :, None]).reshape(-1, 3)
    h = bs.Mesh(nodes, tets, omega)
    p = dict(far_ratio=np.inf, tet_gauss_order=4, n_theta=n_theta, n_phi=n_phi)
    v, cnt = gpu_velocity(h, pts, bs.BS_FP64, **p)
    vg, cntg = gpu_velocity(h, pts, bs.BS_FP64, generic=True, **p)
    assert np.array_equal(cnt, cntg)
    assert cnt[:, 2].sum() > 0
    assert rel_l2(v, vg) <= 1e-13
    vo, co = orc.velocity(nodes, tets, omega, pts, counts=True, **_op(p))
    assert rel_l2(v, vo) <= TOL_FP64_REL_L2
    # float32: the same hits as the float32 dense loop on all but a handful of grazing lines
    v32, c32 = gpu_velocity(h, pts, bs.BS_FP32, **p)
    v32g, c32g = gpu_velocity(h, pts, bs.BS_FP32, generic=True, **p)
    assert np.abs(c32[:, 2] - c32g[:, 2]).sum() <= max(2, 1e-3 * c32g[:, 2].sum())
    assert rms_over_max(v32, vo) <= TOL_FP32_RMS_MAX


def test_matches_dense_loop_on_plain_cube(c1):
    m, h = c1
    for prec, tol in ((bs.BS_FP64, 1e-13), (bs.BS_FP32, 2e-6)):
        v, c = gpu_velocity(h, m.nodes, prec, **ALLRAY)
        vg, cg = gpu_velocity(h, m.nodes, prec, generic=True, **ALLRAY)
        if prec == bs.BS_FP64:
            assert np.array_equal(c, cg) and rel_l2(v, vg) <= tol
        else:
            assert np.array_equal(c[:, :2], cg[:, :2]) and rms_over_max(v, vg) <= tol


def test_ring_mesh_full_size_sampled_against_oracle(orc):
    """The 32^3 Gaussian-ring mesh, all 32768 nodes in one launch; 48 seeded nodes against the oracle."""
    m = config2_ring()
    h = bs.Mesh(m.nodes, m.tets, m.omega)
    v, c = gpu_velocity(h, m.nodes, bs.BS_FP32, **ALLRAY)
    idx = np.random.default_rng(2002).choice(m.n_nodes, size=48, replace=False)
    vo, co = orc.velocity(m.nodes, m.tets, m.omega, m.nodes[idx], counts=True, **_op(ALLRAY))
    assert rms_over_max(v[idx], vo) <= TOL_FP32_RMS_MAX
    assert np.array_equal(c[idx, :2], co[:, :2])
    v64, _ = gpu_velocity(h, m.nodes[idx], bs.BS_FP64, **ALLRAY)
    assert rel_l2(v64, vo) <= TOL_FP64_REL_L2


def test_direction_tables_beyond_shared_memory_use_the_dense_path(orc):
    """n_phi * n_theta > 4096: the call goes to the velocity kernel's all-ray path and still matches."""
    m = config1_plain()
    tets = m.tets[:40]
    h = bs.Mesh(m.nodes, tets, m.omega)
    pts = m.nodes[::37]
    p = dict(far_ratio=np.inf, tet_gauss_order=4, n_theta=64, n_phi=80)
    v, c = gpu_velocity(h, pts, bs.BS_FP64, **p)
    vo, co = orc.velocity(m.nodes, tets, m.omega, pts, counts=True, **_op(p))
    assert rel_l2(v, vo) <= TOL_FP64_REL_L2
    assert np.array_equal(c[:, :2], co[:, :2])
