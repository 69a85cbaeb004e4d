"""The bounded device waits give up, report BS_ERR_TIMEOUT, and leave the handle usable.

Every wait of the library's kernels is bounded (a failure must end a call,
never hang the GPU).  These tests make each bound run out on purpose, without
any fault: the mesh walk gets a step limit below the length of its lines, and
the velocity and all-ray kernels arm their bulk-copy barriers without issuing
the copies (so nothing is ever in flight when they give up).  Each time the
kernel returns, bs_status reports BS_ERR_TIMEOUT, and the next call with the
normal limits matches the oracle.
"""
import time

import numpy as np
import pytest
from gpu_helpers import TOL_FP32_RMS_MAX, TOL_FP64_REL_L2, rel_l2, rms_over_max

from workloads import config1_plain

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")
if not torch.cuda.is_available():
    pytest.skip("no CUDA device", allow_module_level=True)

import paper_0712_1695_gb300 as bs  # noqa: E402
from paper_0712_1695_gb300.binding import BS_ERR_ARG, BS_ERR_TIMEOUT, BSError  # noqa: E402

HYBRID = dict(far_ratio=2.0, tet_gauss_order=4, n_theta=8, n_phi=16)
ALLRAY = dict(far_ratio=float("inf"), tet_gauss_order=4, n_theta=4, n_phi=8)


@pytest.fixture(scope="module")
def c1():
    bs.build()
    m = config1_plain()
    return m, bs.Mesh(m.nodes, m.tets, m.omega)


def _oracle(orc, m, pts, p):
    return orc.velocity(m.nodes, m.tets, m.omega, pts, far_ratio=p["far_ratio"], tet_order=p["tet_gauss_order"],
                        n_theta=p["n_theta"], n_phi=p["n_phi"])


def _expect_timeout(h):
    with pytest.raises(BSError) as ei:
        h.bs_status()
    assert ei.value.code == BS_ERR_TIMEOUT


def test_walk_step_limit_gives_up(orc, c1):
    m, h = c1
    h.bs_set_wait_limits(walk_max_steps=2)  # a line through the 8^3-cell cube crosses more tets than this
    h.bs_velocity_nodes(precision=bs.BS_FP32, **ALLRAY)
    _expect_timeout(h)
    h.bs_set_wait_limits()
    v = h.bs_velocity_nodes(precision=bs.BS_FP32, **ALLRAY).cpu().numpy()
    h.bs_status()
    assert rms_over_max(v, _oracle(orc, m, m.nodes, ALLRAY)) <= TOL_FP32_RMS_MAX


@pytest.mark.parametrize("params,precision", [(HYBRID, bs.BS_FP32), (HYBRID, bs.BS_FP64), (ALLRAY, bs.BS_FP32)],
                         ids=["velocity-fp32", "velocity-fp64", "all-ray-kernel"])
def test_bulk_copy_wait_gives_up(orc, c1, params, precision):
    m, h = c1
    rng = np.random.default_rng(31)
    pts = rng.uniform(0.05, 0.95, size=(300, 3))  # off the nodes: far_ratio = inf runs the all-ray kernel
    dev = torch.from_numpy(pts).cuda()
    h.bs_set_wait_limits(copy_wait_polls=1 << 12, withhold_copies=True)
    t0 = time.perf_counter()
    h.bs_velocity(dev, precision=precision, **params)
    _expect_timeout(h)
    elapsed = time.perf_counter() - t0
    assert elapsed < 30.0  # bounded: every CTA gives up after its poll limit
    h.bs_set_wait_limits()
    v = h.bs_velocity(dev, precision=precision, **params).cpu().numpy()
    h.bs_status()
    vo = _oracle(orc, m, pts, params)
    if precision == bs.BS_FP64:
        assert rel_l2(v, vo) <= TOL_FP64_REL_L2
    else:
        assert rms_over_max(v, vo) <= TOL_FP32_RMS_MAX


def test_wait_limit_arguments(c1):
    _, h = c1
    for bad in (dict(walk_max_steps=-1), dict(copy_wait_polls=-5)):
        with pytest.raises(BSError) as ei:
            h.bs_set_wait_limits(**bad)
        assert ei.value.code == BS_ERR_ARG
    h.bs_set_wait_limits()


def test_batch_copy_wait_gives_up(orc, c1):
    """The batched far kernel follows its first mesh's wait limits: with the copies withheld every CTA gives up,
    bs_batch_status reports BS_ERR_TIMEOUT, and the next launch with the normal limits matches the oracle."""
    from workloads import config5_rings

    m, h = c1
    m2 = config5_rings(10)
    h2 = bs.Mesh(m2.nodes, m2.tets, m2.omega)
    batch = bs.Batch([h, h2])
    outs = [torch.empty((mm.n_nodes, 3), dtype=torch.float64, device="cuda") for mm in (m, m2)]
    h.bs_set_wait_limits(copy_wait_polls=1 << 12, withhold_copies=True)
    try:
        t0 = time.perf_counter()
        batch.bs_batch_velocity(outs, precision=bs.BS_FP32, **HYBRID)
        with pytest.raises(BSError) as ei:
            batch.bs_batch_status()
        assert ei.value.code == BS_ERR_TIMEOUT
        assert time.perf_counter() - t0 < 30.0
    finally:
        h.bs_set_wait_limits()
    batch.bs_batch_velocity(outs, precision=bs.BS_FP32, **HYBRID)
    batch.bs_batch_status()
    for mm, o in zip((m, m2), outs):
        assert rms_over_max(o.cpu().numpy(), _oracle(orc, mm, mm.nodes, HYBRID)) <= TOL_FP32_RMS_MAX
