"""Every kernel variant the library can select, against the FP64 oracle.

The velocity kernel is compiled in many launch shapes per (precision, tet
rule, near rule); bs_autotune, the tuning cache and BS_VARIANT can hand any of
them to a user, so each one is pinned in turn (bs_set_variant) and compared
with the oracle: float64 at relative L2 <= 1e-12, float32 at RMS over max
speed <= 1e-5, near/far counts bit-exact on points whose counts survive
perturbed thresholds (the counts do not depend on the far rule, so the
stability mask is computed once).  The mesh is the 16^3 two-ring grid (20250
tets: every tile size of the table, 8 to 64 tets, leaves a ragged last tile)
and the points are its 4096 nodes (pairs with the point on a tet vertex) plus
512 points off the nodes (inside tets, outside the mesh, on edges), so that
point blocks are ragged too.
"""
import numpy as np
import pytest
from gpu_helpers import TOL_FP32_RMS_MAX, TOL_FP64_REL_L2, oracle_with_stability, rel_l2, rms_over_max

from workloads import config5_rings

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")
if not torch.cuda.is_available():
    pytest.skip("no CUDA device", allow_module_level=True)

import paper_0712_1695_gb300 as bs  # noqa: E402

bs.build()
PARAMS = dict(far_ratio=2.0, n_theta=8, n_phi=16)
CASES = [(prec, q, nr, v)
         for nr in (bs.BS_NEAR_RAY, bs.BS_NEAR_EXACT)
         for prec in (bs.BS_FP32, bs.BS_FP64)
         for q in (1, 4, 8, 27, 64)
         for v in range(bs.bs_num_variants(prec, q, nr))]


def _id(c):
    prec, q, nr, v = c
    s = bs.bs_variant_shape(prec, q, nr, v)
    return (f"{'fp32' if prec == bs.BS_FP32 else 'fp64'}-q{q}-{'exact' if nr else 'ray'}-v{v}-P{s['points_per_thread']}"
            f"T{s['tile']}S{s['stages']}B{s['ctas_per_sm']}D{s['near_drain']}U{s['ray_bundle']}"
            f"{'pp' if s['point_pairs'] else 'qp'}J{s['tet_unroll']}")


@pytest.fixture(scope="module")
def case(orc):
    m = config5_rings(16)
    rng = np.random.default_rng(16)
    tets = m.tets[rng.choice(m.n_tets, size=96, replace=False)]
    off = np.concatenate([rng.uniform(-1.4, 1.4, size=(320, 3)),  # inside tets
                          rng.uniform(-2.0, 2.0, size=(96, 3)),  # partly outside the mesh
                          0.5 * (m.nodes[tets[:, 0]] + m.nodes[tets[:, 1]])])  # edge midpoints
    pts = np.concatenate([m.nodes, off])
    assert len(pts) == 4096 + 512
    # counts and their stability do not depend on the far rule or the near rule's arithmetic
    _, counts, stable = oracle_with_stability(orc, m, pts, rel=1e-5, tet_order=4, **PARAMS)
    # the nodes: at least 99% stable; edge midpoints sit on hit thresholds by construction
    assert stable[:4096].mean() >= 0.99
    h = bs.Mesh(m.nodes, m.tets, m.omega)
    return m, h, pts, torch.from_numpy(pts).cuda(), counts, stable, {}


def _oracle(orc, case, q, nr):
    m, _, pts, _, _, _, memo = case
    if (q, nr) not in memo:
        memo[(q, nr)] = orc.velocity(m.nodes, m.tets, m.omega, pts, tet_order=q, near_rule=nr, **PARAMS)
    return memo[(q, nr)]


@pytest.mark.parametrize("prec,q,nr,variant", CASES, ids=[_id(c) for c in CASES])
def test_variant_matches_oracle(orc, case, prec, q, nr, variant):
    m, h, pts, dev, co, stable, _ = case
    vo = _oracle(orc, case, q, nr)
    cnt = torch.full((len(pts), 3), -1, dtype=torch.int32, device="cuda")
    h.bs_set_variant(prec, q, nr, variant)
    try:
        v = h.bs_velocity(dev, counts_dev=cnt, precision=prec, tet_gauss_order=q, near_rule=nr, **PARAMS)
        h.bs_status()
    finally:
        h.bs_set_variant(prec, q, nr, -1)
    v = v.cpu().numpy()
    c = cnt.cpu().numpy()
    if prec == bs.BS_FP64:
        assert rel_l2(v, vo) <= TOL_FP64_REL_L2
    else:
        assert rms_over_max(v, vo) <= TOL_FP32_RMS_MAX
    assert np.array_equal(c[stable, :2], co[stable, :2])
    assert np.all(c[:, 0] + c[:, 1] == m.n_tets)
    if nr == bs.BS_NEAR_RAY:
        if prec == bs.BS_FP64:
            assert np.array_equal(c[stable, 2], co[stable, 2])
        else:  # float32 may flip a line that grazes an edge; a handful per thousand
            assert np.abs(c[:, 2] - co[:, 2]).sum() <= 1e-3 * co[:, 2].sum()
    else:
        assert np.all(c[:, 2] == 0)  # the exact rule counts no ray hits


def test_variant_api_rejects_bad_arguments(case):
    _, h, *_ = case
    n = bs.bs_num_variants(bs.BS_FP32, 4)
    with pytest.raises(bs.BSError):
        h.bs_set_variant(bs.BS_FP32, 4, bs.BS_NEAR_RAY, n)
    with pytest.raises(bs.BSError):
        bs.bs_variant_shape(bs.BS_FP32, 5, bs.BS_NEAR_RAY, 0)
    h.bs_set_variant(bs.BS_FP32, 4, bs.BS_NEAR_RAY, -1)
