"""Batched evaluation of many uneven meshes in one persistent launch (and its CUDA graph), and the autotuner.

The batch must give each mesh the velocity the single-mesh path gives it
(float64: relative L2 <= 1e-12; float32: RMS over max speed <= 1e-5), keep
doing so when the captured graph is replayed, and pick up a mesh that
bs_update changed in between.  Sampled nodes of two meshes are also checked
against the CPU oracle directly.
"""
import numpy as np
import pytest
from gpu_helpers import TOL_FP32_RMS_MAX, TOL_FP64_REL_L2, rel_l2, rms_over_max

from workloads import config4_batch

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")
if not torch.cuda.is_available():
    pytest.skip("no CUDA device", allow_module_level=True)

import paper_0712_1695_gb300 as bs  # noqa: E402

P = dict(far_ratio=2.0, tet_gauss_order=4, n_theta=8, n_phi=16)


@pytest.fixture(scope="module")
def meshes():
    bs.build()
    ms = config4_batch(count=10, nmin=6, nmax=14)
    return ms, [bs.Mesh(m.nodes, m.tets, m.omega) for m in ms]


def _single(h, m, prec):
    out = h.bs_velocity(torch.from_numpy(m.nodes).cuda(), precision=prec, **P)
    h.bs_status()
    return out.cpu().numpy()


@pytest.mark.parametrize("prec", [bs.BS_FP64, bs.BS_FP32], ids=["fp64", "fp32"])
def test_batch_matches_single_mesh_path(meshes, prec):
    """The batch on a stream of its own, waited for with that stream's synchronize alone: the meshes' near walks
    run on the batch's side streams, so this also checks that they are joined back into the caller's stream."""
    ms, hs = meshes
    batch = bs.Batch(hs)
    stream = torch.cuda.Stream()
    outs = [torch.full((m.n_nodes, 3), float("nan"), dtype=torch.float64, device="cuda") for m in ms]
    with torch.cuda.stream(stream):
        batch.bs_batch_velocity(outs, stream=stream, precision=prec, **P)
    stream.synchronize()
    first = [o.cpu().numpy() for o in outs]
    for m, h, v in zip(ms, hs, first):
        ref = _single(h, m, prec)
        if prec == bs.BS_FP64:
            assert rel_l2(v, ref) <= TOL_FP64_REL_L2
        else:
            assert rms_over_max(v, ref) <= TOL_FP32_RMS_MAX
    # replay (graph) gives the same bits
    for o in outs:
        o.fill_(float("nan"))
    with torch.cuda.stream(stream):
        batch.bs_batch_velocity(outs, stream=stream, precision=prec, **P)
    stream.synchronize()
    for a, o in zip(first, outs):
        assert np.array_equal(a, o.cpu().numpy())


def _placements(prec):
    """A variant that leaves the near pairs to the near pass and one that drains them in the far kernel."""
    n = bs.bs_num_variants(prec, 4)
    drain = [bs.bs_variant_shape(prec, 4, bs.BS_NEAR_RAY, v)["near_drain"] for v in range(n)]
    return [drain.index(3), next(v for v in range(n) if drain[v] != 3)]


PLACEMENTS = [(prec, v, graph) for prec in (bs.BS_FP64, bs.BS_FP32) for v in _placements(prec)
              for graph in (True, False)]


@pytest.mark.parametrize("prec,variant,graph", PLACEMENTS,
                         ids=[f"{'fp64' if p == bs.BS_FP64 else 'fp32'}-v{v}-{'graph' if g else 'direct'}"
                              for p, v, g in PLACEMENTS])
def test_batch_near_placements_match_the_single_path(meshes, prec, variant, graph):
    """The batch with its near pairs left out of the far kernel (the meshes' walks, or the near pass), or drained in
    the far kernel, as a replayed CUDA graph (a side stream) or launched directly (the legacy default stream)."""
    ms, hs = meshes
    refs = [_single(h, m, prec) for m, h in zip(ms, hs)]
    hs[0].bs_set_variant(prec, 4, bs.BS_NEAR_RAY, variant)  # a batch runs its first mesh's pinned variant
    try:
        batch = bs.Batch(hs)
        outs = [torch.full((m.n_nodes, 3), float("nan"), dtype=torch.float64, device="cuda") for m in ms]
        if graph:
            stream = torch.cuda.Stream()
            for _ in range(2):  # capture, then replay
                with torch.cuda.stream(stream):
                    batch.bs_batch_velocity(outs, stream=stream, precision=prec, **P)
            stream.synchronize()
        else:
            batch.bs_batch_velocity(outs, stream=0, precision=prec, **P)
            torch.cuda.synchronize()
    finally:
        hs[0].bs_set_variant(prec, 4, bs.BS_NEAR_RAY, -1)
    for i, (v, ref) in enumerate(zip(outs, refs)):
        v = v.cpu().numpy()
        if prec == bs.BS_FP64:
            assert rel_l2(v, ref) <= TOL_FP64_REL_L2, f"mesh {i}"
        else:
            assert rms_over_max(v, ref) <= TOL_FP32_RMS_MAX, f"mesh {i}"


@pytest.mark.parametrize("prec", [bs.BS_FP64, bs.BS_FP32], ids=["fp64", "fp32"])
def test_batch_near_walk_equals_near_pass(meshes, prec, monkeypatch):
    """At the meshes' nodes the batch's near field comes from each mesh's walk; with the walk switched off
    (BS_WALK=0) from the near pass over every mesh's points: the same rule, equal to rounding."""
    ms, hs = meshes
    v3 = _placements(prec)[0]
    res = []
    for walk in ("1", "0"):
        monkeypatch.setenv("BS_WALK", walk)
        hs[0].bs_set_variant(prec, 4, bs.BS_NEAR_RAY, v3)
        try:
            batch = bs.Batch(hs)
            outs = [torch.full((m.n_nodes, 3), float("nan"), dtype=torch.float64, device="cuda") for m in ms]
            stream = torch.cuda.Stream()
            with torch.cuda.stream(stream):
                batch.bs_batch_velocity(outs, stream=stream, precision=prec, **P)
            stream.synchronize()
        finally:
            hs[0].bs_set_variant(prec, 4, bs.BS_NEAR_RAY, -1)
        res.append([o.cpu().numpy() for o in outs])
    for i, (a, b) in enumerate(zip(*res)):
        if prec == bs.BS_FP64:
            assert rel_l2(a, b) <= TOL_FP64_REL_L2, f"mesh {i}"
        else:
            assert rms_over_max(a, b) <= TOL_FP32_RMS_MAX, f"mesh {i}"
    for h in hs:
        h.bs_status()


def test_batch_against_oracle_and_after_update(orc, meshes):
    ms, hs = meshes
    batch = bs.Batch(hs)
    stream = torch.cuda.Stream()
    outs = [torch.empty((m.n_nodes, 3), dtype=torch.float64, device="cuda") for m in ms]
    with torch.cuda.stream(stream):
        batch.bs_batch_velocity(outs, stream=stream, precision=bs.BS_FP64, **P)
    stream.synchronize()
    for i in (0, 3):
        m = ms[i]
        idx = np.random.default_rng(i).choice(m.n_nodes, size=min(200, m.n_nodes), replace=False)
        ref = orc.velocity(m.nodes, m.tets, m.omega, m.nodes[idx], far_ratio=2.0, tet_order=4, n_theta=8, n_phi=16)
        assert rel_l2(outs[i].cpu().numpy()[idx], ref) <= TOL_FP64_REL_L2
    # move mesh 2's nodes and change its vorticity: the next batch call must use the new mesh
    m = ms[2]
    rng = np.random.default_rng(7)
    nodes2 = m.nodes + 0.02 * (2.0 / (m.n_side - 1)) * rng.standard_normal(m.nodes.shape)
    omega2 = -m.omega
    with torch.cuda.stream(stream):
        hs[2].bs_update(torch.from_numpy(nodes2).cuda(), torch.from_numpy(omega2).cuda(), stream=stream)
        batch.bs_batch_velocity(outs, stream=stream, precision=bs.BS_FP64, **P)
    stream.synchronize()
    idx = np.arange(0, m.n_nodes, max(1, m.n_nodes // 150))
    ref = orc.velocity(nodes2, m.tets, omega2, nodes2[idx], far_ratio=2.0, tet_order=4, n_theta=8, n_phi=16)
    assert rel_l2(outs[2].cpu().numpy()[idx], ref) <= TOL_FP64_REL_L2
    hs[2].bs_update(torch.from_numpy(m.nodes).cuda(), torch.from_numpy(m.omega).cuda())
    hs[2].bs_status()


def test_batch_with_an_empty_mesh(meshes):
    ms, hs = meshes
    e = bs.Mesh(ms[0].nodes, np.zeros((0, 4), dtype=np.int32), ms[0].omega)
    batch = bs.Batch([hs[1], e, hs[4]])
    outs = [torch.full((n, 3), 5.0, dtype=torch.float64, device="cuda")
            for n in (ms[1].n_nodes, ms[0].n_nodes, ms[4].n_nodes)]
    batch.bs_batch_velocity(outs, precision=bs.BS_FP32, **P)
    torch.cuda.synchronize()
    assert torch.all(outs[1] == 0)
    assert rms_over_max(outs[0].cpu().numpy(), _single(hs[1], ms[1], bs.BS_FP64)) <= TOL_FP32_RMS_MAX


def test_autotune_picks_a_variant_and_keeps_results(meshes, monkeypatch, tmp_path):
    monkeypatch.setenv("BS_TUNE_CACHE", str(tmp_path / "tune.json"))  # not the shipped cache
    ms, hs = meshes
    m, h = ms[5], hs[5]
    before = _single(h, m, bs.BS_FP32)
    v = h.bs_autotune(precision=bs.BS_FP32, **P)
    assert 0 <= v < bs.bs_num_variants(bs.BS_FP32, 4)
    after = _single(h, m, bs.BS_FP32)
    assert rms_over_max(after, before) <= TOL_FP32_RMS_MAX
