"""The autotuner and its cache: a miss times every variant and persists the winner as JSON, a hit takes
it without timing, and the chosen variant gives the oracle's velocity (every variant does: see
test_gpu_variants.py)."""
import json
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

P = dict(far_ratio=2.0, tet_gauss_order=4, n_theta=8, n_phi=16)


@pytest.fixture(scope="module")
def c1():
    bs.build()
    m = config1_plain(10)  # 1000 nodes, 4374 tets: a size class of its own
    return m, bs.Mesh(m.nodes, m.tets, m.omega)


@pytest.mark.parametrize("precision", [bs.BS_FP32, bs.BS_FP64], ids=["fp32", "fp64"])
def test_cache_miss_times_and_persists_then_hits(orc, c1, precision, monkeypatch, tmp_path):
    path = tmp_path / "tune.json"
    monkeypatch.setenv("BS_TUNE_CACHE", str(path))
    monkeypatch.setenv("BS_TUNE_FORCE", "1")
    m, h = c1
    t0 = time.perf_counter()
    v = h.bs_autotune(precision=precision, **P)
    miss = time.perf_counter() - t0
    n = bs.bs_num_variants(precision, 4)
    assert 0 <= v < n
    doc = json.loads(path.read_text())  # a valid JSON document
    entries = doc["entries"]
    tag = f"{'fp32' if precision == bs.BS_FP32 else 'fp64'} q4 ray L128"
    # two paths, two entries: bs_velocity (points) and bs_velocity_nodes (nodes: the walk can take the near field)
    for path_tag, vv in (("points", v), ("nodes", h.bs_tuned_variant(precision, 4, at_nodes=True))):
        key = [k for k in entries if tag in k and k.endswith(path_tag)]
        assert len(key) == 1, path_tag
        e = entries[key[0]]
        assert e["variant"] == vv and e["candidates"] == n and e["ms"] > 0
        s = bs.bs_variant_shape(precision, 4, bs.BS_NEAR_RAY, vv)
        assert e["shape"].startswith(f"P{s['points_per_thread']} T{s['tile']} S{s['stages']} B{s['ctas_per_sm']}")
    # a second handle on the same problem: a cache hit, no timing
    monkeypatch.delenv("BS_TUNE_FORCE")
    h2 = bs.Mesh(m.nodes, m.tets, m.omega)
    t0 = time.perf_counter()
    v2 = h2.bs_autotune(precision=precision, **P)
    hit = time.perf_counter() - t0
    assert v2 == v and h2.bs_tuned_variant(precision, 4, at_nodes=True) == h.bs_tuned_variant(precision, 4, True)
    assert hit < 0.1 * miss
    # and the variant it runs gives the oracle's velocity
    pts = torch.from_numpy(m.nodes).cuda()
    out = h2.bs_velocity(pts, precision=precision, **P).cpu().numpy()
    h2.bs_status()
    vo = orc.velocity(m.nodes, m.tets, m.omega, m.nodes, tet_order=4, far_ratio=2.0, n_theta=8, n_phi=16)
    if precision == bs.BS_FP64:
        assert rel_l2(out, vo) <= TOL_FP64_REL_L2
    else:
        assert rms_over_max(out, vo) <= TOL_FP32_RMS_MAX


def test_all_ray_needs_no_tuning(c1, monkeypatch, tmp_path):
    path = tmp_path / "tune.json"
    monkeypatch.setenv("BS_TUNE_CACHE", str(path))
    _, h = c1
    h.bs_autotune(precision=bs.BS_FP32, **dict(P, far_ratio=float("inf")))
    assert not path.exists()


def test_pinned_variant_overrides_the_cache(c1):
    m, h = c1
    pts = torch.from_numpy(m.nodes).cuda()
    n = bs.bs_num_variants(bs.BS_FP32, 4)
    # a variant with another tile size: its tile frames differ, so its float32 rounding does
    t0 = bs.bs_variant_shape(bs.BS_FP32, 4, bs.BS_NEAR_RAY, 0)["tile"]
    other = next(v for v in range(n) if bs.bs_variant_shape(bs.BS_FP32, 4, bs.BS_NEAR_RAY, v)["tile"] != t0)
    outs = []
    for v in (0, other):
        h.bs_set_variant(bs.BS_FP32, 4, bs.BS_NEAR_RAY, v)
        outs.append(h.bs_velocity(pts, precision=bs.BS_FP32, **P).cpu().numpy())
    h.bs_set_variant(bs.BS_FP32, 4, bs.BS_NEAR_RAY, -1)
    h.bs_status()
    assert rms_over_max(outs[0], outs[1]) <= TOL_FP32_RMS_MAX
    assert not np.array_equal(outs[0], outs[1]) or n == 1  # different launch shapes round differently
