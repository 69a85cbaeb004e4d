"""bs_velocity_noalloc, the entry point for callers that may not let the library allocate GPU memory.

Such callers (an application whose device memory is all handed out by its
own pool under a fixed budget, or a time-critical loop that cannot take the
synchronisation or the out-of-memory failure of a driver allocation) cannot
use bs_create / bs_velocity, which allocate the mesh tables and partial sums.
bs_velocity_noalloc keeps those in a fixed array of library-owned device
memory instead.  Its results must agree with bs_velocity on the same mesh and
points, within the tolerances the parity tests use, and keep agreeing on a
second call that reuses the same scratch array, also at the size limits of
that array.  A mesh error found on the device (such callers get no host-side
validation, which would need a synchronisation) must show in the results as
NaN velocities and counts of -1.  This file is named so that pytest collects
it last.
"""
import numpy as np
import pytest
from gpu_helpers import TOL_FP32_RMS_MAX, TOL_FP64_REL_L2, rel_l2, rms_over_max

from workloads import config1_plain

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")
if not torch.cuda.is_available():
    pytest.skip("no CUDA device", allow_module_level=True)

import paper_0712_1695_gb300 as bs  # noqa: E402
from paper_0712_1695_gb300.binding import (  # noqa: E402
    BS_ERR_ARG, BS_ERR_MESH, BS_ERR_ORDER, BSError, bs_noalloc_status, bs_velocity_noalloc)

PARAMS = dict(far_ratio=2.0, tet_gauss_order=4, n_theta=8, n_phi=16)


@pytest.fixture(scope="module")
def case():
    bs.build()
    m = config1_plain()  # 729 nodes, 3072 tets: inside the fixed limits
    dev = {name: torch.from_numpy(np.ascontiguousarray(a)).cuda()
           for name, a in (("nodes", m.nodes), ("omega", m.omega), ("tets", m.tets.astype(np.int32)))}
    rng = np.random.default_rng(3)
    pts = np.concatenate([m.nodes, rng.uniform(0.0, 1.0, size=(300, 3))])
    dev["pts"] = torch.from_numpy(pts).cuda()
    return m, dev


@pytest.mark.parametrize("precision", ["fp64", "fp32"])
def test_noalloc_matches_bs_velocity_on_two_calls(case, precision):
    m, d = case
    prec = bs.BS_FP64 if precision == "fp64" else bs.BS_FP32
    h = bs.Mesh(m.nodes, m.tets, m.omega)
    k = d["pts"].shape[0]
    ref_counts = torch.zeros((k, 3), dtype=torch.int32, device="cuda")
    ref = h.bs_velocity(d["pts"], counts_dev=ref_counts, precision=prec, **PARAMS).cpu().numpy()
    h.bs_status()
    for call in range(2):
        out = torch.full((k, 3), float("nan"), dtype=torch.float64, device="cuda")
        counts = torch.full((k, 3), -1, dtype=torch.int32, device="cuda")
        bs_velocity_noalloc(d["nodes"], d["tets"], d["omega"], d["pts"], out, counts_dev=counts, precision=prec,
                            **PARAMS)
        bs_noalloc_status()  # no error raised on the device
        v = out.cpu().numpy()
        assert np.all(np.isfinite(v)), f"call {call}"
        if prec == bs.BS_FP64:
            assert rel_l2(v, ref) <= TOL_FP64_REL_L2, f"call {call}"
        else:
            assert rms_over_max(v, ref) <= TOL_FP32_RMS_MAX, f"call {call}"
        assert torch.equal(counts, ref_counts), f"call {call}"


def test_noalloc_with_the_exact_near_rule(case):
    m, d = case
    h = bs.Mesh(m.nodes, m.tets, m.omega)
    P = dict(PARAMS, near_rule=bs.BS_NEAR_EXACT)
    ref = h.bs_velocity(d["pts"], precision=bs.BS_FP64, **P).cpu().numpy()
    h.bs_status()
    out = torch.full(tuple(d["pts"].shape), float("nan"), dtype=torch.float64, device="cuda")
    bs_velocity_noalloc(d["nodes"], d["tets"], d["omega"], d["pts"], out, precision=bs.BS_FP64, **P)
    torch.cuda.synchronize()
    assert rel_l2(out.cpu().numpy(), ref) <= TOL_FP64_REL_L2


def test_noalloc_rejects_sizes_beyond_its_scratch(case):
    m, d = case
    out = torch.empty_like(d["pts"])
    with pytest.raises(BSError) as ei:
        bs_velocity_noalloc(d["nodes"], d["tets"], d["omega"], d["pts"], out, **dict(PARAMS, n_theta=128, n_phi=64))
    assert ei.value.code == BS_ERR_ARG and "4096" in str(ei.value)
    with pytest.raises(BSError) as ei:
        bs_velocity_noalloc(d["nodes"], d["tets"], d["omega"], d["pts"], out, **dict(PARAMS, tet_gauss_order=27))
    assert ei.value.code == BS_ERR_ORDER
    many = torch.zeros((4097, 3), dtype=torch.float64, device="cuda")
    with pytest.raises(BSError) as ei:
        bs_velocity_noalloc(d["nodes"], d["tets"], d["omega"], many, torch.empty_like(many), **PARAMS)
    assert ei.value.code == BS_ERR_ARG


def _dev(a, dtype=None):
    t = torch.from_numpy(np.ascontiguousarray(a))
    return (t if dtype is None else t.to(dtype)).cuda()


@pytest.mark.parametrize("precision", ["fp64", "fp32"])
def test_noalloc_at_its_size_limits(precision):
    """The largest Kuhn grid within the fixed limits (12^3 nodes, 7986 tets), 4096 points, 64 x 64 directions."""
    m = config1_plain(12)
    assert m.n_tets <= 8192
    prec = bs.BS_FP64 if precision == "fp64" else bs.BS_FP32
    rng = np.random.default_rng(4096)
    pts = np.concatenate([m.nodes, rng.uniform(-0.2, 1.2, size=(4096 - m.n_nodes, 3))])
    P = dict(PARAMS, n_theta=64, n_phi=64)
    h = bs.Mesh(m.nodes, m.tets, m.omega)
    dp = _dev(pts)
    ref_counts = torch.zeros((4096, 3), dtype=torch.int32, device="cuda")
    ref = h.bs_velocity(dp, counts_dev=ref_counts, precision=prec, **P).cpu().numpy()
    h.bs_status()
    nodes, tets, omega = _dev(m.nodes), _dev(m.tets, torch.int32), _dev(m.omega)
    for call in range(2):
        out = torch.full((4096, 3), float("nan"), dtype=torch.float64, device="cuda")
        counts = torch.full((4096, 3), -1, dtype=torch.int32, device="cuda")
        bs_velocity_noalloc(nodes, tets, omega, dp, out, counts_dev=counts, precision=prec, **P)
        torch.cuda.synchronize()
        v = out.cpu().numpy()
        if prec == bs.BS_FP64:
            assert rel_l2(v, ref) <= TOL_FP64_REL_L2, f"call {call}"
        else:
            assert rms_over_max(v, ref) <= TOL_FP32_RMS_MAX, f"call {call}"
        assert torch.equal(counts[:, :2], ref_counts[:, :2]), f"call {call}"


def test_noalloc_without_tets(case):
    m, d = case
    k = d["pts"].shape[0]
    out = torch.full((k, 3), 5.0, dtype=torch.float64, device="cuda")
    counts = torch.full((k, 3), 7, dtype=torch.int32, device="cuda")
    empty = torch.zeros((0, 4), dtype=torch.int32, device="cuda")
    bs_velocity_noalloc(d["nodes"], empty, d["omega"], d["pts"], out, counts_dev=counts, precision=bs.BS_FP32,
                        **PARAMS)
    torch.cuda.synchronize()
    assert torch.all(out == 0) and torch.all(counts == 0)


@pytest.mark.parametrize("fault", ["flat tet", "node index out of range"])
def test_noalloc_reports_mesh_errors_in_its_results(case, fault):
    m, d = case
    tets = m.tets.copy()
    if fault == "flat tet":
        tets[9] = [tets[9, 0], tets[9, 1], tets[9, 1], tets[9, 2]]
    else:
        tets[17, 2] = m.n_nodes + 3
    k = d["pts"].shape[0]
    out = torch.zeros((k, 3), dtype=torch.float64, device="cuda")
    counts = torch.zeros((k, 3), dtype=torch.int32, device="cuda")
    bs_velocity_noalloc(d["nodes"], _dev(tets, torch.int32), d["omega"], d["pts"], out, counts_dev=counts,
                        precision=bs.BS_FP32, **PARAMS)
    torch.cuda.synchronize()
    assert torch.all(torch.isnan(out)) and torch.all(counts == -1)
    # the flag word itself, read through bs_noalloc_status: a mesh error naming the lowest bad tet
    with pytest.raises(BSError) as err:
        bs_noalloc_status()
    assert err.value.code == BS_ERR_MESH
    assert err.value.first_bad_tet == (9 if fault == "flat tet" else 17)
    # the next call on a valid mesh starts from a cleared flag
    bs_velocity_noalloc(d["nodes"], d["tets"], d["omega"], d["pts"], out, counts_dev=counts, precision=bs.BS_FP32,
                        **PARAMS)
    bs_noalloc_status()
    torch.cuda.synchronize()
    assert torch.all(torch.isfinite(out)) and torch.all(counts >= 0)


def test_noalloc_rejects_counts_it_cannot_write(case):
    m, d = case
    k = d["pts"].shape[0]
    out = torch.empty((k, 3), dtype=torch.float64, device="cuda")
    for bad in (torch.zeros((k, 3), dtype=torch.int32),  # host memory
                torch.zeros((k, 3), dtype=torch.int64, device="cuda"),
                torch.zeros((k - 1, 3), dtype=torch.int32, device="cuda"),
                torch.zeros((3, k), dtype=torch.int32, device="cuda").t()):  # not contiguous
        with pytest.raises(ValueError):
            bs_velocity_noalloc(d["nodes"], d["tets"], d["omega"], d["pts"], out, counts_dev=bad, **PARAMS)
