"""Shared helpers of the GPU parity tests: error metrics and the count-stability filter."""
from __future__ import annotations

import numpy as np

# float64 path vs oracle: relative L2 of the velocity field
TOL_FP64_REL_L2 = 1e-12
# float32 path vs oracle: e = ||dv||_2 / (sqrt(N) max|v|)  (RMS error over the largest speed)
TOL_FP32_RMS_MAX = 1e-5


def rel_l2(v, ref) -> float:
    return float(np.linalg.norm(np.asarray(v) - ref) / np.linalg.norm(ref))


def rms_over_max(v, ref) -> float:
    ref = np.asarray(ref)
    n = ref.shape[0]
    return float(np.linalg.norm(np.asarray(v) - ref) / (np.sqrt(n) * np.linalg.norm(ref, axis=1).max()))


def oracle_with_stability(orc, mesh, pts, rel=1e-9, **params):
    """Oracle velocity and counts, plus a mask of points whose counts survive perturbed thresholds.

    The near/far threshold is moved by a factor (1 +- rel), the chord length
    threshold by (1 +- 1e-3) and the area-coordinate tolerance between 0 and
    1e-9: a point whose counts change under any of these has a decision
    within rounding distance of a threshold, and its counts are not compared
    bit for bit.
    """
    v, c = orc.velocity(mesh.nodes, mesh.tets, mesh.omega, pts, counts=True, **params)
    stable = np.ones(len(pts), dtype=bool)
    fr = params.get("far_ratio", 2.0)
    variants = []
    if np.isfinite(fr):
        variants += [dict(params, far_ratio=fr * (1 + rel)), dict(params, far_ratio=fr * (1 - rel))]
    variants += [dict(params, tau=1e-9 * (1 + 1e-3)), dict(params, tau=1e-9 * (1 - 1e-3)),
                 dict(params, eps_b=0.0), dict(params, eps_b=1e-9)]
    for p in variants:
        _, c2 = orc.velocity(mesh.nodes, mesh.tets, mesh.omega, pts, counts=True, **p)
        stable &= np.all(c2 == c, axis=1)
    return v, c, stable
