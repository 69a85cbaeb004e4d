"""Writes oracle_plain_cube.json: oracle velocities and counts on the plain unit-cube workload.

Calls only ``oracle/`` (and the seeded input generators).  The stored values
anchor the oracle against unnoticed change: a later edit of the oracle's
arithmetic that moves them must regenerate this file and justify the change.
Run from the repository root:  python tests/golden/make_oracle_golden.py
"""
import json
import os
import sys

import numpy as np

ROOT = os.path.dirname(os.path.dirname(os.path.dirname(os.path.abspath(__file__))))
sys.path.insert(0, ROOT)

import oracle  # noqa: E402
from workloads import config1_plain  # noqa: E402

CASES = {
    "default": dict(far_ratio=2.0, tet_order=4, n_theta=8, n_phi=16),
    "pure_ray_4x4": dict(far_ratio=float("inf"), tet_order=4, n_theta=4, n_phi=4),
    "gauss27_16x16": dict(far_ratio=3.0, tet_order=27, n_theta=16, n_phi=16),
}


def main():
    m = config1_plain()
    idx = list(range(0, m.n_nodes, 46))
    out = {"workload": "plain unit cube 9^3 nodes, seed 1001", "node_index": idx, "cases": {}}
    for name, p in CASES.items():
        v, c = oracle.velocity(m.nodes, m.tets, m.omega, m.nodes[idx], counts=True, **p)
        out["cases"][name] = {"params": {k: (str(x) if isinstance(x, float) and np.isinf(x) else x)
                                         for k, x in p.items()},
                              "velocity": v.tolist(), "counts": c.tolist()}
    path = os.path.join(os.path.dirname(os.path.abspath(__file__)), "oracle_plain_cube.json")
    with open(path, "w") as f:
        json.dump(out, f, indent=1)
    print("wrote", path)


if __name__ == "__main__":
    main()
