"""The oracle still reproduces the values stored by tests/golden/make_oracle_golden.py (no GPU)."""
import json
import os

import numpy as np

from workloads import config1_plain

GOLDEN = os.path.join(os.path.dirname(__file__), "golden", "oracle_plain_cube.json")


def test_oracle_matches_stored_values(orc):
    with open(GOLDEN) as f:
        g = json.load(f)
    m = config1_plain()
    idx = g["node_index"]
    for name, case in g["cases"].items():
        p = {k: (float(v) if v == "inf" else v) for k, v in case["params"].items()}
        v, c = orc.velocity(m.nodes, m.tets, m.omega, m.nodes[idx], counts=True, **p)
        ref = np.array(case["velocity"])
        assert np.linalg.norm(v - ref) <= 1e-13 * np.linalg.norm(ref), name
        assert np.array_equal(c, np.array(case["counts"])), name
