"""Planted mistakes in copies of the oracle must each fail at least one pin (no GPU).

Every mutant is a one-line textual edit of ``oracle/bs_oracle.c`` (a dropped
sign, a wrong prefactor, a transposed operand, a wrong index or constant),
compiled into a temporary library.  The shipped oracle passes the same quick
battery.  This shows that the pins constrain each step of the method, not
only the oracle's agreement with itself.
"""
import os

import numpy as np
import pytest
from brute_force import chord_by_sampling, signed_chord_integral

import oracle
import pins

SRC = os.path.join(os.path.dirname(oracle.__file__), "bs_oracle.c")

MUTANTS = {
    "sign(R) dropped for R1 <= 0": (
        "J[j] = -0.5 * (R1 - R0) * (w0[j] + w1[j]);", "J[j] = 0.5 * (R1 - R0) * (w0[j] + w1[j]);"),
    "printed 1/(16 pi^2) prefactor": (
        "k[l] = (M_PI / 16.0) * sin(phi)", "k[l] = (1.0 / (16.0 * M_PI * M_PI)) * sin(phi)"),
    "far rule operands transposed": ("cross3(r, wqv, rxw);", "cross3(wqv, r, rxw);"),
    "pre-check inequality reversed": (
        "if (rs * rs < dot3(r, r) - 2.0 * hmax * hmax) return 0;",
        "if (rs * rs > dot3(r, r) - 2.0 * hmax * hmax) return 0;"),
    "tet rule constant": ("double a = (5.0 + 3.0 * sqrt(5.0)) / 20.0", "double a = (5.0 + 2.0 * sqrt(5.0)) / 20.0"),
    "face area coordinates swapped": (
        "u * om[3 * b + j] + vv * om[3 * c + j]", "vv * om[3 * b + j] + u * om[3 * c + j]"),
    "phi over a quarter circle": (
        "double phi = (1.0 + tN[n]) * M_PI / 2.0;", "double phi = (1.0 + tN[n]) * M_PI / 4.0;"),
    "sin(phi) weight dropped": (
        "k[l] = (M_PI / 16.0) * sin(phi) * wN[n] * wM[m];", "k[l] = (M_PI / 16.0) * wN[n] * wM[m];"),
    "straddling chord halves added": (
        "J[j] = 0.5 * R1 * (wx + w1[j]) - 0.5 * (0.0 - R0) * (w0[j] + wx);",
        "J[j] = 0.5 * R1 * (wx + w1[j]) + 0.5 * (0.0 - R0) * (w0[j] + wx);"),
    "Gauss-Legendre weight": ("w[n - 1 - i] = 2.0 / ((1.0 - x * x) * dpn * dpn);",
                              "w[n - 1 - i] = 1.0 / ((1.0 - x * x) * dpn * dpn);"),
    "triangle edge test dropped": ("if (vv < -eps_b || uu + vv > 1.0 + eps_b) return 0;",
                                   "if (vv < -eps_b || vv > 1.0 + eps_b) return 0;"),
    "circumradius halved": ("*circumradius = sqrt(dot3(dp, dp));", "*circumradius = 0.5 * sqrt(dot3(dp, dp));"),
    "far rule volume factor dropped": ("double f = -inv4pi * wq[q] * vol[e] / (R * R * R);",
                                       "double f = -inv4pi * wq[q] / (R * R * R);"),
    "derivative: boundary term dropped": ("if (!bnd[4 * e + ends[k]]) continue;", "if (1) continue;"),
    "derivative: face-crossing shift sign": ("const double dR = -dot3(n, ed) / dot3(n, s);",
                                             "const double dR = dot3(n, ed) / dot3(n, s);"),
    "derivative: signed chord length": ("dJ[j] = (fabs(R1) - fabs(R0)) * gw[j];", "dJ[j] = (R1 - R0) * gw[j];"),
    "derivative: vorticity gradient index": ("gw[j] += om[3 * i + j] * ge;", "gw[j] += om[3 * ((i + 1) % 4) + j] * ge;"),
    "analytic: curl term dropped": ("vel[j] = c * (S[j] - curl[j] * volint);", "vel[j] = c * S[j];"),
    "analytic: arc tangent term sign": ("I0 += P0 * f - ah * beta;", "I0 += P0 * f + ah * beta;"),
    "analytic: normal part of the face moment": ("q[j] = Ip[j] + h * n[j] * I0;", "q[j] = Ip[j];"),
    "analytic: edge logarithm reversed": ("f = log((Rm - lm) / (Rp - lp));", "f = log((Rp - lp) / (Rm - lm));"),
    "analytic: volume integral factor": ("volint += 0.5 * h * I0;", "volint += h * I0;"),
}


def battery(orc):
    """Quick pins; returns the names of those that fail."""
    failed = []
    # Gauss-Legendre exactness and the half-sphere moments of the direction table
    t, w = orc.gauss_legendre(8)
    if any(abs(np.dot(w, t**m) - (0 if m % 2 else 2 / (m + 1))) > 1e-13 for m in range(16)):
        failed.append("gauss-legendre")
    s, k = orc.directions(16, 16)
    if not np.allclose((k[:, None, None] * s[:, :, None] * s[:, None, :]).sum(0), np.eye(3) / 6, atol=1e-12):
        failed.append("direction moments")
    # tet rule: degree 2 exactness of the 4-point rule
    bary, wq = orc.tet_rule(4)
    xi = bary[:, 1:]
    if abs(np.dot(wq, xi[:, 0] ** 2) - 6 * 2 / 120) > 1e-14 or abs(np.dot(wq, xi[:, 0] * xi[:, 1]) - 6 / 120) > 1e-14:
        failed.append("tet rule")
    # Kuhn tet circumradius
    sde = 0.25
    _, rho, _, _ = orc.tet_geometry(np.array([[0, 0, 0], [sde, 0, 0], [sde, sde, 0], [sde, sde, sde]]))
    if abs(rho - np.sqrt(3) * sde / 2) > 1e-15:
        failed.append("circumradius")
    # chords against sampling, including lines through x inside and behind x
    rng = np.random.default_rng(31)
    V = np.array([[0, 0, 0], [1, 0.1, 0], [0.2, 1, 0.1], [0.1, 0.2, 1.0]])
    om = rng.standard_normal((4, 3))
    bad = False
    for x in (np.array([2.0, 1.5, 1.2]), V.mean(0), np.array([-1.0, -0.8, -0.5])):
        for _ in range(6):
            tgt = V.mean(0) + 0.2 * rng.standard_normal(3)
            sd = (tgt - x) / np.linalg.norm(tgt - x)
            hit, R0, R1, J = orc.line_tet(x, sd, V, om)
            ref = chord_by_sampling(x, sd, V, span=6.0, n=4001)
            if ref is None or ref[1] - ref[0] < 1e-6:
                continue
            if not hit or abs(R0 - ref[0]) > 1e-10 or abs(R1 - ref[1]) > 1e-10:
                bad = True
                continue
            if not np.allclose(J, signed_chord_integral(x, sd, V, om, R0, R1), atol=1e-12):
                bad = True
    if bad:
        failed.append("chords")
    # single tet vs the Duffy-cone integral (inside point, and far point with the tet rule)
    r = pins.single_tet(orc, Ns=(64,), qs=(4, 64))
    if r["inside"]["ray"][0] > 1e-3 or r["far"]["gauss"][1] > 1e-6:
        failed.append("single tet")
    # uniform ball closed form and Hill's vortex (coarse)
    errs, _ = pins.ball(orc, ns=(5, 9), N=32, count=6)
    if errs[-1] > 2e-3:
        failed.append("ball")
    if pins.ball_outside(orc, n=9) > 3e-2:
        failed.append("ball outside")
    if pins.hill(orc, ns=(9,), count=8)[0] > 2e-2:
        failed.append("hill")
    # derivative along a direction (stretching term) against central differences and the ball
    d = pins.dderiv(orc, count=10)
    if d["points"] > 1e-4 or d["nodes"] > 2e-3 or d["ball"] > 2.5e-2:
        failed.append("derivative")
    # exact single-tet integral against the Duffy-cone integral, additivity, divergence
    a = pins.analytic(orc, quick=True)
    if max(a["single"].values()) > 5e-12 or a["split"] > 1e-12 or a["div"] > 5e-6:
        failed.append("analytic")
    return failed


@pytest.fixture(scope="module")
def mutant_dir(tmp_path_factory):
    return tmp_path_factory.mktemp("mutants")


def test_shipped_oracle_passes_battery(orc):
    assert battery(orc) == []


@pytest.mark.parametrize("name", sorted(MUTANTS))
def test_mutant_is_caught(name, mutant_dir):
    old, new = MUTANTS[name]
    src = open(SRC).read()
    assert src.count(old) == 1, f"mutation site for '{name}' not found exactly once"
    slug = "".join(c if c.isalnum() else "_" for c in name)
    path = mutant_dir / f"{slug}.c"
    path.write_text(src.replace(old, new))
    lib = oracle.build(force=True, src=str(path), out=str(mutant_dir / f"lib{slug}.so"))
    failed = battery(oracle.OracleLib(lib))
    assert failed, f"mutant '{name}' passed every pin"
