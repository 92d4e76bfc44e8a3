"""The oracle's lid-driven cavity against the paper's printed Table 2 (drag D of the lid,
reduced flow rate G of the main vortex) for the 16-velocity half-range and full-range sets.

An external pin of the cavity path (walls on all four sides, corners, the moving lid):
the oracle marches D2Q^h_16 and D2Q_16 cavities to their steady state on a 64 x 64 grid and
its D and G agree with the paper's own D2Q^h_16 and D2Q_16 columns within 6 % (the paper's
grid is not stated; on the GPU the same quantities come within 3 % at 128^2 and converge
towards the printed values as the grid is refined).  Readings of the printed table (fixture
header): D = lid-mean |p_xy| / u_w, G = 2 x the centre-line integral of u_x / u_w from the
vortex centre to the lid, D entries of the Kn = 0.2 and 0.4 rows interchanged.  The paper's
claim that the half-range set is the closer one to the kinetic (BGKW) values is checked too.
"""
import os

import numpy as np
import pytest

from oracle.march import CAVITY, make_problem

HERE = os.path.dirname(os.path.abspath(__file__))
SIDE, U_W = 64, 0.01


def _table():
    rows = {}
    for line in open(os.path.join(HERE, "golden", "table2_cavity_drag_flowrate.txt")):
        if line.startswith("#") or not line.strip():
            continue
        v = [float(t) for t in line.split()]
        rows[v[0]] = v[1:]
    # reading: the D entries of the Kn = 0.2 and 0.4 rows are interchanged in print
    out = {}
    for kn, v in rows.items():
        d = rows[{0.2: 0.4, 0.4: 0.2}.get(kn, kn)]
        out[kn] = {"D": {"bgkw": d[0], "half": d[1], "full": d[2]}, "G": {"bgkw": v[3], "half": v[4], "full": v[5]}}
    return out


_cache = {}


def _solve(kind, kn):
    key = (kind, kn)
    if key not in _cache:
        n = 2 if kind == "half" else 4          # D2Q^h_16 and D2Q_16
        p = make_problem(kind, n, CAVITY, SIDE, SIDE, kn, 0.0, U_W)
        h, steps, r = p.march(p.zeros(), 400_000, every=100, tol=1e-9)
        assert r < 1e-9, (kind, kn, steps, r)
        D = abs(p.face_flux_y(h)[SIDE].mean()) / U_W
        ux = p.moments(h)["ux"] / U_W
        line = 0.5 * (ux[:, SIDE // 2 - 1] + ux[:, SIDE // 2])
        y = (np.arange(SIDE) + 0.5) / SIDE
        k = max(i for i in range(SIDE - 1) if line[i] <= 0.0 < line[i + 1])
        yc = y[k] - line[k] * (y[k + 1] - y[k]) / (line[k + 1] - line[k])
        ys = np.concatenate([[yc], y[k + 1:], [1.0]])
        us = np.concatenate([[0.0], line[k + 1:], [line[-1]]])
        G = 2.0 * float(np.sum(0.5 * (us[1:] + us[:-1]) * np.diff(ys)))
        _cache[key] = (D, G)
    return _cache[key]


@pytest.mark.slow
@pytest.mark.parametrize("kn", [0.05, 0.1, 0.2, 0.4])
@pytest.mark.parametrize("kind", ["half", "full"])
def test_cavity_drag_and_flow_rate_match_printed_table(kind, kn):
    printed = _table()[kn]
    D, G = _solve(kind, kn)
    assert abs(D / printed["D"][kind] - 1) < 0.06, (D, printed["D"][kind])
    assert abs(G / printed["G"][kind] - 1) < 0.06, (G, printed["G"][kind])


@pytest.mark.slow
@pytest.mark.parametrize("kn", [0.05, 0.1, 0.2, 0.4])
def test_half_range_set_is_closer_to_kinetic_values(kn):
    """D at every Kn; G from Kn = 0.1 on (at Kn = 0.05 both sets are within 5 % of the
    kinetic G and this grid's own error decides the order: at 128^2 the half-range set is
    the closer one there too)."""
    printed = _table()[kn]
    dh, gh = _solve("half", kn)
    df, gf = _solve("full", kn)
    assert abs(dh - printed["D"]["bgkw"]) < abs(df - printed["D"]["bgkw"])
    if kn >= 0.1:
        assert abs(gh - printed["G"]["bgkw"]) < abs(gf - printed["G"]["bgkw"])
