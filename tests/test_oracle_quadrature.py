"""Pins of the oracle's velocity sets (Table 1 of the paper and quadrature mathematics)."""
import math
import os
from decimal import Decimal

import numpy as np
import pytest

from oracle import quadrature as q

GOLDEN = os.path.join(os.path.dirname(__file__), "golden", "table1_halfrange_gh.txt")


def _table1():
    rows = {}
    with open(GOLDEN) as f:
        for line in f:
            if line.startswith("#") or not line.strip():
                continue
            rule, i, xi, w = line.split()
            rows.setdefault(rule, []).append((xi, w))
    return rows


def _half_unit_last_digit(s: str) -> float:
    mant = s.split(".")[1]
    return 0.5 * 10.0 ** (-len(mant))


@pytest.mark.parametrize("rule,n_half", [("D1Qh4", 2), ("D1Qh6", 3), ("D1Qh8", 4)])
def test_table1_every_printed_digit(rule, n_half):
    """Table 1: nodes and weights of D1Q^h_4/6/8 agree with every digit the paper prints."""
    nodes, weights = q.halfrange_1d(n_half)
    pos_nodes = nodes[n_half:]
    pos_w = weights[n_half:]
    for i, (xs, ws) in enumerate(_table1()[rule]):
        assert abs(float(pos_nodes[i]) - float(xs)) <= _half_unit_last_digit(xs) * 1.0001, (rule, i)
        assert abs(float(pos_w[i]) - float(ws)) <= _half_unit_last_digit(ws) * 1.0001, (rule, i)
        # mirrored half
        assert float(nodes[n_half - 1 - i]) == -float(pos_nodes[i])
        assert float(weights[n_half - 1 - i]) == float(pos_w[i])


def _exact_halfline_moment(k: int) -> float:
    """int_0^inf x^k exp(-x^2/2) dx / sqrt(2 pi) = 2^((k-1)/2) Gamma((k+1)/2) / sqrt(2 pi)."""
    return 2.0 ** ((k - 1) / 2) * math.gamma((k + 1) / 2) / math.sqrt(2 * math.pi)


@pytest.mark.parametrize("n_half", [1, 2, 3, 4, 5, 6, 8])
def test_halfline_rule_exact_to_degree_2n_minus_1(n_half):
    """An N-point Gauss rule on [0, inf) integrates x^k exactly for k <= 2N-1 and not for k = 2N."""
    nodes, weights = q.halfrange_1d(n_half)
    x = np.array([float(v) for v in nodes[n_half:]])
    w = np.array([float(v) for v in weights[n_half:]])
    for k in range(2 * n_half):
        assert abs(np.sum(w * x ** k) - _exact_halfline_moment(k)) <= 1e-13 * _exact_halfline_moment(k), k
    k = 2 * n_half
    rel = abs(np.sum(w * x ** k) - _exact_halfline_moment(k)) / _exact_halfline_moment(k)
    assert rel > 1e-8, "a Gauss rule cannot be exact at degree 2N"


def test_recurrence_closed_forms():
    """alpha_0 = m1/m0 = sqrt(2/pi) and beta_1 = m2/m0 - alpha_0^2 = 1 - 2/pi for the half-line weight."""
    mom = q.halfline_moments(8)
    alpha, beta = q.chebyshev_recurrence(mom, 4)
    assert abs(float(alpha[0]) - math.sqrt(2 / math.pi)) < 1e-15
    assert abs(float(beta[1]) - (1 - 2 / math.pi)) < 1e-15
    assert float(beta[0]) == 0.5


@pytest.mark.parametrize("n_half", [2, 4, 6])
def test_halfrange_flux_and_normalisation(n_half):
    """Each half carries weight 1/2 and sum_{xi>0} w xi = 1/sqrt(2 pi): the factor of Eq. (9)."""
    nodes, weights = q.halfrange_1d(n_half)
    x = np.array([float(v) for v in nodes])
    w = np.array([float(v) for v in weights])
    assert abs(w[x > 0].sum() - 0.5) < 1e-15
    assert abs((w * x)[x > 0].sum() - 1 / math.sqrt(2 * math.pi)) < 1e-15
    assert abs((w * x * x).sum() - 1.0) < 1e-14


@pytest.mark.parametrize("m", [2, 3, 4, 5, 6, 8, 12])
def test_fullrange_matches_textbook_gauss_hermite(m):
    """Full-range rule (weight exp(-x^2/2)/sqrt(2pi)) equals numpy's probabilists' Gauss-Hermite, normalised."""
    nodes, weights = q.fullrange_1d(m)
    xr, wr = np.polynomial.hermite_e.hermegauss(m)
    wr = wr / math.sqrt(2 * math.pi)
    np.testing.assert_allclose([float(v) for v in nodes], xr, rtol=0, atol=1e-13)
    np.testing.assert_allclose([float(v) for v in weights], wr, rtol=1e-12, atol=0)


def test_d2q9_is_the_standard_lattice():
    """M = 3 full range: nodes 0, +-sqrt(3), weights 2/3, 1/6 (the standard D2Q9 of the paper)."""
    xi_x, xi_y, w = q.velocity_set_2d("full", 3)
    assert len(w) == 9
    one_d = sorted(set(xi_x))
    assert abs(one_d[0] + math.sqrt(3)) < 1e-15 and one_d[1] == 0.0 and abs(one_d[2] - math.sqrt(3)) < 1e-15
    assert abs(max(w) - 4 / 9) < 1e-16 and abs(min(w) - 1 / 36) < 1e-17


@pytest.mark.parametrize("kind,n", [("half", 2), ("half", 4), ("half", 6), ("full", 3), ("full", 4)])
def test_2d_tensor_set_moments(kind, n):
    """2-D sets reproduce the Maxwellian moments the equilibrium of Eq. (5) needs (degree <= 2)."""
    xi_x, xi_y, w = (np.array(v) for v in q.velocity_set_2d(kind, n))
    m = int(round(math.sqrt(len(w))))
    assert m * m == len(w)
    assert abs(w.sum() - 1) < 1e-15
    assert abs((w * xi_x).sum()) < 1e-15 and abs((w * xi_y).sum()) < 1e-15
    assert abs((w * xi_x * xi_x).sum() - 1) < 1e-14 and abs((w * xi_y * xi_y).sum() - 1) < 1e-14
    assert abs((w * xi_x * xi_y).sum()) < 1e-15
    # ordering: alpha = iy * M + ix, ascending nodes
    assert np.all(np.diff(xi_x[:m]) > 0) and np.all(xi_y[:m] == xi_y[0])


def test_largest_nodes_of_the_sets_used():
    """Largest |xi| of D2Q^h_64 is the last Table 1 node; of D2Q^h_144 it exceeds it (N = 6)."""
    n4, _ = q.halfrange_1d(4)
    assert abs(float(n4[-1]) - 3.199890790) < 5e-10
    n6, _ = q.halfrange_1d(6)
    assert float(n6[-1]) > 4.0
