"""Gauss-Hermite velocity sets in extended precision (oracle; test infrastructure only).

Follows Table 1 of the paper and the text around it: the one-dimensional
half-range rule D1Q^h_{2N} uses the N Gauss nodes of the weight
exp(-xi^2/2)/sqrt(2 pi) on [0, inf), mirrored to the negative half-line, and the
two-dimensional set D2Q^h_{(2N)^2} is the tensor product of two such rules.
The full-range rules D2Q_{M^2} (standard LB sets, e.g. D2Q9 with M=3) are the
Gauss rules of the same weight on the whole line.

Method (Golub-Welsch on the three-term recurrence):

1. exact moments m_k of the weight, written out from the Gamma function at
   half-integers;
2. recurrence coefficients (alpha_k, beta_k) of the monic orthogonal
   polynomials from those moments by Chebyshev's algorithm;
3. nodes = eigenvalues of the symmetric tridiagonal Jacobi matrix, weights =
   m_0 * (first component of the normalised eigenvector)^2, with the eigen
   decomposition done by cyclic Jacobi rotations.

All arithmetic is Python ``decimal`` at 80 significant digits; the results are
rounded to float64 only at the very end.  Pinned by: Table 1 (10 printed
digits), exactness on monomials up to degree 2N-1 and failure at degree 2N,
the closed forms alpha_0 = sqrt(2/pi), beta_1 = 1 - 2/pi, and the full-range
rule against the textbook probabilists' Gauss-Hermite routine.
"""
from __future__ import annotations

from decimal import Decimal, localcontext

PREC = 80


def _pi() -> Decimal:
    """pi to the working precision (Machin's formula, pure Decimal)."""
    def arctan_inv(x: int) -> Decimal:
        x = Decimal(x)
        x2 = x * x
        term = Decimal(1) / x
        total = term
        k = 1
        eps = Decimal(10) ** (-(PREC + 5))
        while True:
            term = -term / x2
            delta = term / (2 * k + 1)
            if abs(delta) < eps:
                break
            total += delta
            k += 1
        return total

    return 4 * (4 * arctan_inv(5) - arctan_inv(239))


def halfline_moments(nmom: int) -> list[Decimal]:
    """m_k = int_0^inf xi^k exp(-xi^2/2) / sqrt(2 pi) dxi, k = 0..nmom-1.

    Even k = 2p:   m_k = (2p-1)!! / 2          (so m_0 = 1/2: each half of a
                                                 Table 1 rule carries weight 1/2)
    Odd  k = 2p+1: m_k = 2^p p! / sqrt(2 pi)
    """
    inv_sqrt_2pi = 1 / (2 * _pi()).sqrt()
    out = []
    for k in range(nmom):
        if k % 2 == 0:
            p = k // 2
            dfact = Decimal(1)
            for j in range(1, 2 * p, 2):
                dfact *= j
            out.append(dfact / 2)
        else:
            p = (k - 1) // 2
            fact = Decimal(1)
            for j in range(1, p + 1):
                fact *= j
            out.append(Decimal(2) ** p * fact * inv_sqrt_2pi)
    return out


def fullline_moments(nmom: int) -> list[Decimal]:
    """Moments of exp(-xi^2/2)/sqrt(2 pi) on the whole line: (k-1)!! for even k, 0 for odd."""
    out = []
    for k in range(nmom):
        if k % 2 == 1:
            out.append(Decimal(0))
        else:
            dfact = Decimal(1)
            for j in range(1, k, 2):
                dfact *= j
            out.append(dfact)
    return out


def chebyshev_recurrence(mom: list[Decimal], n: int) -> tuple[list[Decimal], list[Decimal]]:
    """Chebyshev's algorithm: (alpha_k, beta_k), k < n, of the monic orthogonal
    polynomials p_{k+1}(x) = (x - alpha_k) p_k(x) - beta_k p_{k-1}(x), from the
    2n moments mom[0..2n-1]; beta_0 = mom[0]."""
    assert len(mom) >= 2 * n
    alpha = [Decimal(0)] * n
    beta = [Decimal(0)] * n
    sig_prev = [Decimal(0)] * (2 * n)          # sigma_{k-2, l}
    sig = list(mom[: 2 * n])                   # sigma_{k-1, l}
    alpha[0] = mom[1] / mom[0]
    beta[0] = mom[0]
    for k in range(1, n):
        sig_new = [Decimal(0)] * (2 * n)
        for l in range(k, 2 * n - k):
            sig_new[l] = sig[l + 1] - alpha[k - 1] * sig[l] - beta[k - 1] * sig_prev[l]
        alpha[k] = sig_new[k + 1] / sig_new[k] - sig[k] / sig[k - 1]
        beta[k] = sig_new[k] / sig[k - 1]
        sig_prev, sig = sig, sig_new
    return alpha, beta


def jacobi_eigh(a: list[list[Decimal]]) -> tuple[list[Decimal], list[list[Decimal]]]:
    """Eigen-decomposition of a small symmetric matrix by cyclic Jacobi rotations.

    Returns (eigenvalues, V) with column j of V the unit eigenvector of eigenvalue j."""
    n = len(a)
    a = [row[:] for row in a]
    v = [[Decimal(1) if i == j else Decimal(0) for j in range(n)] for i in range(n)]
    tiny = Decimal(10) ** (-(PREC - 5))
    for _sweep in range(100):
        off = sum((a[i][j] * a[i][j] for i in range(n) for j in range(n) if i != j), Decimal(0))
        if off.sqrt() < tiny:
            break
        for p in range(n - 1):
            for q in range(p + 1, n):
                if a[p][q] == 0:
                    continue
                tau = (a[q][q] - a[p][p]) / (2 * a[p][q])
                sgn = Decimal(1) if tau >= 0 else Decimal(-1)
                t = sgn / (abs(tau) + (1 + tau * tau).sqrt())
                c = 1 / (1 + t * t).sqrt()
                s = t * c
                for k in range(n):          # A <- A J   (columns p, q)
                    akp, akq = a[k][p], a[k][q]
                    a[k][p] = c * akp - s * akq
                    a[k][q] = s * akp + c * akq
                for k in range(n):          # A <- J^T A (rows p, q)
                    apk, aqk = a[p][k], a[q][k]
                    a[p][k] = c * apk - s * aqk
                    a[q][k] = s * apk + c * aqk
                for k in range(n):          # V <- V J
                    vkp, vkq = v[k][p], v[k][q]
                    v[k][p] = c * vkp - s * vkq
                    v[k][q] = s * vkp + c * vkq
    else:
        raise RuntimeError("Jacobi rotations did not converge")
    return [a[i][i] for i in range(n)], v


def gauss_rule(mom: list[Decimal], n: int) -> tuple[list[Decimal], list[Decimal]]:
    """Golub-Welsch: n-point Gauss rule (ascending nodes, weights) for the given moments."""
    alpha, beta = chebyshev_recurrence(mom, n)
    jac = [[Decimal(0)] * n for _ in range(n)]
    for i in range(n):
        jac[i][i] = alpha[i]
        if i + 1 < n:
            jac[i][i + 1] = jac[i + 1][i] = beta[i + 1].sqrt()
    lam, vec = jacobi_eigh(jac)
    pairs = sorted((lam[j], mom[0] * vec[0][j] * vec[0][j]) for j in range(n))
    return [p[0] for p in pairs], [p[1] for p in pairs]


def halfrange_1d(n_half: int) -> tuple[list[Decimal], list[Decimal]]:
    """D1Q^h_{2N}: nodes ascending (-xi_N .. -xi_1, xi_1 .. xi_N), weights (each half sums to 1/2)."""
    with localcontext() as ctx:
        ctx.prec = PREC
        x, w = gauss_rule(halfline_moments(2 * n_half), n_half)
        nodes = [-xi for xi in reversed(x)] + list(x)
        weights = list(reversed(w)) + list(w)
        return nodes, weights


def fullrange_1d(m: int) -> tuple[list[Decimal], list[Decimal]]:
    """Full-range M-point Gauss-Hermite rule of exp(-xi^2/2)/sqrt(2 pi) (weights sum to 1)."""
    with localcontext() as ctx:
        ctx.prec = PREC
        x, w = gauss_rule(fullline_moments(2 * m), m)
        # symmetrise exactly: the rule is symmetric about 0
        nodes = [(x[i] - x[m - 1 - i]) / 2 for i in range(m)]
        weights = [(w[i] + w[m - 1 - i]) / 2 for i in range(m)]
        return nodes, weights


def velocity_set_2d(kind: str, n: int):
    """Tensor-product 2-D set as float64 lists (xi_x, xi_y, w), alpha = iy*M + ix.

    kind 'half': n = N nodes per half-axis, M = 2N (D2Q^h_{(2N)^2}).
    kind 'full': n = M nodes per axis (D2Q_{M^2}; D2Q9 is M = 3).
    """
    if kind == "half":
        nodes, weights = halfrange_1d(n)
    elif kind == "full":
        nodes, weights = fullrange_1d(n)
    else:
        raise ValueError(kind)
    m = len(nodes)
    with localcontext() as ctx:
        ctx.prec = PREC
        xi_x, xi_y, w = [], [], []
        for iy in range(m):
            for ix in range(m):
                xi_x.append(float(nodes[ix]))
                xi_y.append(float(nodes[iy]))
                w.append(float(weights[ix] * weights[iy]))
    return xi_x, xi_y, w


def mixed_set_2d(x_nodes, x_weights, y_nodes, y_weights):
    """Tensor product of two different 1-D rules (x-axis rule, y-axis rule), float64 lists."""
    with localcontext() as ctx:
        ctx.prec = PREC
        xi_x, xi_y, w = [], [], []
        for iy in range(len(y_nodes)):
            for ix in range(len(x_nodes)):
                xi_x.append(float(x_nodes[ix]))
                xi_y.append(float(y_nodes[iy]))
                w.append(float(Decimal(x_weights[ix]) * Decimal(y_weights[iy])))
    return xi_x, xi_y, w
