"""1D point sets on [0,1] (oracle; test infrastructure only).

Gauss-Lobatto-Legendre (GLL) nodes of order p: the endpoints plus the roots
of P'_p, the derivative of the Legendre polynomial of degree p. The paper
lists the nodal Lagrange basis at Gauss-Lobatto points among the H1 bases
(Sec. 3.3, "Finite Elements").

Gauss-Legendre rule with q points: roots x_k of P_q with weights
2 / ((1 - x_k^2) P'_q(x_k)^2) on [-1,1]; mapped to [0,1] the weights halve
and sum to 1 (quadrature in reference space, Sec. 4.3).

Both are found by Newton's method on the three-term Legendre recurrence,
carried out in numpy long double and rounded to float64 at the end.
"""

import numpy as np

_LD = np.longdouble


def legendre(n, x):
    """(P_n(x), P'_n(x)) by the recurrence
    (k+1) P_{k+1} = (2k+1) x P_k - k P_{k-1}, and
    P'_n = n (x P_n - P_{n-1}) / (x^2 - 1)  (for |x| < 1)."""
    x = np.asarray(x, dtype=_LD)
    p0 = np.ones_like(x)
    if n == 0:
        return p0, np.zeros_like(x)
    p1 = x.copy()
    for k in range(1, n):
        p0, p1 = p1, ((2 * k + 1) * x * p1 - k * p0) / (k + 1)
    dp = n * (x * p1 - p0) / (x * x - 1)
    return p1, dp


def legendre_d2(n, x):
    """P''_n from the Legendre ODE: (1-x^2) P'' = 2x P' - n(n+1) P."""
    P, dP = legendre(n, x)
    x = np.asarray(x, dtype=_LD)
    return (2 * x * dP - n * (n + 1) * P) / (1 - x * x)


def gauss_legendre(q):
    """q-point Gauss-Legendre rule on [0,1]: (points, weights), float64."""
    if q < 1:
        raise ValueError("q >= 1")
    k = np.arange(1, q + 1, dtype=_LD)
    x = -np.cos(_LD(np.pi) * (k - _LD(0.25)) / (q + _LD(0.5)))   # initial guesses, ascending
    for _ in range(100):
        P, dP = legendre(q, x)
        dx = P / dP
        x = x - dx
        if np.max(np.abs(dx)) < _LD(1e-30):
            break
    P, dP = legendre(q, x)
    w = 2 / ((1 - x * x) * dP * dP)
    pts = (x + 1) / 2
    wts = w / 2
    return pts.astype(np.float64), wts.astype(np.float64)


def gll_nodes(p):
    """The p+1 Gauss-Lobatto-Legendre nodes on [0,1], ascending, float64."""
    if p < 1:
        raise ValueError("p >= 1")
    if p == 1:
        return np.array([0.0, 1.0])
    k = np.arange(1, p, dtype=_LD)
    x = -np.cos(_LD(np.pi) * k / p)            # Chebyshev-Lobatto initial guesses
    for _ in range(100):
        _, dP = legendre(p, x)
        d2P = legendre_d2(p, x)
        dx = dP / d2P
        x = x - dx
        if np.max(np.abs(dx)) < _LD(1e-30):
            break
    x = np.concatenate([[_LD(-1)], x, [_LD(1)]])
    return ((x + 1) / 2).astype(np.float64)
