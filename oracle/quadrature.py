"""Degree-5 triangle quadrature with seven points, derived from its moment
equations (oracle; test infrastructure only).

The rule is fully symmetric: the centroid plus two orbits of three points
with barycentric coordinates (a, a, 1-2a) and (b, b, 1-2b).  Its five unknowns
(three weights, a, b) are found by solving the exactness conditions on the
reference triangle {x >= 0, y >= 0, x + y <= 1} for all monomials of degree
<= 5 with a Gauss-Newton least-squares solve; exactness is then asserted on
every such monomial.  Nothing is taken from a printed table.
"""
from functools import lru_cache
from math import factorial

import numpy as np
from scipy.optimize import least_squares


def monomial_integral(i, j):
    """Exact integral of x^i y^j over the reference triangle: i! j! / (i+j+2)!."""
    return factorial(i) * factorial(j) / factorial(i + j + 2)


def _points(a, b):
    lam = [(1 / 3, 1 / 3, 1 / 3)]
    for t in (a, b):
        u = 1.0 - 2.0 * t
        lam += [(u, t, t), (t, u, t), (t, t, u)]
    lam = np.asarray(lam)
    # reference coordinates (x, y) = (lambda_1, lambda_2)
    return lam[:, 1:3], lam


def _weights(w0, wa, wb):
    return np.array([w0, wa, wa, wa, wb, wb, wb])


def _residual(z):
    w0, wa, wb, a, b = z
    xy, _ = _points(a, b)
    w = _weights(w0, wa, wb)
    res = []
    for d in range(6):
        for i in range(d + 1):
            j = d - i
            res.append(np.sum(w * xy[:, 0] ** i * xy[:, 1] ** j) - monomial_integral(i, j))
    return np.asarray(res)


@lru_cache(maxsize=None)
def triangle_rule_deg5():
    """Return (xy [7, 2], lam [7, 3], w [7]) on the reference triangle (area 1/2).

    Reference coordinates (x, y) map to barycentric (1-x-y, x, y).
    """
    sol = least_squares(_residual, x0=[0.1, 0.06, 0.06, 0.1, 0.45], xtol=1e-15, ftol=1e-15,
                        gtol=1e-15)
    w0, wa, wb, a, b = sol.x
    if a > b:
        a, b, wa, wb = b, a, wb, wa
    xy, lam = _points(a, b)
    w = _weights(w0, wa, wb)
    assert np.max(np.abs(_residual([w0, wa, wb, a, b]))) < 1e-15
    assert np.all(w > 0) and 0 < a < 0.5 and 0 < b < 0.5
    return xy, lam, w
