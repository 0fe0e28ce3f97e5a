"""Quadrature on a tetrahedron in barycentric coordinates (oracle, test infrastructure).

* ``exact_monomial``: the closed form of the integral of a barycentric
  monomial, int_T prod lam_i^a_i = |T| 3! prod(a_i!) / (|a|+3)!.
* ``sym14``: the symmetric 14-point, degree-5, positive-weight rule (orbits
  4+4+6; published e.g. by Walkington, "Quadrature on simplices of arbitrary
  dimension", 2000).  The oracle does not copy a table: it solves the six
  symmetric moment equations for degree <= 5 by Newton's method, starting
  from rounded published values, so the rule is fixed by the mathematics.
* ``stroud_conical``: the conical-product (collapsed Gauss-Jacobi) rule of
  Stroud with q^3 points and degree 2q-1; used only to bound the
  quadrature error of ``sym14`` on smooth coefficients.

The paper only names its forms by quadrature order (Sec. 5.2, operator
examples) and gives no rule; the variable-coefficient P2 operator here uses
``sym14`` on both sides.  Pinned by exactness on all monomials of degree <= 5
(sym14) and <= 2q-1 (conical rule) against ``exact_monomial``.
"""
from __future__ import annotations

import itertools
import math

import numpy as np
from scipy.optimize import fsolve
from scipy.special import roots_jacobi


def exact_monomial(alpha) -> float:
    """Integral of prod lam_i^alpha_i over a tetrahedron of unit volume."""
    s = sum(alpha)
    return 6.0 * math.prod(math.factorial(a) for a in alpha) / math.factorial(s + 3)


def _orbit4(a):
    return [tuple(1.0 - 3.0 * a if i == j else a for i in range(4)) for j in range(4)]


def _orbit6(a):
    b = 0.5 - a
    return sorted(set(itertools.permutations([a, a, b, b])))


def _sym14_points(p):
    w1, a1, w2, a2, w3, a3 = p
    pts = [(w1, q) for q in _orbit4(a1)] + [(w2, q) for q in _orbit4(a2)] + \
          [(w3, q) for q in _orbit6(a3)]
    return pts


_SYM14_START = (0.07349304311636, 0.09273525031089, 0.11268792571802,
                0.31088591926330, 0.04254602077708, 0.45449629587435)
# one monomial per symmetric invariant of degree 0, 2, 3, 4, 4, 5
_SYM14_EQ = [(0, 0, 0, 0), (2, 0, 0, 0), (3, 0, 0, 0), (4, 0, 0, 0), (2, 2, 0, 0), (5, 0, 0, 0)]


def sym14():
    """Return (bary (14,4), weights (14,)) with weights summing to 1."""
    def resid(p):
        pts = _sym14_points(p)
        return [sum(w * np.prod([q[i] ** al[i] for i in range(4)]) for w, q in pts)
                - exact_monomial(al) for al in _SYM14_EQ]
    p = fsolve(resid, _SYM14_START, xtol=1e-14)
    pts = _sym14_points(p)
    bary = np.array([q for _, q in pts], dtype=np.float64)
    w = np.array([w for w, _ in pts], dtype=np.float64)
    return bary, w


def stroud_conical(q: int):
    """Conical product rule with q^3 points, exact for degree 2q-1.

    Collapsed coordinates: Gauss-Jacobi(2,0), (1,0), (0,0) on [0,1].
    Returns (bary (q^3,4), weights summing to 1).
    """
    def gj(a):
        x, w = roots_jacobi(q, a, 0.0)          # on [-1,1], weight (1-x)^a
        return (x + 1.0) / 2.0, w / 2.0 ** (a + 1)
    x1, w1 = gj(2.0)
    x2, w2 = gj(1.0)
    x3, w3 = gj(0.0)
    bary, wts = [], []
    for a, wa in zip(x1, w1):
        for b, wb in zip(x2, w2):
            for c, wc in zip(x3, w3):
                s = a
                t = (1.0 - a) * b
                u = (1.0 - a) * (1.0 - b) * c
                bary.append((1.0 - s - t - u, s, t, u))
                wts.append(wa * wb * wc)
    wts = np.array(wts) * 6.0
    return np.array(bary), wts
