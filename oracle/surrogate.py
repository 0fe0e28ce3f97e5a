"""Polynomial surrogate stencils for the variable-coefficient P1 operator
(Sec. 5.2, surrogates): on a structured macro cell the stencil entries of
-div(k grad) vary smoothly with the position when k does, so each entry is
replaced by a low-degree polynomial in the lattice coordinates.

ORACLE: test infrastructure only.  tests/, the smoke check and the bench's
CPU baseline may use it; the product path never does.

Definitions, written out plainly:
* The exact operator A is the assembled P1 -div(k grad) matrix (k_T = mean of
  the vertex values, ``fem.p1_divkgrad``).
* At a point (i, j, k) inside macro cell c (no macro face, edge or vertex)
  the stencil weight of direction d (the 15 lattice directions) is the matrix
  entry A[p, p + d].
* Per macro cell and direction, the weights at all interior points are
  fitted by least squares with the monomials (i/n)^a (j/n)^b (k/n)^c,
  a + b + c <= degree (``numpy.linalg.lstsq``).
* The surrogate operator uses the fitted polynomial at interior points and
  the exact rows of A at all other points.

Parity: pinned by exact reproduction of A for a coefficient linear in x
(the weights are then affine in the position, so degree 1 is exact) and for a
constant coefficient with degree 0, and by the error falling with the degree
for a smooth coefficient.
"""
from __future__ import annotations

import itertools

import numpy as np
import scipy.sparse as sp

from . import fem
from .mesh import RefinedMesh, coord_key

DIRS = np.array([[0, 0, 0], [1, 0, 0], [-1, 0, 0], [0, 1, 0], [0, -1, 0], [0, 0, 1], [0, 0, -1],
                 [-1, 1, 0], [1, -1, 0], [-1, 0, 1], [1, 0, -1], [0, -1, 1], [0, 1, -1],
                 [1, -1, 1], [-1, 1, -1]])


def exponents(degree):
    return [e for e in itertools.product(range(degree + 1), repeat=3) if sum(e) <= degree]


class SurrogateLevel:
    """Exact div-k-grad operator of one level and its per-cell surrogate data."""

    def __init__(self, macro, level, kfun):
        self.rm = rm = RefinedMesh(macro, level)
        self.macro = macro
        self.n = n = rm.n
        kv = kfun(rm.xyz)[rm.cells]
        self.A = fem.assemble(rm.cells, fem.p1_divkgrad(rm.cell_xyz, kv), rm.n_vertices).tocsr()
        keys = coord_key(rm.coords, rm.side)
        # interior lattice points of each cell and the global ids of them and their neighbours
        ijk = np.array([(i, j, k) for k in range(1, n) for j in range(1, n - k)
                        for i in range(1, n - k - j)], dtype=np.int64).reshape(-1, 3)
        self.ijk = ijk
        self.cells = []
        for cell in macro.cells:
            V = macro.vertices[cell]
            E = np.stack([V[1] - V[0], V[2] - V[0], V[3] - V[0]])

            def gid(p):
                kk = coord_key((V[0] << level) + p @ E, rm.side)
                idx = np.searchsorted(keys, kk)
                assert np.array_equal(keys[idx], kk)
                return idx
            ids = gid(ijk)
            nb = np.stack([gid(ijk + d) for d in DIRS], axis=1)       # (P, 15)
            sub = self.A[ids[:, None], nb]                            # exact weights
            w = sub.toarray() if sp.issparse(sub) else np.asarray(sub)
            self.cells.append((ids, nb, w))

    def surrogate(self, degree):
        """The surrogate matrix: fitted weights at cell-interior points, exact
        rows elsewhere."""
        ex = exponents(degree)
        u = self.ijk / self.n
        B = np.stack([u[:, 0] ** a * u[:, 1] ** b * u[:, 2] ** c for a, b, c in ex], axis=1)
        A = self.A.tolil(copy=True)
        for ids, nb, w in self.cells:
            coef, *_ = np.linalg.lstsq(B, w, rcond=None)               # (terms, 15)
            ws = B @ coef
            for d in range(len(DIRS)):
                A[ids, nb[:, d]] = ws[:, d]
        return A.tocsr()
