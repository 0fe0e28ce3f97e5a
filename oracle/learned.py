"""The learned smoothing step and its training samples (oracle, test infrastructure).

The paper has no learned component; the step extends its matrix-vector plus
diagonal smoothers (Sec. 5.2, Jacobi-type smoothing) by a local network N
(``oracle.mlp``) that reads the Jacobi-scaled residual s = D^-1 r around a
micro-vertex.  Written from the library's stated definition (the reading
taken where the paper is silent):

* s = r / D on the non-Dirichlet DoFs (D the diagonal of the assembled
  operator), 0 on the Dirichlet DoFs;
* at a vertex inside a macro cell (i, j, k >= 1, i + j + k <= n - 1), the
  features F are s at the vertex and at its 14 lattice neighbours in that
  cell's own lattice directions, in the order (0,0,0), (+1,0,0), (-1,0,0),
  (0,+1,0), (0,-1,0), (0,0,+1), (0,0,-1), (-1,+1,0), (+1,-1,0), (-1,0,+1),
  (+1,0,-1), (0,-1,+1), (0,+1,-1), (+1,-1,+1), (-1,+1,-1), then a 0;
* the step: x' = x + omega s + N(F) at those vertices, x + omega s at the
  other non-Dirichlet vertices, x at the Dirichlet vertices;
* a training sample at such a vertex: features F / |F| (the 15 values) and
  target (x* - x - omega s) / |F|, the samples taken at every stride-th
  cell-interior vertex in the order cell, then k, j, i.

Neighbours are found from exact integer coordinates (the vertex at
v0 + (i (v1-v0) + j (v2-v0) + k (v3-v0)) / n), independent of any storage
order.  Pinned by: a zero network gives the weighted Jacobi step; a network
that returns max(F_d, 0) reproduces s at the neighbour found from physical
coordinates, for every direction d and on cells listed in permuted vertex
order; positive homogeneity; unit-norm features (tests/test_oracle_learned.py).
"""
from __future__ import annotations

import numpy as np

from . import mlp as om
from .mesh import coord_key

DIRS = np.array([(0, 0, 0), (1, 0, 0), (-1, 0, 0), (0, 1, 0), (0, -1, 0), (0, 0, 1), (0, 0, -1),
                 (-1, 1, 0), (1, -1, 0), (-1, 0, 1), (1, 0, -1), (0, -1, 1), (0, 1, -1),
                 (1, -1, 1), (-1, 1, -1)], dtype=np.int64)


def cell_interior_points(n: int) -> np.ndarray:
    """(i, j, k) with i, j, k >= 1 and i + j + k <= n - 1, k slowest, then j, i."""
    return np.array([(i, j, k) for k in range(1, n) for j in range(1, n - k)
                     for i in range(1, n - k - j)], dtype=np.int64).reshape(-1, 3)


def vertex_ids(macro, rm, cell: int, pts: np.ndarray) -> np.ndarray:
    """Canonical ids of the cell-local lattice points pts (m,3) of macro cell `cell`."""
    V = np.asarray(macro.vertices, dtype=np.int64)
    X0, X1, X2, X3 = (V[q] for q in macro.cells[cell])
    P = X0[None] * rm.n + pts[:, :1] * (X1 - X0) + pts[:, 1:2] * (X2 - X0) + pts[:, 2:3] * (X3 - X0)
    keys = coord_key(rm.coords, rm.side)
    q = coord_key(P, rm.side)
    ids = np.searchsorted(keys, q)
    ids = np.minimum(ids, len(keys) - 1)
    if not np.array_equal(keys[ids], q):
        raise ValueError("point outside the refined mesh")
    return ids


def scaled_residual(rm, r: np.ndarray, D: np.ndarray) -> np.ndarray:
    """s = r / D on the non-Dirichlet vertices, 0 on the Dirichlet ones."""
    s = np.zeros(rm.n_vertices)
    ii = rm.interior
    s[ii] = r[ii] / D[ii]
    return s


def features(macro, rm, s: np.ndarray):
    """Per macro cell: (ids of the cell-interior vertices, features F (m,16))."""
    pts = cell_interior_points(rm.n)
    out = []
    for c in range(len(macro.cells)):
        ids = vertex_ids(macro, rm, c, pts)
        F = np.zeros((len(pts), 16))
        for d, off in enumerate(DIRS):
            F[:, d] = s[vertex_ids(macro, rm, c, pts + off[None])]
        out.append((ids, F))
    return out


def learned_step(macro, rm, x, r, D, W1, W2, w3, omega, forward=None):
    """One learned smoothing step; forward(W1, W2, w3, F) -> N(F) (default: exact FP64)."""
    fwd = forward or (lambda a, b, c, F: om.forward(a, b, c, F)[0])
    s = scaled_residual(rm, r, D)
    out = np.asarray(x, dtype=np.float64).copy()
    ii = rm.interior
    out[ii] = x[ii] + omega * s[ii]
    for ids, F in features(macro, rm, s):
        if len(ids):
            out[ids] += fwd(W1, W2, w3, F)
    return out


def learned_samples(macro, rm, r, D, xstar, x, omega, stride, offset):
    """Training samples (X (m,16), t (m,)) at the cell-interior vertices of rank
    q with q % stride == offset, rank counted cell by cell in (k, j, i) order."""
    s = scaled_residual(rm, r, D)
    Xs, ts = [], []
    for ids, F in features(macro, rm, s):
        nrm = np.sqrt((F[:, :15] ** 2).sum(axis=1))
        sc = np.where(nrm > 0, 1.0 / np.where(nrm > 0, nrm, 1.0), 0.0)
        Xs.append(F * sc[:, None])
        ts.append((xstar[ids] - x[ids] - omega * s[ids]) * sc)
    X = np.concatenate(Xs) if Xs else np.zeros((0, 16))
    t = np.concatenate(ts) if ts else np.zeros(0)
    q = np.arange(len(t))
    keep = q % stride == offset
    return X[keep], t[keep]
