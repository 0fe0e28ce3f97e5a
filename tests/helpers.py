"""Shared helpers of the tests: oracle-side views of the product's stored layout.

The stored layout (cell c at [c*stride, (c+1)*stride), point (i,j,k) at
t_{n+1}(i,j,k)) is the one documented in include/hytet.h; the oracle side of
every helper here uses only ``oracle`` code and the paper's t_w.
"""
import numpy as np

from oracle import indexing as ix
from oracle.mesh import coord_key


def oracle_stored_to_canonical(macro, rm, stride):
    """Canonical (oracle) vertex id of every stored P1 slot; -1 for padding."""
    n = rm.n
    w = n + 1
    pts = np.array(ix.index_set_tet(w), dtype=np.int64)                # (N,3) i,j,k
    t = np.array([ix.tw(w, *p) for p in pts], dtype=np.int64)
    keys = coord_key(rm.coords, rm.side)
    out = np.full(stride * len(macro.cells), -1, dtype=np.int64)
    V = macro.vertices
    for c, cell in enumerate(macro.cells):
        X0, X1, X2, X3 = (V[cell[q]] for q in range(4))
        P = X0[None] * n + pts[:, :1] * (X1 - X0) + pts[:, 1:2] * (X2 - X0) + pts[:, 2:3] * (X3 - X0)
        out[c * stride + t] = np.searchsorted(keys, coord_key(P, rm.side))
    return out


def rel_err(a, b):
    a = np.asarray(a, dtype=np.float64)
    b = np.asarray(b, dtype=np.float64)
    den = np.abs(b).max()
    return np.abs(a - b).max() / (den if den > 0 else 1.0)
