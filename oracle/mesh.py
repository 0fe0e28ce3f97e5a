"""Refined meshes in exact integer coordinates (oracle, test infrastructure).

* ``bey_children``/``refine``: Bey's regular refinement (Sec. 3.1, the rule
  T -> T1..T8 built from the vertices and edge midpoints), applied
  recursively L times to every macro cell.  Coordinates are scaled by 2^L so
  every midpoint is an exact integer.
* ``lattice_cells``: an independent enumeration of the same micro-cells as
  six translation-invariant subgroups (Sec. 3.2): anchors p with |p| < w and
  fixed vertex offsets.  Used only to pin ``refine`` (set equality).
* ``number_vertices``: global numbering of micro-vertices by their exact
  integer coordinates; canonical order is ascending key with
  key = X + S*(Y + S*Z), i.e. z slowest, x fastest.
* ``dirichlet_vertices``: vertices on the domain boundary, found as the
  vertices of micro-faces that belong to exactly one micro-cell.

Parity: pinned by set equality of Bey vs lattice cells, 8^L cells per macro
cell, (n+1)(n+2)(n+3)/6 vertices per macro cell, (m n + 1)^3 vertices of a
Kuhn cube, and the Euler characteristic of one refined tetrahedron.
"""
from __future__ import annotations

import numpy as np

E1 = np.array([1, 0, 0])
E2 = np.array([0, 1, 0])
E3 = np.array([0, 0, 1])


def bey_children(t: np.ndarray) -> np.ndarray:
    """Split tetrahedra t (T,4,3) into their 8 Bey children (8T,4,3).

    With v_ij the midpoint of v_i v_j:
      T1=[v0,v01,v02,v03]  T2=[v01,v1,v12,v13]  T3=[v02,v12,v2,v23]
      T4=[v03,v13,v23,v3]  T5=[v01,v02,v03,v13] T6=[v01,v02,v12,v13]
      T7=[v02,v03,v13,v23] T8=[v02,v12,v13,v23]
    """
    v0, v1, v2, v3 = t[:, 0], t[:, 1], t[:, 2], t[:, 3]
    if np.any((v0 + v1) % 2) or np.any((v0 + v2) % 2) or np.any((v1 + v3) % 2):
        raise ValueError("coordinates not even: scale by 2^L before refining")
    m01, m02, m03 = (v0 + v1) // 2, (v0 + v2) // 2, (v0 + v3) // 2
    m12, m13, m23 = (v1 + v2) // 2, (v1 + v3) // 2, (v2 + v3) // 2
    kids = [
        (v0, m01, m02, m03),
        (m01, v1, m12, m13),
        (m02, m12, v2, m23),
        (m03, m13, m23, v3),
        (m01, m02, m03, m13),
        (m01, m02, m12, m13),
        (m02, m03, m13, m23),
        (m02, m12, m13, m23),
    ]
    out = np.stack([np.stack(k, axis=1) for k in kids], axis=1)  # (T,8,4,3)
    return out.reshape(-1, 4, 3)


def refine(vertices: np.ndarray, cells: np.ndarray, level: int) -> np.ndarray:
    """Micro-cells of all macro cells after `level` recursive Bey steps.

    Returns int64 (nc * 8^level, 4, 3) in integer coordinates scaled by
    2^level; micro-cells of macro cell c occupy rows [c*8^L, (c+1)*8^L).
    """
    t = (np.asarray(vertices, dtype=np.int64)[np.asarray(cells)] << level)
    for _ in range(level):
        t = bey_children(t)
    return t


def lattice_cells(n: int) -> np.ndarray:
    """Micro-cells of the reference tetrahedron with n intervals per edge.

    Six subgroups, anchors p=(i,j,k) with i+j+k < w (Sec. 3.2, Table 1):
      I-up   (w=n)  : [p, p+e1, p+e2, p+e3]
      I-down (w=n-2): [p+e1+e2, p+e1+e3, p+e2+e3, p+e1+e2+e3]
      four cells of the octahedron (w=n-1), all containing the inner edge
      p+e2 -- p+e1+e3, with the pairs (p+e1,p+e3), (p+e3,p+e2+e3),
      (p+e2+e3,p+e1+e2), (p+e1+e2,p+e1).
    Returns integer coordinates in lattice units (T,4,3).
    """
    def anchors(w):
        return np.array([(i, j, k) for k in range(max(w, 0)) for j in range(w - k)
                         for i in range(w - k - j)], dtype=np.int64).reshape(-1, 3)

    def build(w, offs):
        a = anchors(w)
        return np.stack([a + o for o in offs], axis=1) if len(a) else np.zeros((0, 4, 3), np.int64)

    z = np.zeros(3, dtype=np.int64)
    groups = [
        build(n, [z, E1, E2, E3]),
        build(n - 2, [E1 + E2, E1 + E3, E2 + E3, E1 + E2 + E3]),
        build(n - 1, [E2, E1 + E3, E1, E3]),
        build(n - 1, [E2, E1 + E3, E3, E2 + E3]),
        build(n - 1, [E2, E1 + E3, E2 + E3, E1 + E2]),
        build(n - 1, [E2, E1 + E3, E1 + E2, E1]),
    ]
    return np.concatenate(groups, axis=0)


def coord_key(xyz_int: np.ndarray, side: int) -> np.ndarray:
    """Integer key X + S*(Y + S*Z) with S = side+1; ascending key = z slowest."""
    s = np.int64(side + 1)
    x = np.asarray(xyz_int, dtype=np.int64)
    return x[..., 0] + s * (x[..., 1] + s * x[..., 2])


def number_vertices(micro: np.ndarray):
    """Unique micro-vertices in canonical order.

    Returns (coords (N,3) int64, cell_vertex_ids (T,4) int64, side) where
    ``side`` is the largest coordinate value (keys use S = side+1).
    """
    side = int(micro.max())
    keys = coord_key(micro.reshape(-1, 3), side)
    uniq, inv = np.unique(keys, return_inverse=True)
    s = side + 1
    coords = np.stack([uniq % s, (uniq // s) % s, uniq // (s * s)], axis=1)
    return coords, inv.reshape(micro.shape[0], 4), side


def faces_of(cell_ids: np.ndarray) -> np.ndarray:
    """All 4 faces of every cell as sorted vertex-id triples (4T,3)."""
    f = cell_ids[:, [[1, 2, 3], [0, 2, 3], [0, 1, 3], [0, 1, 2]]].reshape(-1, 3)
    return np.sort(f, axis=1)


def edges_of(cell_ids: np.ndarray) -> np.ndarray:
    """All 6 edges of every cell as sorted vertex-id pairs (6T,2)."""
    e = cell_ids[:, [[0, 1], [0, 2], [0, 3], [1, 2], [1, 3], [2, 3]]].reshape(-1, 2)
    return np.sort(e, axis=1)


def dirichlet_vertices(cell_ids: np.ndarray, n_vertices: int) -> np.ndarray:
    """Boolean mask of vertices lying on a micro-face owned by one cell only."""
    f = faces_of(cell_ids)
    uf, cnt = np.unique(f, axis=0, return_counts=True)
    mask = np.zeros(n_vertices, dtype=bool)
    mask[uf[cnt == 1].ravel()] = True
    return mask


class RefinedMesh:
    """A macro mesh refined to one level, with canonical vertex numbering."""

    def __init__(self, macro, level: int):
        self.macro = macro
        self.level = level
        self.n = 2 ** level
        self.micro = refine(macro.vertices, macro.cells, level)        # (T,4,3)
        self.coords, self.cells, self.side = number_vertices(self.micro)
        # physical coordinates: integer / (scale * 2^level)
        self.denom = macro.scale * self.n
        self.xyz = self.coords.astype(np.float64) / self.denom
        self.n_vertices = len(self.coords)
        self.boundary = dirichlet_vertices(self.cells, self.n_vertices)
        self.interior = np.flatnonzero(~self.boundary)

    @property
    def cell_xyz(self) -> np.ndarray:
        """Physical vertex coordinates of every micro-cell (T,4,3)."""
        return self.micro.astype(np.float64) / self.denom
