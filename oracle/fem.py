"""Textbook element matrices and assembly (oracle, test infrastructure).

Element-wise operator evaluation is the sum over elements of local matrices
(Sec. 5.2, element-wise pattern: a_ij = sum_T int_T grad phi_i . grad phi_j);
here the local matrices are assembled once into a global CSR matrix
(COO -> CSR, duplicates summed) and the matrix-vector product is SciPy's
CSR SpMV.

* P1 stiffness  K_T = |T| G G^T, G = gradients of the barycentric functions.
* P1 mass       M_T = |T|/20 (1 + delta_ij).
* P1 div-k-grad K_T = k_T |T| G G^T with k_T the mean of the 4 vertex values
  (exact integral of k grad phi_i . grad phi_j for P1-interpolated k).
* P2 (vertex + edge DoFs; local order v0..v3, e01,e02,e03,e12,e13,e23)
  stiffness with coefficient k(x):  sum_q w_q |T| k(x_q) grad phi_i . grad phi_j
  at the points of a fixed rule (``quadrature.sym14``); P2 mass by the exact
  barycentric-monomial integrals.

Parity: pinned by symmetry, zero row sums of the Neumann matrices, the
linear patch test, 1^T M 1 = |Omega|, the closed-form reference-tetrahedron
stencil, and the 7-point identity on Kuhn cubes (tests).
"""
from __future__ import annotations

import numpy as np
import scipy.sparse as sp

from . import quadrature

P2_EDGES = ((0, 1), (0, 2), (0, 3), (1, 2), (1, 3), (2, 3))


def jacobian(X: np.ndarray):
    """J = [x1-x0, x2-x0, x3-x0] (columns) for tetrahedra X (T,4,3)."""
    return np.stack([X[:, 1] - X[:, 0], X[:, 2] - X[:, 0], X[:, 3] - X[:, 0]], axis=2)


def bary_gradients(X: np.ndarray):
    """(G (T,4,3), vol (T,)) with G[t,i] = grad lambda_i on tetrahedron t."""
    J = jacobian(X)
    Jinv = np.linalg.inv(J)                  # rows of J^-1 are grad lambda_1..3
    G = np.empty((X.shape[0], 4, 3))
    G[:, 1:] = Jinv
    G[:, 0] = -Jinv.sum(axis=1)
    vol = np.abs(np.linalg.det(J)) / 6.0
    return G, vol


def p1_stiffness(X: np.ndarray) -> np.ndarray:
    G, vol = bary_gradients(X)
    return vol[:, None, None] * np.einsum("tid,tjd->tij", G, G)


def p1_mass(X: np.ndarray) -> np.ndarray:
    _, vol = bary_gradients(X)
    base = (np.ones((4, 4)) + np.eye(4)) / 20.0
    return vol[:, None, None] * base[None]


def p1_divkgrad(X: np.ndarray, k_vertex: np.ndarray) -> np.ndarray:
    """k_vertex (T,4): coefficient values at the 4 vertices of each cell."""
    kT = k_vertex.mean(axis=1)
    return kT[:, None, None] * p1_stiffness(X)


def p2_basis_gradients(lam: np.ndarray, G: np.ndarray) -> np.ndarray:
    """Gradients of the 10 P2 basis functions at barycentric point lam (4,).

    vertex i: lam_i (2 lam_i - 1) -> (4 lam_i - 1) grad lam_i
    edge ij : 4 lam_i lam_j       -> 4 (lam_i grad lam_j + lam_j grad lam_i)
    G: (T,4,3).  Returns (T,10,3).
    """
    B = np.empty((G.shape[0], 10, 3))
    for i in range(4):
        B[:, i] = (4.0 * lam[i] - 1.0) * G[:, i]
    for e, (i, j) in enumerate(P2_EDGES):
        B[:, 4 + e] = 4.0 * (lam[i] * G[:, j] + lam[j] * G[:, i])
    return B


def p2_stiffness(X: np.ndarray, kfun=None, rule=None) -> np.ndarray:
    """P2 stiffness with coefficient kfun(points (T,3)) by the given rule."""
    bary, w = quadrature.sym14() if rule is None else rule
    G, vol = bary_gradients(X)
    K = np.zeros((X.shape[0], 10, 10))
    for lam, wq in zip(bary, w):
        B = p2_basis_gradients(lam, G)
        xq = np.einsum("i,tid->td", lam, X)
        kq = np.ones(X.shape[0]) if kfun is None else kfun(xq)
        K += (wq * vol * kq)[:, None, None] * np.einsum("tid,tjd->tij", B, B)
    return K


def _p2_basis_poly():
    """P2 basis functions as {monomial exponent tuple: coefficient}."""
    def mono(*idx):
        a = [0, 0, 0, 0]
        for i in idx:
            a[i] += 1
        return tuple(a)
    basis = []
    for i in range(4):
        basis.append({mono(i, i): 2.0, mono(i): -1.0})
    for (i, j) in P2_EDGES:
        basis.append({mono(i, j): 4.0})
    return basis


def p2_mass_reference() -> np.ndarray:
    """P2 mass matrix of a unit-volume tetrahedron, exact monomial integrals."""
    basis = _p2_basis_poly()
    M = np.zeros((10, 10))
    for a in range(10):
        for b in range(10):
            s = 0.0
            for ma, ca in basis[a].items():
                for mb, cb in basis[b].items():
                    s += ca * cb * quadrature.exact_monomial(tuple(x + y for x, y in zip(ma, mb)))
            M[a, b] = s
    return M


def p2_mass(X: np.ndarray) -> np.ndarray:
    _, vol = bary_gradients(X)
    return vol[:, None, None] * p2_mass_reference()[None]


def assemble(dofs: np.ndarray, Ke: np.ndarray, n: int) -> sp.csr_matrix:
    """Global CSR from element matrices Ke (T,m,m) on element DoFs (T,m)."""
    m = dofs.shape[1]
    rows = np.repeat(dofs, m, axis=1).ravel()
    cols = np.tile(dofs, (1, m)).ravel()
    return sp.coo_matrix((Ke.ravel(), (rows, cols)), shape=(n, n)).tocsr()


class P2Numbering:
    """P2 DoFs (micro-vertices and micro-edge midpoints) in canonical order.

    Keys use doubled integer coordinates: a vertex X maps to 2X and an edge
    (X_a, X_b) to X_a + X_b; canonical order is ascending key, z slowest.
    """

    def __init__(self, rm):
        from .mesh import coord_key
        micro = rm.micro
        pts_v = 2 * micro                                       # (T,4,3)
        pts_e = np.stack([micro[:, i] + micro[:, j] for i, j in P2_EDGES], axis=1)
        pts = np.concatenate([pts_v, pts_e], axis=1)            # (T,10,3)
        side = 2 * rm.side
        keys = coord_key(pts.reshape(-1, 3), side)
        uniq, inv = np.unique(keys, return_inverse=True)
        s = side + 1
        self.coords2 = np.stack([uniq % s, (uniq // s) % s, uniq // (s * s)], axis=1)
        self.dofs = inv.reshape(-1, 10)
        self.n = len(uniq)
        self.xyz = self.coords2.astype(np.float64) / (2 * rm.denom)
        # boundary: P2 DoFs on boundary micro-faces (vertices and face edges)
        bmask = np.zeros(self.n, dtype=bool)
        from .mesh import faces_of
        fv = faces_of(rm.cells)
        uf, cnt = np.unique(fv, axis=0, return_counts=True)
        bf = uf[cnt == 1]
        bpts = np.concatenate([
            2 * rm.coords[bf].reshape(-1, 3),
            rm.coords[bf[:, 0]] + rm.coords[bf[:, 1]],
            rm.coords[bf[:, 0]] + rm.coords[bf[:, 2]],
            rm.coords[bf[:, 1]] + rm.coords[bf[:, 2]],
        ], axis=0)
        bk = coord_key(bpts, side)
        bmask[np.searchsorted(uniq, np.unique(bk))] = True
        self.boundary = bmask
        self.interior = np.flatnonzero(~bmask)
