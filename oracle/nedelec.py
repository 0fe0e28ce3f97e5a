"""Lowest-order Nedelec edge elements of the first kind for the curl-curl
problem  alpha curl curl u + beta u = f in Omega,  u x n = 0 on the boundary
(Sec. 6, Nedelec elements for the curl-curl problem).

ORACLE: test infrastructure only.  tests/, the smoke check and the bench's
CPU baseline may use it; the product path never does.

The standard Whitney-form construction the paper cites, written out from the
definitions on SciPy matrices:
* DoFs: one per micro-edge e = (a, b), oriented from the endpoint with the
  smaller canonical vertex id to the larger; the DoF of a field u is the
  tangential line integral  u_e = int_0^1 u(x_a + s (x_b - x_a)) . (x_b - x_a) ds.
* Basis: w_e = lam_a grad lam_b - lam_b grad lam_a (barycentric lam),
  curl w_e = 2 grad lam_a x grad lam_b.
* Element matrices: curl-curl K_ef = |T| curl w_e . curl w_f; mass
  M_ef = int_T w_e . w_f expanded into int_T lam_i lam_j = |T| (1 + d_ij) / 20.
  Local edges (0,1),(0,2),(0,3),(1,2),(1,3),(2,3) run from the lower to the
  higher local vertex; a sign per (cell, local edge) maps them to the global
  orientation.
* Numbering: one DoF per unique micro-edge, keyed by the midpoint on the
  doubled lattice (the same keys as the P2 edge DoFs), ascending.  Boundary
  DoFs (u x n = 0): edges of micro-faces owned by one cell.
* Discrete gradient G (edges x vertices): (G phi)_e = phi_b - phi_a, the
  exact N1 representation of grad phi for P1 phi.
* Prolongation between levels: fine DoF = tangential line integral of the
  coarse N1 function, evaluated inside one coarse cell that contains the fine
  edge (exact: the coarse function is linear there); by grad lam . (x_q - x_p)
  = lam(q) - lam(p) the weights are rational in the barycentric coordinates.
* Hiptmair's hybrid smoother (Sec. 6): one smoothing step on A, the
  residual taken to the potential space by G^T, one smoothing step with the
  potential-space operator A_p = G^T A G (= beta times the P1 Laplacian for
  this A), and the correction G e_p added.  V(nu1, nu2) cycles with an exact
  coarsest solve; full multigrid as in ``gmg.fmg``.

Parity: pinned by pointwise reproduction of constant and rotational fields
c x x by the basis, finite-difference curls of the basis, a quadrature check
of the mass matrix, curl-curl G = 0, G^T M G = the P1 stiffness matrix, the
energies of interpolated constant and rotational fields, the commuting
relation P G_c = G_f P_1 of the transfers, the null-space dimension of the
curl-curl matrix, O(h) decay of the L2 interpolation error, and
level-independent convergence of the Hiptmair V-cycle.
"""
from __future__ import annotations

import numpy as np
import scipy.linalg as sla
import scipy.sparse as sp

from . import fem, gmg
from .mesh import RefinedMesh, bey_children, coord_key, faces_of

LOCAL_EDGES = fem.P2_EDGES


def whitney(lam: np.ndarray, G: np.ndarray) -> np.ndarray:
    """Whitney basis values w_e(x) = lam_a grad lam_b - lam_b grad lam_a in
    local orientation.  lam (..., 4), G (4, 3) -> (..., 6, 3)."""
    out = np.empty(lam.shape[:-1] + (6, 3))
    for e, (a, b) in enumerate(LOCAL_EDGES):
        out[..., e, :] = lam[..., a, None] * G[b] - lam[..., b, None] * G[a]
    return out


def whitney_curls(G: np.ndarray) -> np.ndarray:
    """curl w_e = 2 grad lam_a x grad lam_b.  G (T, 4, 3) -> (T, 6, 3)."""
    return np.stack([2.0 * np.cross(G[:, a], G[:, b]) for a, b in LOCAL_EDGES], axis=1)


def curlcurl_local(X: np.ndarray) -> np.ndarray:
    G, vol = fem.bary_gradients(X)
    C = whitney_curls(G)
    return vol[:, None, None] * np.einsum("tid,tjd->tij", C, C)


def mass_local(X: np.ndarray) -> np.ndarray:
    G, vol = fem.bary_gradients(X)
    GG = np.einsum("tid,tjd->tij", G, G)
    L = (np.ones((4, 4)) + np.eye(4)) / 20.0          # int lam_i lam_j / |T|
    M = np.empty((X.shape[0], 6, 6))
    for e, (a, b) in enumerate(LOCAL_EDGES):
        for f, (c, d) in enumerate(LOCAL_EDGES):
            M[:, e, f] = (L[a, c] * GG[:, b, d] - L[a, d] * GG[:, b, c]
                          - L[b, c] * GG[:, a, d] + L[b, d] * GG[:, a, c])
    return vol[:, None, None] * M


# 5-point Gauss-Legendre rule on [0, 1] (exact to degree 9) for line integrals
_GL_X, _GL_W = np.polynomial.legendre.leggauss(5)
_GL_X = 0.5 * (_GL_X + 1.0)
_GL_W = 0.5 * _GL_W


class NedelecLevel:
    """N1 space, matrices and discrete gradient on one refinement level."""

    def __init__(self, macro, level: int, alpha: float = 1.0, beta: float = 1.0):
        self.rm = rm = RefinedMesh(macro, level)
        self.alpha, self.beta = alpha, beta
        ids = rm.cells
        va = ids[:, [a for a, _ in LOCAL_EDGES]]
        vb = ids[:, [b for _, b in LOCAL_EDGES]]
        self.sign = np.where(va < vb, 1.0, -1.0)                  # local -> global orientation
        side = 2 * rm.side
        mid2 = rm.coords[va] + rm.coords[vb]                       # doubled-lattice midpoints
        self.keys, inv = np.unique(coord_key(mid2.reshape(-1, 3), side), return_inverse=True)
        self.dofs = inv.reshape(-1, 6)
        self.n = len(self.keys)
        self.ends = np.empty((self.n, 2), dtype=np.int64)
        self.ends[inv, 0] = np.minimum(va, vb).ravel()
        self.ends[inv, 1] = np.maximum(va, vb).ravel()
        fv = faces_of(ids)
        uf, cnt = np.unique(fv, axis=0, return_counts=True)
        bf = uf[cnt == 1]
        c = rm.coords
        bmid = np.concatenate([c[bf[:, 0]] + c[bf[:, 1]], c[bf[:, 0]] + c[bf[:, 2]],
                               c[bf[:, 1]] + c[bf[:, 2]]], axis=0)
        self.boundary = np.zeros(self.n, dtype=bool)
        self.boundary[np.searchsorted(self.keys, np.unique(coord_key(bmid, side)))] = True
        self.interior = np.flatnonzero(~self.boundary)
        X = rm.cell_xyz
        S = self.sign[:, :, None] * self.sign[:, None, :]
        self.K_full = fem.assemble(self.dofs, curlcurl_local(X) * S, self.n)
        self.M_full = fem.assemble(self.dofs, mass_local(X) * S, self.n)
        self.A_full = alpha * self.K_full + beta * self.M_full
        ii = self.interior
        self.A = self.A_full[ii][:, ii].tocsr()
        self.D = self.A.diagonal()
        e = np.arange(self.n)
        self.G_full = sp.coo_matrix(
            (np.concatenate([-np.ones(self.n), np.ones(self.n)]),
             (np.concatenate([e, e]), np.concatenate([self.ends[:, 0], self.ends[:, 1]]))),
            shape=(self.n, rm.n_vertices)).tocsr()
        self.Gi = self.G_full[ii][:, rm.interior].tocsr()
        self.Ap = (self.Gi.T @ self.A @ self.Gi).tocsr()
        self.Dp = self.Ap.diagonal()

    def interpolate(self, u) -> np.ndarray:
        """Edge DoFs of the field u (callable (N,3) -> (N,3)): tangential line
        integrals by the 5-point Gauss rule."""
        xa = self.rm.xyz[self.ends[:, 0]]
        xb = self.rm.xyz[self.ends[:, 1]]
        t = xb - xa
        out = np.zeros(self.n)
        for s, w in zip(_GL_X, _GL_W):
            out += w * np.einsum("nd,nd->n", u(xa + s * t), t)
        return out

    def evaluate(self, x: np.ndarray, lam: np.ndarray) -> np.ndarray:
        """Values of the N1 function with DoFs x at barycentric points lam (Q, 4)
        of every micro-cell: (T, Q, 3)."""
        G, _ = fem.bary_gradients(self.rm.cell_xyz)
        coef = x[self.dofs] * self.sign                            # (T, 6) local DoFs
        out = np.zeros((len(G), len(lam), 3))
        for e, (a, b) in enumerate(LOCAL_EDGES):
            w = lam[None, :, a, None] * G[:, None, b] - lam[None, :, b, None] * G[:, None, a]
            out += coef[:, e, None, None] * w
        return out

    def load_vector(self, f, rule) -> np.ndarray:
        """b_e = int f . w_e by the given tetrahedron rule (bary (Q,4), weights (Q,), sum 1)."""
        bary, wq = rule
        X = self.rm.cell_xyz
        G, vol = fem.bary_gradients(X)
        pts = np.einsum("qi,tid->tqd", bary, X)
        fv = f(pts.reshape(-1, 3)).reshape(pts.shape)              # (T, Q, 3)
        be = np.zeros((len(X), 6))
        for e, (a, b) in enumerate(LOCAL_EDGES):
            w = bary[None, :, a, None] * G[:, None, b] - bary[None, :, b, None] * G[:, None, a]
            be[:, e] = vol * np.einsum("q,tqd,tqd->t", wq, fv, w)
        out = np.zeros(self.n)
        np.add.at(out, self.dofs.ravel(), (be * self.sign).ravel())
        return out


def _bey_fine_edges():
    """The 25 fine edges inside one coarse cell, as pairs of doubled
    barycentric coordinates (4 integers summing to 2)."""
    ref = np.array([[[0, 0, 0], [2, 0, 0], [0, 2, 0], [0, 0, 2]]], dtype=np.int64)
    kids = bey_children(ref)                                        # (8, 4, 3)
    lam = np.concatenate([2 - kids.sum(axis=2, keepdims=True), kids], axis=2)   # (8, 4, 4)
    pairs = set()
    for k in lam:
        for a, b in LOCAL_EDGES:
            p, q = tuple(k[a]), tuple(k[b])
            pairs.add((min(p, q), max(p, q)))
    return sorted(pairs)


def nedelec_prolongation(fine: NedelecLevel, coarse: NedelecLevel) -> sp.csr_matrix:
    """Coarse N1 functions' tangential line integrals over the fine edges."""
    cm = coarse.rm.micro                       # (Tc, 4, 3) coarse integer coords
    fkeys_v = coord_key(fine.rm.coords, fine.rm.side)
    Gc_sign = coarse.sign
    rows, cols, vals = [], [], []
    for p2, q2 in _bey_fine_edges():
        p2 = np.array(p2)
        q2 = np.array(q2)
        Xp = np.einsum("i,tid->td", p2, cm)    # fine integer coords (fine = 2 x coarse units)
        Xq = np.einsum("i,tid->td", q2, cm)
        fe = np.searchsorted(fine.keys, coord_key(Xp + Xq, 2 * fine.rm.side))
        idp = np.searchsorted(fkeys_v, coord_key(Xp, fine.rm.side))
        idq = np.searchsorted(fkeys_v, coord_key(Xq, fine.rm.side))
        flip = np.where(idp < idq, 1.0, -1.0)  # global fine orientation p -> q or q -> p
        lp, lq = p2 / 2.0, q2 / 2.0
        lm = 0.5 * (lp + lq)
        for e, (a, b) in enumerate(LOCAL_EDGES):
            w = lm[a] * (lq[b] - lp[b]) - lm[b] * (lq[a] - lp[a])
            if w == 0.0:
                continue
            rows.append(fe)
            cols.append(coarse.dofs[:, e])
            vals.append(w * flip * Gc_sign[:, e])
    r = np.concatenate(rows)
    c = np.concatenate(cols)
    v = np.concatenate(vals)
    key = r.astype(np.int64) * coarse.n + c
    _, first = np.unique(key, return_index=True)
    return sp.coo_matrix((v[first], (r[first], c[first])), shape=(fine.n, coarse.n)).tocsr()


class NedelecHierarchy:
    """Levels lmin..lmax with interior N1 prolongations."""

    def __init__(self, macro, lmin, lmax, alpha=1.0, beta=1.0):
        self.lmin, self.lmax = lmin, lmax
        self.levels = {l: NedelecLevel(macro, l, alpha, beta) for l in range(lmin, lmax + 1)}
        self.P = {}
        for l in range(lmin + 1, lmax + 1):
            f, c = self.levels[l], self.levels[l - 1]
            self.P[l] = nedelec_prolongation(f, c)[f.interior][:, c.interior].tocsr()
        cA = self.levels[lmin].A.toarray()
        self.coarse_chol = sla.cho_factor(cA) if cA.size else None


def hiptmair_step(lev: NedelecLevel, x, b, edge_smoother, potential_smoother):
    """One hybrid smoothing step: edge space, then the potential space."""
    x = edge_smoother(lev.A, lev.D, x, b)
    rp = lev.Gi.T @ (b - lev.A @ x)
    ep = potential_smoother(lev.Ap, lev.Dp, np.zeros_like(rp), rp)
    return x + lev.Gi @ ep


def jacobi_smoother(omega):
    return lambda A, D, x, b: gmg.jacobi(A, D, x, b, omega)


def vcycle(H: NedelecHierarchy, l, x, b, nu1=1, nu2=1, edge_smoother=None,
           potential_smoother=None):
    lev = H.levels[l]
    if l == H.lmin:
        return sla.cho_solve(H.coarse_chol, b) if H.coarse_chol is not None else x
    es = edge_smoother or jacobi_smoother(0.5)
    ps = potential_smoother or jacobi_smoother(0.5)
    for _ in range(nu1):
        x = hiptmair_step(lev, x, b, es, ps)
    bc = H.P[l].T @ (b - lev.A @ x)
    ec = vcycle(H, l - 1, np.zeros_like(bc), bc, nu1, nu2, edge_smoother, potential_smoother)
    x = x + H.P[l] @ ec
    for _ in range(nu2):
        x = hiptmair_step(lev, x, b, es, ps)
    return x


def fmg(H: NedelecHierarchy, b, cycles=5, **kw):
    """Full multigrid: rhs restricted to every level, exact coarsest solve,
    prolongated start plus `cycles` V-cycles per finer level."""
    bs = {H.lmax: b}
    for l in range(H.lmax, H.lmin, -1):
        bs[l - 1] = H.P[l].T @ bs[l]
    x = vcycle(H, H.lmin, np.zeros_like(bs[H.lmin]), bs[H.lmin])
    for l in range(H.lmin + 1, H.lmax + 1):
        x = H.P[l] @ x
        for _ in range(cycles):
            x = vcycle(H, l, x, bs[l], **kw)
    return x


def manufactured(xyz):
    """u = (sin pi y sin pi z, sin pi x sin pi z, sin pi x sin pi y) on the unit
    cube (u x n = 0 on its faces, div u = 0), so curl curl u = 2 pi^2 u."""
    s = np.sin(np.pi * xyz)
    return np.stack([s[:, 1] * s[:, 2], s[:, 0] * s[:, 2], s[:, 0] * s[:, 1]], axis=1)
