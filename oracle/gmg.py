"""Textbook geometric multigrid on assembled matrices (oracle, test infrastructure).

The level hierarchy is the one produced by refinement (multigrid by design:
functions live on a range of levels, Sec. 5.1).  Everything here is the
standard algorithm written out on SciPy CSR matrices:

* A_l: the assembled Neumann matrix of level l restricted to the interior
  (non-Dirichlet) DoFs; homogeneous Dirichlet values on the boundary.
* P_l: nodal interpolation between nested spaces (P1: coarse vertices are
  copied, coarse-edge midpoints get the mean of the two endpoints; P2:
  coarse quadratics evaluated at the fine DoF points).  R_l = P_l^T.
* Coarse operators by rediscretisation on the coarse mesh.
* Smoothers: weighted Jacobi x += w D^-1 (b - A x) (the paper names
  matvec+diagonal smoothers, Sec. 5.2.1), 4-colour Gauss-Seidel, or
  Chebyshev-accelerated Jacobi (Sec. 5.2.1 and the FMG solver of Sec. 6:
  Chebyshev smoothers of order 2 after Adams et al. 2003): the Chebyshev
  semi-iteration for D^-1 A on [0.1, 1.1] * lambda_max, lambda_max from a
  fixed power iteration on D^-1 A.
* ``fmg``: full multigrid (nested iteration, Sec. 6: five V(1,1) cycles per
  level): the right-hand side is restricted to every level, the coarsest is
  solved exactly, and each finer level starts from the prolongated coarser
  solution and runs a fixed number of V-cycles.
* V(nu1,nu2) recursion with a dense Cholesky solve on the coarsest level.
* ``solve``: x0 = 0, one V-cycle per iteration, stop when
  ||b - A x||_2 <= tol ||b||_2 on the interior DoFs.

Parity: pinned by contraction-rate and O(h^2) convergence tests, by the
Galerkin identity P^T A_f P = A_c for the P1 Laplacian, by exact solutions of
the coarse problem, by the closed-form Chebyshev error polynomial on a
diagonal matrix, by the power-iteration limit, and by FMG reaching an
algebraic error below the discretization error.
"""
from __future__ import annotations

import numpy as np
import scipy.linalg as sla
import scipy.sparse as sp

from . import fem
from .mesh import RefinedMesh, coord_key


class Level:
    """One level: mesh, assembled matrices and interior restriction."""

    def __init__(self, macro, level, space="P1", kind="laplace", coeff=None):
        self.rm = RefinedMesh(macro, level)
        self.space = space
        X = self.rm.cell_xyz
        if space == "P1":
            self.n = self.rm.n_vertices
            self.dofs = self.rm.cells
            self.xyz = self.rm.xyz
            self.boundary = self.rm.boundary
            if kind == "laplace":
                Ke = fem.p1_stiffness(X)
            elif kind == "divkgrad":
                kv = coeff(self.xyz)[self.dofs]
                Ke = fem.p1_divkgrad(X, kv)
            else:
                raise ValueError(kind)
            Me = fem.p1_mass(X)
        elif space == "P2":
            self.num = fem.P2Numbering(self.rm)
            self.n = self.num.n
            self.dofs = self.num.dofs
            self.xyz = self.num.xyz
            self.boundary = self.num.boundary
            Ke = fem.p2_stiffness(X, coeff)
            Me = fem.p2_mass(X)
        else:
            raise ValueError(space)
        self.A_full = fem.assemble(self.dofs, Ke, self.n)
        self.M_full = fem.assemble(self.dofs, Me, self.n)
        self.interior = np.flatnonzero(~self.boundary)
        ii = self.interior
        self.A = self.A_full[ii][:, ii].tocsr()
        self.D = self.A.diagonal()


def p1_prolongation(fine: Level, coarse: Level) -> sp.csr_matrix:
    """Nodal interpolation P1(coarse) -> P1(fine) on all DoFs."""
    fkeys = coord_key(fine.rm.coords, fine.rm.side)
    def fidx(c2):
        return np.searchsorted(fkeys, coord_key(c2, fine.rm.side))
    cc = coarse.rm.coords
    rows = [fidx(2 * cc)]
    cols = [np.arange(coarse.n)]
    vals = [np.ones(coarse.n)]
    e = np.unique(fem_edges(coarse.rm.cells), axis=0)
    mid = fidx(cc[e[:, 0]] + cc[e[:, 1]])
    for end in (0, 1):
        rows.append(mid)
        cols.append(e[:, end])
        vals.append(np.full(len(e), 0.5))
    return sp.coo_matrix((np.concatenate(vals), (np.concatenate(rows), np.concatenate(cols))),
                         shape=(fine.n, coarse.n)).tocsr()


def fem_edges(cells):
    from .mesh import edges_of
    return edges_of(cells)


def p2_prolongation(fine: Level, coarse: Level) -> sp.csr_matrix:
    """Coarse P2 functions evaluated at the fine P2 DoF points.

    The fine DoF points inside a coarse micro-cell have barycentric
    coordinates (a,b,c,d)/4 with a+b+c+d = 4 (35 points); the 10 coarse basis
    functions are evaluated there.  Shared points get identical (exact
    dyadic) values from every cell, so duplicates are dropped.
    """
    cm = coarse.rm.micro                                  # coarse units
    pts4 = 4 * cm                                         # fine doubled units
    patt = [(a, b, c, 4 - a - b - c) for a in range(5) for b in range(5 - a)
            for c in range(5 - a - b)]
    fkeys = coord_key(fine.num.coords2, 2 * fine.rm.side)
    rows, cols, vals = [], [], []
    for p in patt:
        lam = np.array(p, dtype=np.float64) / 4.0
        X = (p[0] * pts4[:, 0] + p[1] * pts4[:, 1] + p[2] * pts4[:, 2] + p[3] * pts4[:, 3]) // 4
        fi = np.searchsorted(fkeys, coord_key(X, 2 * fine.rm.side))
        phi = [lam[i] * (2 * lam[i] - 1) for i in range(4)] + \
              [4 * lam[i] * lam[j] for i, j in fem.P2_EDGES]
        for loc in range(10):
            if phi[loc] != 0.0:
                rows.append(fi)
                cols.append(coarse.dofs[:, loc])
                vals.append(np.full(len(fi), phi[loc]))
    r = np.concatenate(rows)
    c = np.concatenate(cols)
    v = np.concatenate(vals)
    key = r.astype(np.int64) * coarse.n + c
    _, first = np.unique(key, return_index=True)
    return sp.coo_matrix((v[first], (r[first], c[first])), shape=(fine.n, coarse.n)).tocsr()


class Hierarchy:
    """Levels lmin..lmax with interior prolongations."""

    def __init__(self, macro, lmin, lmax, space="P1", kind="laplace", coeff=None):
        self.lmin, self.lmax = lmin, lmax
        self.levels = {l: Level(macro, l, space, kind, coeff) for l in range(lmin, lmax + 1)}
        self.P = {}
        for l in range(lmin + 1, lmax + 1):
            f, c = self.levels[l], self.levels[l - 1]
            Pf = p1_prolongation(f, c) if space == "P1" else p2_prolongation(f, c)
            self.P[l] = Pf[f.interior][:, c.interior].tocsr()
        cA = self.levels[lmin].A.toarray()
        self.coarse_chol = sla.cho_factor(cA) if cA.size else None


def jacobi(A, D, x, b, omega):
    return x + omega * (b - A @ x) / D


def gauss_seidel_colours(A, D, x, b, colour):
    """One sweep over 4 colours: x_c += (b - A x)_c / D_c for c = 0..3."""
    x = x.copy()
    for c in range(4):
        sel = colour == c
        r = b - A @ x
        x[sel] += r[sel] / D[sel]
    return x


def vcycle(H: Hierarchy, l, x, b, nu1=3, nu2=3, omega=2.0 / 3.0, smoother=None):
    lev = H.levels[l]
    if l == H.lmin:
        return sla.cho_solve(H.coarse_chol, b) if H.coarse_chol is not None else x
    sm = smoother or (lambda A, D, x, b: jacobi(A, D, x, b, omega))
    for _ in range(nu1):
        x = sm(lev.A, lev.D, x, b)
    r = b - lev.A @ x
    bc = H.P[l].T @ r
    ec = vcycle(H, l - 1, np.zeros_like(bc), bc, nu1, nu2, omega, smoother)
    x = x + H.P[l] @ ec
    for _ in range(nu2):
        x = sm(lev.A, lev.D, x, b)
    return x


def solve(H: Hierarchy, b, tol=1e-10, max_iter=100, **kw):
    """x0 = 0; V-cycles until ||b - A x|| <= tol ||b||.  Returns (x, iters, history)."""
    A = H.levels[H.lmax].A
    x = np.zeros_like(b)
    nb = np.linalg.norm(b)
    hist = [1.0]
    it = 0
    while hist[-1] > tol and it < max_iter:
        x = vcycle(H, H.lmax, x, b, **kw)
        it += 1
        hist.append(np.linalg.norm(b - A @ x) / nb)
    return x, it, hist


def power_lambda_max(A, D, v0, iters=20):
    """Largest eigenvalue of D^-1 A by a fixed power iteration from v0:
    w = D^-1 A v, lambda = ||w|| / ||v||, v = w / ||w||; returns the last lambda."""
    v = v0 / np.linalg.norm(v0)
    lam = 0.0
    for _ in range(iters):
        w = (A @ v) / D
        nw = np.linalg.norm(w)
        lam = nw
        v = w / nw
    return lam


def chebyshev(A, D, x, b, lam_max, order=2, lo=0.1, hi=1.1):
    """Chebyshev semi-iteration (Saad, Iterative Methods, Alg. 12.1) for
    D^-1 A on the interval [lo, hi] * lam_max: `order` residual evaluations."""
    a, c = lo * lam_max, hi * lam_max
    theta, delta = 0.5 * (c + a), 0.5 * (c - a)
    sigma = theta / delta
    rho = 1.0 / sigma
    r = b - A @ x
    d = r / (D * theta)
    x = x + d
    for _ in range(order - 1):
        rho_new = 1.0 / (2.0 * sigma - rho)
        r = b - A @ x
        d = rho_new * rho * d + (2.0 * rho_new / delta) * (r / D)
        x = x + d
        rho = rho_new
    return x


def fmg(H: Hierarchy, b, cycles=5, nu1=1, nu2=1, smoother=None, **kw):
    """Full multigrid for the finest-level right-hand side b (interior DoFs):
    b restricted to every level (b_{l-1} = P_l^T b_l), exact coarsest solve,
    then on each finer level x_l = P_l x_{l-1} followed by `cycles` V-cycles."""
    bs = {H.lmax: b}
    for l in range(H.lmax, H.lmin, -1):
        bs[l - 1] = H.P[l].T @ bs[l]
    x = vcycle(H, H.lmin, np.zeros_like(bs[H.lmin]), bs[H.lmin])
    for l in range(H.lmin + 1, H.lmax + 1):
        x = H.P[l] @ x
        for _ in range(cycles):
            x = vcycle(H, l, x, bs[l], nu1, nu2, smoother=smoother, **kw)
    return x
