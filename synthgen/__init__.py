"""Seeded synthetic inputs shared by the CUDA path's tests/bench and by the oracle.

This module holds inputs only: coarse (macro) meshes given by integer vertex
coordinates, seeded random vectors, the random-Fourier-feature parameters of the
log-normal coefficient field, and the per-problem draw of the batched workload.
It contains none of the method's arithmetic (no refinement, no indexing, no
finite-element quantities), so both sides can import it without sharing code.

Coordinates are exact: every macro vertex is an integer triple ``V`` and the
physical point is ``V / scale``.  All workloads of the paper's kind used here
(reference tetrahedron, unit cube split into Kuhn tetrahedra) are dyadic, so
refined vertex coordinates stay exact integers after multiplying by ``2**L``.
"""
from __future__ import annotations

import itertools
from dataclasses import dataclass

import numpy as np

__all__ = [
    "MacroMesh", "reference_tet", "kuhn_cube", "uniform_vector",
    "rff_params", "rff_eval", "batched_problem_draw", "WORKLOADS",
    "SINPROD_AB", "sinprod_coefficient", "sinprod_manufactured",
]


@dataclass(frozen=True)
class MacroMesh:
    """Coarse tetrahedral mesh: integer vertices, cells as 4 vertex ids.

    ``vertices`` has shape (nv, 3) int64; physical coordinates are
    ``vertices / scale``.  ``cells`` has shape (nc, 4) int64; the order of the
    four ids in a row is the local vertex order v0..v3 of that macro cell,
    which fixes how the cell is refined (inner edge v02-v13 of Bey's rule).
    """
    vertices: np.ndarray
    cells: np.ndarray
    scale: int
    name: str

    @property
    def xyz(self) -> np.ndarray:
        return self.vertices.astype(np.float64) / float(self.scale)


def reference_tet() -> MacroMesh:
    """The reference tetrahedron (0,0,0),(1,0,0),(0,1,0),(0,0,1)."""
    v = np.array([[0, 0, 0], [1, 0, 0], [0, 1, 0], [0, 0, 1]], dtype=np.int64)
    return MacroMesh(v, np.array([[0, 1, 2, 3]], dtype=np.int64), 1, "reference_tet")


def kuhn_cube(m: int) -> MacroMesh:
    """Unit cube as m x m x m sub-cubes, each split into 6 Kuhn tetrahedra.

    Each sub-cube with lower corner c is split along its main diagonal into
    the 6 tetrahedra (c, c+e_s1, c+e_s1+e_s2, c+(1,1,1)) for the 6
    permutations s of the axes.  Vertex order is this path order.
    """
    if m < 1:
        raise ValueError("m must be >= 1")
    g = m + 1
    idx = lambda x, y, z: x + g * (y + g * z)
    verts = np.array([[x, y, z] for z in range(g) for y in range(g) for x in range(g)],
                     dtype=np.int64)
    unit = np.eye(3, dtype=np.int64)
    cells = []
    for cz in range(m):
        for cy in range(m):
            for cx in range(m):
                c = np.array([cx, cy, cz], dtype=np.int64)
                for perm in itertools.permutations(range(3)):
                    p0 = c
                    p1 = p0 + unit[perm[0]]
                    p2 = p1 + unit[perm[1]]
                    p3 = p2 + unit[perm[2]]
                    cells.append([idx(*p) for p in (p0, p1, p2, p3)])
    return MacroMesh(verts, np.array(cells, dtype=np.int64), m, f"kuhn_cube_m{m}")


def permuted_cells(macro: MacroMesh, seed: int) -> MacroMesh:
    """The same mesh with every cell's local vertex order permuted by a seeded
    draw (PCG64): the refinement and all local orientations change, the
    domain does not."""
    g = np.random.Generator(np.random.PCG64(seed))
    cells = np.array([row[g.permutation(4)] for row in macro.cells], dtype=np.int64)
    return MacroMesh(macro.vertices, cells, macro.scale, f"{macro.name}_perm{seed}")


def uniform_vector(seed: int, n: int, lo: float = -1.0, hi: float = 1.0) -> np.ndarray:
    """n values U[lo, hi) in FP64 from numpy's PCG64 stream with the given seed.

    The values are consumed in canonical DoF order (ascending integer
    coordinate key, z slowest) by both sides.
    """
    return np.random.Generator(np.random.PCG64(seed)).uniform(lo, hi, size=n)


def rff_params(seed: int, n_features: int = 1024, corr_len: float = 0.1,
               sigma: float = 1.0):
    """Random Fourier features of a squared-exponential Gaussian field.

    g(x) = sigma * sqrt(2/F) * sum_f cos(omega_f . x + beta_f) with
    omega_f ~ N(0, corr_len^-2 I) and beta_f ~ U[0, 2 pi)
    (Rahimi & Recht 2007).  Returns (omega (F,3), beta (F,), amplitude).
    """
    rng = np.random.Generator(np.random.PCG64(seed))
    omega = rng.normal(0.0, 1.0 / corr_len, size=(n_features, 3))
    beta = rng.uniform(0.0, 2.0 * np.pi, size=n_features)
    amp = sigma * np.sqrt(2.0 / n_features)
    return omega, beta, amp


def rff_eval(params, xyz: np.ndarray) -> np.ndarray:
    """k = exp(g(x)) at the given points (N,3), FP64."""
    omega, beta, amp = params
    xyz = np.asarray(xyz, dtype=np.float64)
    out = np.empty(len(xyz))
    for s in range(0, len(xyz), 65536):
        blk = xyz[s:s + 65536]
        out[s:s + 65536] = amp * np.cos(blk @ omega.T + beta).sum(axis=1)
    return np.exp(out)


def rff_eval_torch(params, xyz, device="cuda", dtype=None):
    """rff_eval with torch on a device, for large point sets (same formula;
    FP64 by default, FP32 on request for speed)."""
    import torch
    dtype = dtype or torch.float64
    omega, beta, amp = params
    om = torch.tensor(omega, dtype=dtype, device=device)
    be = torch.tensor(beta, dtype=dtype, device=device)
    X = torch.as_tensor(np.asarray(xyz, dtype=np.float64), device=device).to(dtype)
    out = torch.empty(len(X), dtype=dtype, device=device)
    for s in range(0, len(X), 1 << 18):
        out[s:s + (1 << 18)] = amp * torch.cos(X[s:s + (1 << 18)] @ om.T + be).sum(dim=1)
    return torch.exp(out).double().cpu().numpy()


# The smooth coefficient of the P2 workload, k(x) = a + b sin(2 pi x) sin(2 pi y)
# sin(2 pi z), as (a, b).
SINPROD_AB = (1.0, 0.5)


def sinprod_coefficient(a: float = SINPROD_AB[0], b: float = SINPROD_AB[1]):
    """k(x) = a + b sin(2 pi x) sin(2 pi y) sin(2 pi z) as a callable on (N,3) points."""
    def k(X):
        X = np.asarray(X, dtype=np.float64)
        return a + b * np.prod(np.sin(2.0 * np.pi * X), axis=1)
    return k


def sinprod_manufactured(xyz, a: float = SINPROD_AB[0], b: float = SINPROD_AB[1]):
    """u = sin(pi x) sin(pi y) sin(pi z) and f = -div(k grad u) for the sinprod k,
    in closed form (f = 3 pi^2 k u - grad k . grad u), at points (N,3)."""
    X = np.asarray(xyz, dtype=np.float64)
    s1, c1 = np.sin(np.pi * X), np.cos(np.pi * X)
    s2, c2 = np.sin(2 * np.pi * X), np.cos(2 * np.pi * X)
    u = np.prod(s1, axis=1)
    k = a + b * np.prod(s2, axis=1)
    gu = np.pi * np.stack([c1[:, 0] * s1[:, 1] * s1[:, 2], s1[:, 0] * c1[:, 1] * s1[:, 2],
                           s1[:, 0] * s1[:, 1] * c1[:, 2]], axis=1)
    gk = 2 * np.pi * b * np.stack([c2[:, 0] * s2[:, 1] * s2[:, 2], s2[:, 0] * c2[:, 1] * s2[:, 2],
                                   s2[:, 0] * s2[:, 1] * c2[:, 2]], axis=1)
    f = 3 * np.pi ** 2 * k * u - np.sum(gk * gu, axis=1)
    return u, f


def batched_problem_draw(seed: int = 42, count: int = 512):
    """Per-problem (m, level) of the batched workload: m in {1,2,3}, level in {3..6}."""
    rng = np.random.Generator(np.random.PCG64(seed))
    m = 1 + rng.integers(0, 3, size=count)
    lv = 3 + rng.integers(0, 4, size=count)
    return [(int(a), int(b)) for a, b in zip(m, lv)]


# The five workloads, by what they are (shapes and sizes of the paper's kind).
WORKLOADS = {
    "tet_L4_p1": dict(mesh=("reference_tet",), level=4, space="P1"),
    "cube6_L7_p1": dict(mesh=("kuhn_cube", 1), level=7, space="P1"),
    "cube48_L6_p2_sinprod": dict(mesh=("kuhn_cube", 2), level=6, space="P2"),
    "batch512_p1": dict(mesh=None, level=None, space="P1"),
    "cube384_L6_p1_lognormal": dict(mesh=("kuhn_cube", 4), level=6, space="P1"),
}
