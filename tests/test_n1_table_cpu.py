"""The library's Nedelec prolongation class table (host, no GPU) against the
oracle's exact N1 prolongation.

On single-cell meshes the lattice points of the cell map one to one onto the
oracle's DoFs, so applying the table at every fine edge point (with the
cell's orientation signs) must reproduce P u_c for any coarse vector u_c.
The cells are the reference tetrahedron, vertex-permuted copies of it (other
local orientations and refinements) and a skewed integer tetrahedron."""
import numpy as np
import pytest

import synthgen as sg
from oracle import nedelec as ne
from oracle.mesh import coord_key

import paper_2308_01792_gb300 as hg

DIRS = np.array([[1, 0, 0], [0, 1, 0], [-1, 1, 0], [0, 0, 1], [-1, 0, 1], [0, -1, 1], [1, -1, 1]])
SKEW = sg.MacroMesh(np.array([[0, 0, 0], [2, 1, 0], [1, 3, 1], [0, 1, 2]], dtype=np.int64),
                    np.array([[0, 1, 2, 3]], dtype=np.int64), 1, "skew_tet")
MESHES = [sg.reference_tet(), sg.permuted_cells(sg.reference_tet(), 1),
          sg.permuted_cells(sg.reference_tet(), 2), SKEW, sg.permuted_cells(SKEW, 4)]


def _signs(E):
    out = []
    for d in DIRS:
        v = d @ E
        first = next(c for c in (v[2], v[1], v[0]) if c != 0)
        out.append(1.0 if first > 0 else -1.0)
    return np.array(out)


def _edge_points(lev, V0, E, level):
    """Odd points q of the doubled lattice of `level` and their oracle N1 indices."""
    m = 2 << level
    q = np.array([(x, y, z) for z in range(m + 1) for y in range(m + 1 - z)
                  for x in range(m + 1 - z - y) if (x | y | z) & 1])
    keys = coord_key((V0 << (level + 1)) + q @ E, 2 * lev.rm.side)
    idx = np.searchsorted(lev.keys, keys)
    assert np.array_equal(lev.keys[idx], keys)
    return q, idx


@pytest.mark.parametrize("macro", MESHES, ids=lambda m: m.name)
def test_table_reproduces_the_oracle_prolongation(macro):
    T = hg.n1_prolong_table()
    V = macro.vertices[macro.cells[0]]
    E = np.stack([V[1] - V[0], V[2] - V[0], V[3] - V[0]])
    s = _signs(E)
    L = 2
    fine, coarse = ne.NedelecLevel(macro, L), ne.NedelecLevel(macro, L - 1)
    qf, fi = _edge_points(fine, V[0], E, L)
    qc, ci = _edge_points(coarse, V[0], E, L - 1)
    assert len(fi) == fine.n and len(ci) == coarse.n
    cidx = {tuple(p): i for p, i in zip(qc, ci)}
    uc = sg.uniform_vector(31, coarse.n)
    ref = ne.nedelec_prolongation(fine, coarse) @ uc
    got = np.zeros(fine.n)
    for q, i in zip(qf, fi):
        r, p = q % 4, q // 4
        cl = r[0] + 4 * r[1] + 16 * r[2]
        assert T["fine_dir"][cl] >= 0
        acc = 0.0
        for t in range(T["n"][cl]):
            o = T["off"][cl, t]
            c = tuple(2 * p + np.array([o & 3, (o >> 2) & 3, o >> 4]))
            acc += T["w"][cl, t] * s[T["dir"][cl, t]] * uc[cidx[c]]
        got[i] = s[T["fine_dir"][cl]] * acc
    assert np.allclose(got, ref, rtol=0, atol=1e-14)


def test_table_shape():
    T = hg.n1_prolong_table()
    par = np.array([(c & 1) | ((c >> 2 & 1) << 1) | ((c >> 4 & 1) << 2) for c in range(64)])
    assert np.array_equal(T["fine_dir"] >= 0, par > 0)
    assert np.all(T["n"][par == 0] == 0) and np.all((T["n"][par > 0] >= 1) & (T["n"][par > 0] <= 6))
    # half-edges of coarse edges take half of the coarse DoF
    w = T["w"][T["w"] != 0]
    assert set(np.abs(w)) <= {0.25, 0.5}


@pytest.mark.parametrize("macro", MESHES, ids=lambda m: m.name)
def test_restriction_lists_are_the_transpose(macro):
    R = hg.n1_restrict_table()
    V = macro.vertices[macro.cells[0]]
    E = np.stack([V[1] - V[0], V[2] - V[0], V[3] - V[0]])
    s = _signs(E)
    L = 2
    fine, coarse = ne.NedelecLevel(macro, L), ne.NedelecLevel(macro, L - 1)
    qf, fi = _edge_points(fine, V[0], E, L)
    qc, ci = _edge_points(coarse, V[0], E, L - 1)
    fidx = {tuple(p): i for p, i in zip(qf, fi)}
    rf = sg.uniform_vector(32, fine.n)
    ref = ne.nedelec_prolongation(fine, coarse).T @ rf
    got = np.zeros(coarse.n)
    for c, i in zip(qc, ci):
        pc = (c[0] & 1) | ((c[1] & 1) << 1) | ((c[2] & 1) << 2)
        acc = 0.0
        for e in range(R["start"][pc], R["start"][pc + 1]):
            dd = R["d"][e]
            q = tuple(2 * c + np.array([(dd & 31) - 8, ((dd >> 5) & 31) - 8, (dd >> 10) - 8]))
            if q in fidx:
                acc += R["w"][e] * s[R["fine_dir"][e]] * rf[fidx[q]]
        got[i] = s[pc - 1] * acc
    assert np.allclose(got, ref, rtol=0, atol=1e-14)


@pytest.mark.parametrize("macro", [sg.kuhn_cube(1), sg.permuted_cells(sg.kuhn_cube(1), 3),
                                   sg.permuted_cells(sg.kuhn_cube(2), 7)],
                         ids=["cube1", "cube1perm", "cube2perm"])
def test_table_on_multi_cell_meshes_gives_identical_copies(macro):
    """Every cell applies the table with its own orientation signs to its own
    lattice points; the copies of an interface edge (one per cell) must agree
    exactly and equal the oracle's P u_c.  Weights and signs are exact, so a
    transfer kernel needs no exchange between the copies."""
    T = hg.n1_prolong_table()
    L = 2
    fine, coarse = ne.NedelecLevel(macro, L), ne.NedelecLevel(macro, L - 1)
    uc = sg.uniform_vector(33, coarse.n)
    ref = ne.nedelec_prolongation(fine, coarse) @ uc
    seen = {}
    for cell in macro.cells:
        V = macro.vertices[cell]
        E = np.stack([V[1] - V[0], V[2] - V[0], V[3] - V[0]])
        s = _signs(E)
        qf, fi = _edge_points(fine, V[0], E, L)
        qc, ci = _edge_points(coarse, V[0], E, L - 1)
        cidx = {tuple(p): i for p, i in zip(qc, ci)}
        for q, i in zip(qf, fi):
            r, p = q % 4, q // 4
            cl = r[0] + 4 * r[1] + 16 * r[2]
            acc = 0.0
            for t in range(T["n"][cl]):
                o = T["off"][cl, t]
                c = tuple(2 * p + np.array([o & 3, (o >> 2) & 3, o >> 4]))
                acc += T["w"][cl, t] * s[T["dir"][cl, t]] * uc[cidx[c]]
            v = s[T["fine_dir"][cl]] * acc
            if i in seen:
                assert v == seen[i], (i, v, seen[i])
            seen[i] = v
    assert len(seen) == fine.n
    got = np.array([seen[i] for i in range(fine.n)])
    assert np.allclose(got, ref, rtol=0, atol=1e-14)
