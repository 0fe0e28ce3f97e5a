"""CPU checks of the C-ABI library: it loads, exports every declared symbol,
and its host-only logic (mesh checks, t_w) behaves.  No GPU calls."""
import os
import re
import subprocess

import numpy as np
import pytest

import paper_2308_01792_gb300 as hg
import synthgen as sg
from oracle import indexing as ix

HDR = os.path.join(os.path.dirname(os.path.dirname(__file__)), "include", "hytet.h")


def _declared():
    src = open(HDR).read()
    src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
    return sorted(set(re.findall(r"\b(hg_[a-z0-9_]+)\s*\(", src)))


@pytest.fixture(scope="module")
def built():
    if not os.path.exists(hg.LIB_PATH):
        from paper_2308_01792_gb300 import build
        build.build()
    return hg.lib()


def test_every_declared_symbol_is_exported(built):
    out = subprocess.run(["nm", "-D", "--defined-only", hg.LIB_PATH], capture_output=True,
                         text=True).stdout
    exported = set(re.findall(r"\bT (hg_[a-z0-9_]+)", out))
    declared = _declared()
    assert declared, "no declarations parsed"
    missing = [d for d in declared if d not in exported]
    assert not missing, missing
    assert set(declared) == set(hg.SIGNATURES), "binding and header disagree"


def test_host_tw_matches_oracle(built):
    for w in (1, 2, 3, 9, 33, 129):
        for (i, j, k) in ix.index_set_tet(w)[:: max(1, ix.n_tet(w) // 500)]:
            assert hg.index_tw(w, i, j, k) == ix.tw(w, i, j, k)
    with pytest.raises(hg.HGError):
        hg.index_tw(3, 2, 1, 0)


def test_host_tw_rejects_what_it_cannot_index(built):
    """t_w is defined on I_tet(w); w above 2^20 would overflow N_tet in int64."""
    big = 1 << 20
    assert hg.index_tw(big, big - 1, 0, 0) == big - 1
    assert hg.index_tw(big, 5, 7, big - 13) == ix.tw(big, 5, 7, big - 13)
    for args in ((big + 1, 0, 0, 0), (3, -1, 0, 0), (3, 1, 1, 1), (0, 0, 0, 0)):
        with pytest.raises(hg.HGError) as e:
            hg.index_tw(*args)
        assert e.value.code == -1


def test_mesh_primitive_graph_counts(built):
    for m in (1, 2, 3):
        mm = sg.kuhn_cube(m)
        c = hg.Mesh(mm.xyz, mm.cells).counts()
        assert c["cells"] == 6 * m ** 3 and c["vertices"] == (m + 1) ** 3
        assert c["boundary_faces"] == 12 * m * m
        # Euler characteristic of the macro mesh of a ball
        assert c["vertices"] - c["edges"] + c["faces"] - c["cells"] == 1
    r = sg.reference_tet()
    assert hg.Mesh(r.xyz, r.cells).counts()["boundary_faces"] == 4


def test_bad_meshes_are_rejected(built):
    r = sg.reference_tet()
    with pytest.raises(hg.HGError) as e:
        hg.Mesh(r.xyz, np.array([[0, 1, 2, 2]]))
    assert e.value.code == -2
    with pytest.raises(hg.HGError):
        hg.Mesh(r.xyz, np.array([[0, 1, 2, 7]]))
    flat = np.array([[0, 0, 0], [1, 0, 0], [0, 1, 0], [1, 1, 0]], dtype=float)
    with pytest.raises(hg.HGError):
        hg.Mesh(flat, np.array([[0, 1, 2, 3]]))
    # three cells on one face: not conforming
    xyz = np.array([[0, 0, 0], [1, 0, 0], [0, 1, 0], [0, 0, 1], [0, 0, -1], [1, 1, 1]], float)
    with pytest.raises(hg.HGError):
        hg.Mesh(xyz, np.array([[0, 1, 2, 3], [0, 1, 2, 4], [0, 1, 2, 5]]))


def test_vertices_of_no_cell_are_rejected(built):
    """Every macro vertex is a primitive with a copy in each containing cell;
    a vertex that no cell lists is refused at creation."""
    r = sg.reference_tet()
    xyz = np.vstack([np.asarray(r.xyz, dtype=float), [[5.0, 5.0, 5.0]]])
    with pytest.raises(hg.HGError) as e:
        hg.Mesh(xyz, np.asarray(r.cells))
    assert e.value.code == -2 and "vertex 4 belongs to no cell" in str(e.value)


def test_overlapping_cells_are_rejected(built):
    """Cells meet only in common faces, edges or vertices (Sec. 2): the two
    cells of an interior face lie on opposite sides of it.  A cell listed
    twice (in any vertex order) or folded over a shared face overlaps its
    neighbour; two cells on opposite sides pass."""
    r = sg.reference_tet()
    for cells in ([[0, 1, 2, 3], [0, 1, 2, 3]], [[0, 1, 2, 3], [1, 0, 2, 3]]):
        with pytest.raises(hg.HGError) as e:
            hg.Mesh(r.xyz, np.array(cells))
        assert e.value.code == -2 and "overlap" in str(e.value)
    base = [[0, 0, 0], [1, 0, 0], [0, 1, 0], [0, 0, 1]]
    two = np.array([[0, 1, 2, 3], [0, 1, 2, 4]])
    with pytest.raises(hg.HGError) as e:
        hg.Mesh(np.array(base + [[0.2, 0.2, 0.5]], float), two)
    assert "same side" in str(e.value)
    hg.Mesh(np.array(base + [[0, 0, -1]], float), two)
    for m in (1, 2, 3):
        for seed in range(4):
            c = sg.permuted_cells(sg.kuhn_cube(m), seed)
            hg.Mesh(c.xyz, c.cells)


def test_quadrature_rule_exact_to_degree_five():
    """The library derives its P2 rule from the moment equations: positive
    weights summing to 1, points inside the tetrahedron, every barycentric
    monomial of degree <= 5 integrated exactly (closed form 3! prod a_i! /
    (|a|+3)!), and degree 6 not (so the rule is the degree-5 one)."""
    import itertools
    import math
    b, w = hg.quadrature_rule()
    assert b.shape == (14, 4) and np.all(w > 0) and abs(w.sum() - 1) < 1e-15
    assert np.all(b >= 0) and np.allclose(b.sum(axis=1), 1, atol=1e-15)
    worst = {}
    for al in itertools.product(range(7), repeat=4):
        d = sum(al)
        if d > 6:
            continue
        ex = 6 * math.prod(math.factorial(a) for a in al) / math.factorial(d + 3)
        got = float(np.sum(w * np.prod(b ** np.array(al), axis=1)))
        worst[d] = max(worst.get(d, 0.0), abs(got - ex))
    assert max(worst[d] for d in range(6)) < 1e-15
    assert worst[6] > 1e-6


def _fan_mesh(g=7):
    """A cube's surface cut into 2 g^2 triangles per side, each joined to the
    centre: a conforming mesh of 12 g^2 cells that all share the centre
    vertex (integer corners, centre at half-integers)."""
    verts = {}
    xyz = []

    def vid(p):
        if p not in verts:
            verts[p] = len(xyz)
            xyz.append(p)
        return verts[p]

    centre = vid((g / 2, g / 2, g / 2))
    cells = []
    for ax in range(3):
        for side in (0, g):
            for a in range(g):
                for b in range(g):
                    def pt(u, v):
                        p = [0, 0, 0]
                        p[ax], p[(ax + 1) % 3], p[(ax + 2) % 3] = side, u, v
                        return vid(tuple(float(c) for c in p))
                    q = [pt(a, b), pt(a + 1, b), pt(a + 1, b + 1), pt(a, b + 1)]
                    cells += [[centre, q[0], q[1], q[2]], [centre, q[0], q[2], q[3]]]
    return np.array(xyz, dtype=float), np.array(cells, dtype=np.int64)


def test_hierarchy_limits_are_checked_before_any_allocation(built):
    """Sizes the per-level tables cannot represent are refused with
    HG_ERR_UNSUPPORTED before the GPU is touched (so this runs without one):
    more than 2^31 - 1 stored points, lattice coordinates of magnitude 2^20 or
    more (the canonical keys' 21 bits), and a primitive shared by more than
    255 cells (the interface items' 8-bit copy count)."""
    c = sg.kuhn_cube(4)                      # 384 cells x N_tet(513) > 2^31 at level 9
    with pytest.raises(hg.HGError) as e:
        hg.Hierarchy(hg.Mesh(c.xyz, c.cells), 0, 9)
    assert e.value.code == -7 and "stored points" in str(e.value)
    r = sg.reference_tet()
    big = np.asarray(r.xyz, dtype=float) * 4096   # 4096 x 2^9 = 2^21
    with pytest.raises(hg.HGError) as e:
        hg.Hierarchy(hg.Mesh(big, r.cells), 0, 9)
    assert e.value.code == -7 and "2^20" in str(e.value)
    xyz, cells = _fan_mesh()
    m = hg.Mesh(xyz, cells)
    assert m.counts()["cells"] == len(cells) == 588 and m.counts()["boundary_faces"] == 588
    with pytest.raises(hg.HGError) as e:
        hg.Hierarchy(m, 0, 1)
    assert e.value.code == -7 and "shared by 588 cells" in str(e.value)


def _prototypes():
    """name -> (return type is void, parameter count) from include/hytet.h,
    comments removed."""
    src = open(HDR).read()
    src = re.sub(r"/\*.*?\*/", " ", src, flags=re.S)
    out = {}
    for m in re.finditer(r"\b(void|int|const\s+char\s*\*)\s+(hg_[a-z0-9_]+)\s*\(([^)]*)\)\s*;", src):
        params = m.group(3).strip()
        n = 0 if params in ("", "void") else params.count(",") + 1
        out[m.group(2)] = (m.group(1) == "void", n)
    return out


def test_binding_signatures_match_the_header_prototypes(built):
    """Each ctypes signature has as many arguments as its C prototype, and
    void functions have no result type: a mismatch would pass arguments in
    the wrong registers."""
    protos = _prototypes()
    assert set(protos) == set(hg.SIGNATURES)
    for name, (res, args) in hg.SIGNATURES.items():
        is_void, n = protos[name]
        assert len(args) == n, (name, len(args), n)
        assert (res is None) == is_void, name
