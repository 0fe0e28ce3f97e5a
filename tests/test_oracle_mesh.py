"""Pins of the oracle's refined meshes (Sec. 3.1 Bey refinement, Sec. 3.2 subgroups)."""
import numpy as np
import pytest

import synthgen as sg
from oracle import indexing as ix
from oracle import mesh as om


def _canon(tets):
    """Each cell as a sorted tuple of its vertex tuples (orientation-free)."""
    return sorted(tuple(sorted(map(tuple, t))) for t in tets)


@pytest.mark.parametrize("level", [0, 1, 2, 3, 4])
def test_bey_equals_lattice_subgroups(level):
    ref = sg.reference_tet()
    bey = om.refine(ref.vertices, ref.cells, level)
    lat = om.lattice_cells(2 ** level)
    assert len(bey) == len(lat) == 8 ** level
    assert _canon(bey) == _canon(lat)


def _det(t):
    return int(round(np.linalg.det((t[:, 1:] - t[:, :1]).astype(float).transpose(0, 2, 1)).sum()))


def test_bey_children_have_one_eighth_volume_and_cover_parent():
    rng = np.random.default_rng(3)
    for _ in range(20):
        t = rng.integers(-8, 9, size=(1, 4, 3)) * 2
        v = np.linalg.det((t[0, 1:] - t[0, 0]).astype(float))
        if abs(v) < 1e-9:
            continue
        kids = om.bey_children(t)
        vk = [abs(np.linalg.det((k[1:] - k[0]).astype(float))) for k in kids]
        assert np.allclose(vk, abs(v) / 8)
        assert np.isclose(sum(vk), abs(v))


def test_inner_edge_is_v02_v13():
    t = np.array([[[0, 0, 0], [2, 0, 0], [0, 2, 0], [0, 0, 2]]])
    kids = om.bey_children(t)
    v02, v13 = (0, 1, 0), (1, 0, 1)
    inner = [k for k in kids[4:] if {v02, v13} <= set(map(tuple, k))]
    assert len(inner) == 4


@pytest.mark.parametrize("m,level", [(1, 0), (1, 1), (1, 3), (2, 2), (3, 1), (2, 3)])
def test_kuhn_cube_vertex_count_and_conformity(m, level):
    rm = om.RefinedMesh(sg.kuhn_cube(m), level)
    n = 2 ** level
    assert rm.n_vertices == (m * n + 1) ** 3
    assert len(rm.cells) == 6 * m ** 3 * 8 ** level
    f = om.faces_of(rm.cells)
    _, cnt = np.unique(f, axis=0, return_counts=True)
    assert cnt.max() == 2                         # conforming: no face in 3 cells
    assert (cnt == 1).sum() == 6 * 2 * (m * n) ** 2
    # Dirichlet vertices are exactly those on the cube surface
    c = rm.coords
    on_surf = np.any((c == 0) | (c == m * n), axis=1)
    assert np.array_equal(rm.boundary, on_surf)


@pytest.mark.parametrize("level", [0, 1, 2, 4])
def test_reference_tet_vertex_count(level):
    rm = om.RefinedMesh(sg.reference_tet(), level)
    assert rm.n_vertices == ix.n_tet(2 ** level + 1)
    n = 2 ** level
    c = rm.coords
    on_surf = (c.min(axis=1) == 0) | (c.sum(axis=1) == n)
    assert np.array_equal(rm.boundary, on_surf)
