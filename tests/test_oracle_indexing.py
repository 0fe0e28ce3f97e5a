"""Pins of the oracle's index functions (Sec. 3.2 cardinalities, Sec. 4 t_w)."""
import itertools
import os

import numpy as np
import pytest

from oracle import indexing as ix
from oracle import mesh as om


def test_cardinalities_match_their_sum_definitions():
    for w in range(0, 40):
        assert ix.n_tri(w) == sum(range(1, w + 1))
        assert ix.n_tet(w) == sum(sum(range(1, k + 1)) for k in range(1, w + 1))
        assert ix.n_tet(w) == len(ix.index_set_tet(w))
        assert ix.n_tri(w) == len([(i, j) for j in range(w) for i in range(w - j)])


@pytest.mark.parametrize("w", list(range(1, 14)))
def test_tw_closed_form_equals_loop_order_counting(w):
    cnt = ix.tw_by_counting(w)
    vals = [ix.tw(w, i, j, k) for (i, j, k) in cnt]
    assert vals == list(cnt.values())
    assert sorted(vals) == list(range(ix.n_tet(w)))


def test_tw_worked_example_w3():
    path = os.path.join(os.path.dirname(__file__), "golden", "tw_w3_zdown.txt")
    rows = [tuple(map(int, l.split())) for l in open(path) if l.strip() and not l.startswith("#")]
    assert len(rows) == ix.n_tet(3)
    for i, j, k, t in rows:
        assert ix.tw(3, i, j, k) == t


def test_aos_soa_are_bijections():
    for w, m in [(1, 1), (3, 2), (5, 3), (7, 4)]:
        pts = ix.index_set_tet(w)
        a = sorted(ix.aos(w, m, i, j, k, d) for (i, j, k) in pts for d in range(m))
        s = sorted(ix.soa(w, m, i, j, k, d) for (i, j, k) in pts for d in range(m))
        assert a == list(range(m * ix.n_tet(w))) == s
        # consecutive access in the printed loop orders
        seq = [ix.aos(w, m, i, j, k, d) for (i, j, k) in pts for d in range(m)]
        assert seq == list(range(m * ix.n_tet(w)))
        seq = [ix.soa(w, m, i, j, k, d) for d in range(m) for (i, j, k) in pts]
        assert seq == list(range(m * ix.n_tet(w)))


def _brute_counts(level):
    n = 2 ** level
    ref = np.array([[0, 0, 0], [1, 0, 0], [0, 1, 0], [0, 0, 1]])
    micro = om.refine(ref, np.array([[0, 1, 2, 3]]), level)
    coords, cells, _ = om.number_vertices(micro)
    nf = len(np.unique(om.faces_of(cells), axis=0))
    ne = len(np.unique(om.edges_of(cells), axis=0))
    return len(coords), ne, nf, len(cells)


@pytest.mark.parametrize("level", [0, 1, 2, 3, 4])
def test_subgroup_widths_count_every_micro_primitive(level):
    nv, ne, nf, nc = _brute_counts(level)
    wd = ix.subgroup_widths(level)
    by = lambda kind: sum(ix.n_tet(w) for (t, _), w in wd.items() if t == kind)
    assert nv == by("vertex") == ix.n_tet(2 ** level + 1)
    assert ne == by("edge")
    assert nc == by("cell") == 8 ** level
    assert nv - ne + nf - nc == 1            # Euler characteristic of a ball
    if level >= 1:
        assert nf == by("face")


def test_table_xyz_down_face_width_as_printed_undercounts():
    # Table 1 prints 2^l - 2 for xyz-down; with that value the faces do not add up.
    for level in (2, 3, 4):
        _, _, nf, _ = _brute_counts(level)
        wd = ix.subgroup_widths(level)
        printed = sum(ix.n_tet(w) for (t, s), w in wd.items() if t == "face") \
            - ix.n_tet(2 ** level - 1) + ix.n_tet(2 ** level - 2)
        assert printed != nf
