"""The anchors of the library's element-wise P2/N1 colour phases (host, no
GPU): exactly the lattice anchors, grouped by parity colour, the closed cubes
of one colour disjoint (so the threads of a phase read and write disjoint
DoFs and the plain read-modify-write per point is race-free), and the six
micro-cell types over all anchors give the 8^level micro-cells of Bey's
refinement (Sec. 3)."""
import numpy as np
import pytest

from oracle import indexing as ix

import paper_2308_01792_gb300 as hg

DELTA = [0, 2, 1, 1, 1, 1]   # largest anchor sum of type t is n - 1 - DELTA[t]


@pytest.mark.parametrize("level", [1, 2, 3, 4, 5, 6])
def test_phase_anchors_are_complete_and_race_free(level):
    n = 1 << level
    P, off = hg.p2_anchors(level)
    s = P.sum(axis=1)
    assert off[0] == 0 and off[8] == len(P)
    expect = {(i, j, k) for k in range(n) for j in range(n - k) for i in range(n - k - j)}
    assert {tuple(p) for p in P} == expect and len(P) == len(expect)
    m = 2 * n + 1
    for c in range(8):
        Q = P[off[c]:off[c + 1]]
        par = (Q[:, 0] & 1) | ((Q[:, 1] & 1) << 1) | ((Q[:, 2] & 1) << 2)
        assert np.all(par == c)
        # doubled-lattice points of every cube of this colour: no point twice
        d = np.array([(a, b, e) for e in range(3) for b in range(3) for a in range(3)])
        pts = (2 * Q[:, None, :] + d[None]).reshape(-1, 3)
        key = pts[:, 0] + m * (pts[:, 1] + m * pts[:, 2])
        assert len(np.unique(key)) == len(key)
    cells = sum(int(np.sum(s <= n - 1 - DELTA[t])) for t in range(6))
    assert cells == 8 ** level
    assert ix.n_tet(n) == len(P)
