"""The apply kernels' lane walk over the library's plane-window tiles, emulated
on the CPU (no GPU): every cell-interior point is the output of exactly one
(tile, window, lane); every load stays inside the padded cell; and the seven
row loads and eight shuffled neighbours of every output are the right
lattice neighbours (the 15-point stencil of Sec. 5.2 in t_w order, Sec. 4).

The emulation restates the kernels' per-lane arithmetic (lane placement, the
row walk, the clamp at the plane end, the output condition and the seven row
offsets) and checks it against the lattice through the oracle's index
function."""
import numpy as np
import pytest

from oracle import indexing as ix

import paper_2308_01792_gb300 as hg


def _coords(w):
    n_tet = ix.n_tet(w)
    c = np.full((n_tet, 3), -1, dtype=np.int64)
    for k in range(w):
        for j in range(w - k):
            for i in range(w - k - j):
                c[ix.tw(w, i, j, k)] = (i, j, k)
    return c


@pytest.mark.parametrize("level", [2, 3, 4, 5, 6, 7])
def test_lane_walk_covers_the_interior_once_with_the_right_neighbours(level):
    n = 1 << level
    w = n + 1
    n_tet = ix.n_tet(w)
    stride = (n_tet + 32 + 31) // 32 * 32
    C = _coords(w)
    covered = np.zeros(n_tet, dtype=np.int64)
    lanes = np.arange(32)

    def walk(r, ln, j, g, gb):
        while True:
            m = (r >= ln) & (g <= gb + 1)
            if not m.any():
                return
            r[m] -= ln[m]
            ln[m] -= 1
            j[m] += 1

    for t in hg.plane_tiles(level):
        k, nwin = int(t[0]) & 0xFFFF, int(t[0]) >> 16
        Tp, Tm = ix.n_tri(w - k - 1), ix.n_tri(w - k)
        gb = ix.tw(w, 0, n - k - 2, k) + 1
        j = np.full(32, int(t[2]) >> 16)
        r = (int(t[2]) & 0xFFFF) + lanes
        ln = w - k - j
        g = int(t[1]) + lanes
        walk(r, ln, j, g, gb)
        for q in range(nwin):
            if q > 0:
                g += 30
                r += 30
                walk(r, ln, j, g, gb)
            inn = g <= gb + 1
            gq = np.where(inn, g, gb + 1)
            lq = np.where(inn, ln, 3)
            ok = inn & (g <= gb) & (lanes != 0) & (lanes != 31) & (r >= 1) & (r <= ln - 2)
            rows = {"c": gq, "up": gq + lq, "dn": gq - lq - 1, "p1c": gq + Tp + lq, "p1m": gq + Tp,
                    "m1c": gq - Tm - lq - 1, "m1p": gq - Tm}
            for off in rows.values():
                assert off.min() >= 0 and off.max() < stride
            o = np.flatnonzero(ok)
            if not len(o):
                continue
            P = C[gq[o]]
            assert np.all(P > 0) and np.all(P.sum(axis=1) <= n - 1)       # interior points only
            expect = {"c": (0, 0, 0), "up": (0, 1, 0), "dn": (0, -1, 0), "p1c": (0, 0, 1),
                      "p1m": (0, -1, 1), "m1c": (0, 0, -1), "m1p": (0, 1, -1)}
            for name, d in expect.items():
                assert np.array_equal(C[rows[name][o]], P + np.array(d)), name
            # shuffled neighbours: lane - 1 for cm, upm, p1cm, m1pm; lane + 1 for cp, dnp, p1mp, m1cp
            shuf = {("c", -1): (-1, 0, 0), ("c", 1): (1, 0, 0), ("up", -1): (-1, 1, 0),
                    ("dn", 1): (1, -1, 0), ("p1c", -1): (-1, 0, 1), ("p1m", 1): (1, -1, 1),
                    ("m1c", 1): (1, 0, -1), ("m1p", -1): (-1, 1, -1)}
            for (name, dl), d in shuf.items():
                assert np.array_equal(C[rows[name][o + dl]], P + np.array(d)), (name, dl)
            np.add.at(covered, gq[o], 1)
    interior = (C.min(axis=1) > 0) & (C.sum(axis=1) <= n - 1)
    assert np.all(covered[interior] == 1)
    assert np.all(covered[~interior] == 0)
