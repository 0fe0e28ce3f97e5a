"""The column-march constant-stencil kernel's items and loads, emulated on the
CPU (no GPU) over the library's own items (hg_march_items).

For every item and lane the emulation replays the kernel's row march: the
clamped column, every load it issues (the seven-point and the general
15-point forms) and the rotation of the centre rows.  It checks that every
load index lies inside the cell's lattice storage, that every cell-interior
point (i, j, k >= 1, i + j + k <= n - 1) is stored by exactly one lane, and
that each value a stored point uses is its lattice neighbour in the stencil
direction it is weighted with (the 15-point order of Sec. 5.2, t_w of Sec. 4,
through the oracle's index function)."""
import numpy as np
import pytest

from oracle import indexing as ix

import paper_2308_01792_gb300 as hg


def _ntri(m):
    return m * (m + 1) // 2 if m > 0 else 0


def _emulate(level):
    n = 1 << level
    w = n + 1
    ntet = ix.n_tet(w)
    stride = (ntet + 32 + 31) // 32 * 32
    TW = {}
    for k in range(w):
        for j in range(w - k):
            for i in range(w - k - j):
                TW[(i, j, k)] = ix.tw(w, i, j, k)
    items = hg.march_items(level)
    seen = np.zeros(ntet, dtype=np.int64)
    lanes = np.arange(32)

    def ld(idx):
        assert idx.min() >= 0 and idx.max() < stride, (level, idx.min(), idx.max())
        return idx

    def expect(idx, ok, i, j, k, di, dj, dk):
        for q in np.flatnonzero(ok):
            assert idx[q] == TW[(i[q] + di, j + dj, k + dk)], (level, i[q], j, k, di, dj, dk)

    for kx, jy in items:
        k, i0, j0, j1 = kx & 0xffff, kx >> 16, jy & 0xffff, jy >> 16
        assert 1 <= k and 1 <= j0 < j1 and i0 >= 1
        Tp, Tm = _ntri(w - k - 1), _ntri(w - k)
        i = i0 + lanes
        ln = w - k - j0
        r0 = ix.tw(w, 0, j0, k)
        ic = np.minimum(i, ln - 2)
        # centre triple of row j0 and row j0 - 1 at i, i + 1
        cen = [ld(r0 + ic - 1), ld(r0 + ic), ld(r0 + ic + 1)]
        dn = [ld(r0 - ln - 1 + ic), ld(r0 - ln + ic)]
        ok0 = i <= ln - 2
        expect(cen[1], ok0, i, j0, k, 0, 0, 0)
        expect(dn[0], ok0, i, j0, k, 0, -1, 0)
        for j in range(j0, j1):
            ic = np.minimum(i, ln - 2)
            ok = i <= ln - 2
            assert ok[0], (level, k, i0, j)                 # lane 0 has a point on every row
            rjp = r0 + ln
            nxt = [ld(rjp + ic - 1), ld(rjp + ic), ld(rjp + ic + 1)]
            p1m, m1p = ld(r0 + Tp + ic), ld(r0 - Tm + ic)
            rkp, rkm = r0 + Tp + ln, r0 - Tm - ln - 1
            gen = {5: ld(rkp + ic), 9: ld(rkp + ic - 1), 13: ld(r0 + Tp + ic + 1),
                   6: ld(rkm + ic), 10: ld(rkm + ic + 1), 14: ld(r0 - Tm + ic - 1)}
            # the values each stored point is weighted with, by direction
            expect(cen[1], ok, i, j, k, 0, 0, 0)
            expect(cen[2], ok, i, j, k, 1, 0, 0)
            expect(cen[0], ok, i, j, k, -1, 0, 0)
            expect(nxt[1], ok, i, j, k, 0, 1, 0)
            expect(dn[0], ok, i, j, k, 0, -1, 0)
            expect(nxt[0], ok, i, j, k, -1, 1, 0)
            expect(dn[1], ok, i, j, k, 1, -1, 0)
            expect(p1m, ok, i, j, k, 0, -1, 1)
            expect(m1p, ok, i, j, k, 0, 1, -1)
            expect(gen[5], ok, i, j, k, 0, 0, 1)
            expect(gen[9], ok, i, j, k, -1, 0, 1)
            expect(gen[13], ok, i, j, k, 1, -1, 1)
            expect(gen[6], ok, i, j, k, 0, 0, -1)
            expect(gen[10], ok, i, j, k, 1, 0, -1)
            expect(gen[14], ok, i, j, k, -1, 1, -1)
            out = r0 + i[ok]
            assert all(o == TW[(ii, j, k)] for o, ii in zip(out, i[ok]))
            seen[out] += 1
            dn = [cen[1], cen[2]]
            cen = nxt
            r0 = rjp
            ln -= 1
    interior = [TW[(i, j, k)] for k in range(1, n) for j in range(1, n - k)
                for i in range(1, n - k - j)]
    mask = np.zeros(ntet, dtype=bool)
    mask[interior] = True
    assert np.all(seen[mask] == 1) and np.all(seen[~mask] == 0), level


@pytest.mark.parametrize("level", [0, 1, 2, 3, 4, 5, 6])
def test_march_items_cover_interior_and_load_neighbours(level):
    _emulate(level)
