"""The streaming constant-stencil kernel's plan and index arithmetic, emulated
on the CPU (no GPU).

For every CTA of the library's own plan (hg_stream_plan) and shared-memory
layout (hg_stream_layout) the emulation replays the producer (copy c of the
CTA into slot c mod R) and the consumers' walk over the items (32 columns at
a time marching the rows, the loads of each step, then the boundary points),
with the kernel's virtual slot bases.  It checks that:
  * every bulk copy starts on a 16-byte boundary, stays inside the padded
    cell and fits its slot;
  * an item's copies sit in distinct slots, and every slot phase receives
    exactly the number of arrivals its barrier expects;
  * every shared-memory index any lane forms (also lanes past a row's end,
    whose values are discarded) stays inside the guards around the ring;
  * every lattice point of every cell is formed by exactly one lane;
  * every value a point reads is its lattice neighbour (the 15-point stencil
    of Sec. 5.2 in t_w order, Sec. 4) and lies inside the copy it is read from.
The lattice is checked through the oracle's index function."""
import numpy as np
import pytest

from oracle import indexing as ix

import paper_2308_01792_gb300 as hg

DIRS = [(0, 0, 0), (1, 0, 0), (-1, 0, 0), (0, 1, 0), (0, -1, 0), (0, 0, 1), (0, 0, -1),
        (-1, 1, 0), (1, -1, 0), (-1, 0, 1), (1, 0, -1), (0, -1, 1), (0, 1, -1), (1, -1, 1),
        (-1, 1, -1)]
ARRIVE = 256


def _tw_table(w):
    """Offset of (i, j, k) in I_tet(w), -1 outside (oracle index function)."""
    t = np.full((w + 2, w + 2, w + 2), -1, dtype=np.int64)
    for k in range(w):
        for j in range(w - k):
            for i in range(w - k - j):
                t[i, j, k] = ix.tw(w, i, j, k)
    return t


def _ntri(m):
    return m * (m + 1) // 2 if m > 0 else 0


def _emulate(level, ncells, nctas, dtype_code):
    n = 1 << level
    w = n + 1
    E = 4 if dtype_code == hg.HG_F32 else 8
    V = 16 // E
    n_tet = ix.n_tet(w)
    stride = (n_tet + 32 + 31) // 32 * 32
    R, SE, guard = hg.stream_layout(level, dtype_code)
    P = hg.stream_plan(level, ncells, nctas, dtype_code)
    cop, items, cc, ci = P["copies"], P["items"], P["cta_copies"], P["cta_items"]
    assert cc[0] == 0 and cc[-1] == len(cop) and np.all(np.diff(cc) >= 0)
    assert ci[0] == 0 and ci[-1] == len(items) and np.all(np.diff(ci) >= 0)
    TW = _tw_table(w)
    visits = np.zeros((ncells, n_tet), dtype=np.int64)
    lanes = np.arange(32)
    lo_bound, hi_bound = -guard, R * SE + guard
    for c in cop:
        cell, ga, ne, _ = (int(v) for v in c)
        assert 0 <= cell < ncells and ga % V == 0 and ne % V == 0 and 0 < ne <= SE
        assert ga >= 0 and ga + ne <= stride
    for g in range(nctas):
        ncop = cc[g + 1] - cc[g]
        arrivals = np.zeros(ncop, dtype=np.int64)
        for t in range(ci[g], ci[g + 1]):
            it = [int(v) for v in items[t]]
            cell, k, ja, jb, cnts = it[0], it[1], it[2] & 0xffff, it[2] >> 16, it[3]
            c0, cm, cp = it[4], it[5], it[6]
            ga0, gam, gap = it[8], it[9], it[10]
            assert 0 <= ja < jb <= w - k
            refs = {0: (c0, ga0)}
            if cm >= 0:
                refs[-1] = (cm, gam)
            if cp >= 0:
                refs[1] = (cp, gap)
            for pl, (cx, gx) in refs.items():
                assert 0 <= cx < ncop
                C = cop[cc[g] + cx]
                assert int(C[0]) == cell and int(C[1]) == gx
            distinct = list(dict.fromkeys([c0] + [x for x in (cm, cp) if x >= 0]))
            assert len({x % R for x in distinct}) == len(distinct)
            arrivals[c0] += cnts & 1023
            if cm >= 0 and cm != c0:
                arrivals[cm] += (cnts >> 10) & 1023
            if cp >= 0 and cp != c0 and cp != cm:
                arrivals[cp] += (cnts >> 20) & 1023
            # slot base (in ring elements) minus the copy's first element; a
            # plane that is not in the stream aliases plane k
            vb = {pl: (cx % R) * SE - gx for pl, (cx, gx) in refs.items()}
            vb.setdefault(1, vb[0])
            vb.setdefault(-1, vb[0])
            span = {pl: (gx, gx + int(cop[cc[g] + cx][2])) for pl, (cx, gx) in refs.items()}

            def check(i, valid, j, rs, strict):
                """Neighbours of the points (i, j, k): lattice offsets, inside the copy."""
                ln = w - k - j
                base = {0: vb[0] + rs, 1: vb[1] + rs + _ntri(w - k) - j,
                        -1: vb[-1] + rs - _ntri(w - k + 1) + j}
                rowoff = {(0, 0): 0, (0, 1): ln, (0, -1): -(ln + 1), (1, 0): 0, (1, -1): -ln,
                          (-1, 0): 0, (-1, 1): ln + 1}
                for (di, dj, dk) in DIRS:
                    a, bb, c2 = i + di, j + dj, k + dk
                    inc = (a >= 0) & (bb >= 0) & (c2 >= 0) & (a + bb + c2 <= n)
                    addr = base[dk] + rowoff[(dk, dj)] + a
                    if strict:
                        # every load the interior loop issues, valid lanes or not
                        assert addr.min() >= lo_bound and addr.max() < hi_bound, (level, g, t, j)
                    chk = valid & inc
                    if not chk.any():
                        continue
                    assert dk in refs, (level, k, (di, dj, dk))
                    got = addr[chk] - vb[dk]
                    assert np.array_equal(got, TW[a[chk], bb, c2]), (level, k, j, (di, dj, dk))
                    lo, hi = span[dk]
                    assert got.min() >= lo and got.max() < hi, (level, k, j, (di, dj, dk))

            # interior: 32 columns at a time, marching the rows; every load the
            # kernel issues (also for lanes past a row's end) is in bounds and,
            # for the points it serves, is the lattice point it stands for
            def lds(pl, addr, di, dj, i, j, use):
                """A load of plane k+pl at ring address addr meant for (i+di, j+dj, k+pl)."""
                assert addr.min() >= lo_bound and addr.max() < hi_bound, (level, g, t)
                a, bb, c2 = i + di, j + dj, k + pl
                inc = (a >= 0) & (bb >= 0) & (c2 >= 0) & (a + bb + c2 <= n)
                chk = use & inc
                if chk.any():
                    assert pl in refs
                    got = addr[chk] - vb[pl]
                    assert np.array_equal(got, TW[a[chk], bb, c2]), (level, k, j, (di, dj, pl))
                    lo, hi = span[pl]
                    assert got.min() >= lo and got.max() < hi

            j1 = max(ja, 1)
            if k >= 1 and j1 < jb:
                len1 = w - k - j1
                rs1 = ix.tw(w, 0, j1, k)
                Tk, Tk1 = _ntri(w - k), _ntri(w - k + 1)
                for c0 in range(1, len1 - 1, 32):
                    i = c0 + lanes
                    ln, j = len1, j1
                    a0 = vb[0] + rs1 + i
                    ap = vb[1] + rs1 + Tk - j1 + i
                    am = vb[-1] + rs1 - Tk1 + j1 + i
                    gg = rs1 + i
                    use = i <= ln - 2
                    # the first values: row j at i-1, i, i+1, row j-1 at i, i+1; the
                    # 15-point form's plane k+1 row j-1 and plane k-1 row j at i, i+1
                    lds(0, a0 - 1, -1, 0, i, j, use)
                    lds(0, a0, 0, 0, i, j, use)
                    lds(0, a0 + 1, 1, 0, i, j, use)
                    lds(0, a0 - ln - 1, 0, -1, i, j, use)
                    lds(0, a0 - ln, 1, -1, i, j, use)
                    lds(1, ap - ln, 0, -1, i, j, use)
                    lds(1, ap - ln + 1, 1, -1, i, j, use)
                    lds(-1, am, 0, 0, i, j, use)
                    lds(-1, am + 1, 1, 0, i, j, use)
                    while j < jb and c0 <= ln - 2:
                        use = i <= ln - 2
                        lds(0, a0 + ln - 1, -1, 1, i, j, use)
                        lds(0, a0 + ln, 0, 1, i, j, use)
                        lds(0, a0 + ln + 1, 1, 1, i, j, use)
                        lds(1, ap - ln, 0, -1, i, j, use)
                        lds(-1, am + ln + 1, 0, 1, i, j, use)
                        lds(1, ap - 1, -1, 0, i, j, use)
                        lds(1, ap, 0, 0, i, j, use)
                        lds(1, ap + 1, 1, 0, i, j, use)
                        lds(-1, am + ln, -1, 1, i, j, use)
                        lds(-1, am + ln + 2, 1, 1, i, j, use)
                        visits[cell, gg[use]] += 1
                        assert np.array_equal(gg[use], TW[i[use], j, k])
                        gg = gg + ln
                        a0 = a0 + ln
                        ap = ap + ln - 1
                        am = am + ln + 1
                        ln -= 1
                        j += 1
            # boundary points: whole rows in plane 0 and row 0, row ends elsewhere
            rs = ix.tw(w, 0, ja, k)
            for j in range(ja, jb):
                ln = w - k - j
                ib = np.arange(ln) if (k == 0 or j == 0) else np.array(sorted({0, ln - 1}))
                visits[cell, rs + ib] += 1
                check(ib, np.ones(len(ib), bool), j, rs, False)
                rs += ln
        assert np.all(arrivals == ARRIVE), (g, arrivals)
    assert np.all(visits == 1), np.argwhere(visits != 1)[:5]


@pytest.mark.parametrize("level", [0, 1, 2, 3, 4, 5, 6])
@pytest.mark.parametrize("dtype_code", [hg.HG_F32, hg.HG_F64])
def test_stream_single_cell(level, dtype_code):
    for nctas in (1, 3, 152):
        _emulate(level, 1, nctas, dtype_code)


@pytest.mark.parametrize("level,ncells,nctas,dtype_code",
                         [(3, 6, 152, hg.HG_F32), (4, 6, 7, hg.HG_F64), (4, 48, 152, hg.HG_F32),
                          (7, 1, 152, hg.HG_F32), (7, 1, 152, hg.HG_F64), (8, 1, 152, hg.HG_F32)])
def test_stream_multi_cell_and_bands(level, ncells, nctas, dtype_code):
    _emulate(level, ncells, nctas, dtype_code)


def test_stream_plan_balances_points():
    """The level-7 six-cell FP32 plan over 152 CTAs: no CTA forms more than
    1.35x the mean number of lattice points."""
    level, ncells, nctas = 7, 6, 152
    w = (1 << level) + 1
    P = hg.stream_plan(level, ncells, nctas, hg.HG_F32)
    pts = np.zeros(nctas)
    for g in range(nctas):
        for t in range(P["cta_items"][g], P["cta_items"][g + 1]):
            it = P["items"][t]
            k, ja, jb = it[1], it[2] & 0xffff, it[2] >> 16
            pts[g] += sum(w - k - j for j in range(ja, jb))
    assert pts.sum() == ncells * ix.n_tet(w)
    assert pts.max() <= 1.35 * pts.mean()
