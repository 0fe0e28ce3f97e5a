"""The streaming constant-stencil kernel's schedule and index arithmetic,
emulated on the CPU (no GPU).

For every CTA the emulation replays the producer's plane stream (the staged
row range of each plane of each run, its 16-byte rounding and its ring slot)
and the consumers' walk (the 32-point chunks of every band row, the row
bases in planes k-1, k, k+1 and the fifteen neighbour offsets), with the
library's own schedule (hg_stream_schedule) and shared-memory layout
(hg_stream_layout).  It checks that:
  * every bulk copy starts on a 16-byte boundary, stays inside the padded
    cell and fits its slot;
  * every shared-memory index any lane forms (also lanes past a row's end,
    whose values are discarded) stays inside the guards around the ring;
  * every lattice point of every cell is visited by exactly one lane;
  * the fifteen values an interior point reads are its lattice neighbours
    (the 15-point stencil of Sec. 5.2 in t_w order, Sec. 4), and so are the
    in-cell neighbours a boundary point reads.
The lattice is checked through the oracle's index function."""
import numpy as np
import pytest

from oracle import indexing as ix

import paper_2308_01792_gb300 as hg

DIRS = [(0, 0, 0), (1, 0, 0), (-1, 0, 0), (0, 1, 0), (0, -1, 0), (0, 0, 1), (0, 0, -1),
        (-1, 1, 0), (1, -1, 0), (-1, 0, 1), (1, 0, -1), (0, -1, 1), (0, 1, -1), (1, -1, 1),
        (-1, 1, -1)]
BAND = 8


def _tw_table(w):
    """Offset of (i, j, k) in I_tet(w), -1 outside (oracle index function)."""
    t = np.full((w + 2, w + 2, w + 2), -1, dtype=np.int64)
    for k in range(w):
        for j in range(w - k):
            for i in range(w - k - j):
                t[i, j, k] = ix.tw(w, i, j, k)
    return t


def _row_start(w, j, k):
    return ix.tw(w, 0, j, k)


def _staged(w, j0, rows, kk, V):
    jlo, jhi = max(j0 - 1, 0), min(j0 + rows, w - 1 - kk)
    g0 = _row_start(w, jlo, kk)
    g1 = _row_start(w, jhi, kk) + (w - kk - jhi)
    return g0 & ~(V - 1), (g1 + V - 1) & ~(V - 1)


def _ntri(m):
    return m * (m + 1) // 2 if m > 0 else 0


def _emulate(level, ncells, nctas, dtype_code):
    n = 1 << level
    w = n + 1
    V = 4 if dtype_code == hg.HG_F32 else 2
    esize = 4 if dtype_code == hg.HG_F32 else 8
    n_tet = ix.n_tet(w)
    stride = (n_tet + 32 + 31) // 32 * 32
    R, slot, guard = hg.stream_layout(level, dtype_code)
    units, begin = hg.stream_schedule(level, ncells, nctas)
    assert begin[0] == 0 and begin[-1] == len(units) and np.all(np.diff(begin) >= 0)
    TW = _tw_table(w)
    visits = np.zeros((ncells, n_tet), dtype=np.int64)
    lanes = np.arange(32)
    lo_bound, hi_bound = -guard, R * slot + guard
    for g in range(nctas):
        q = 0
        for u in range(begin[g], begin[g + 1]):
            cell, yy, zz, _ = (int(v) for v in units[u])
            j0, rows, k0, k1 = yy & 0xffff, yy >> 16, zz & 0xffff, zz >> 16
            assert 0 <= cell < ncells and 1 <= rows <= BAND and 0 <= k0 < k1 <= w - j0
            kf, kl = max(k0 - 1, 0), min(k1, w - 1)
            qs, gas = {}, {}
            for kk in range(kf, kl + 1):           # producer: plane kk -> stream position q
                ga, ge = _staged(w, j0, rows, kk, V)
                assert ga >= 0 and ge <= stride and (ga * esize) % 16 == 0
                assert (ge - ga) * esize % 16 == 0 and ge - ga <= slot
                qs[kk], gas[kk] = q, ga
                q += 1
            for k in range(k0, k1):                # consumers
                # planes k-1, k, k+1 sit in three distinct slots while k is computed
                s0 = qs[k] % R
                ga0 = gas[k]
                has_m, has_p = k > kf, k < kl
                gam = gas[k - 1] if has_m else None
                gap = gas[k + 1] if has_p else None
                used = [qs[kk] % R for kk in (k - 1, k, k + 1) if kf <= kk <= kl]
                assert len(set(used)) == len(used)
                # value at ring index idx of the slot holding plane kk: offset ga + (idx - slot base)
                base = {0: s0 * slot}
                if has_m:
                    base[-1] = (qs[k - 1] % R) * slot
                if has_p:
                    base[1] = (qs[k + 1] % R) * slot
                gaof = {0: ga0, -1: gam, 1: gap}
                jn = min(rows, w - k - j0)
                for r in range(jn):
                    j = j0 + r
                    ln = w - k - j
                    rs0 = _row_start(w, j, k)
                    p0 = base[0] + rs0 - ga0
                    pp = base[1] + rs0 + _ntri(w - k) - j - gap if has_p else p0
                    pm = base[-1] + rs0 - _ntri(w - k + 1) + j - gam if has_m else p0
                    for c in range((ln + 31) // 32):
                        i = c * 32 + lanes
                        # every index formed by the unconditional loads
                        idx = np.concatenate([p0 + i, p0 + i + 1, p0 + i - 1, p0 + ln + i - 1,
                                              p0 + i - ln, pp + i - ln, pm + ln + 1 + i,
                                              p0 + ln + i, p0 + i - ln - 1, pp + i, pm + i,
                                              pp + i - 1, pm + i + 1, pp + i - ln + 1, pm + ln + i])
                        assert idx.min() >= lo_bound and idx.max() < hi_bound, (level, g, u, k, j)
                        valid = i < ln
                        visits[cell, rs0 + i[valid]] += 1
                        interior = valid & (i >= 1) & (i <= ln - 2) & (j >= 1) & (k >= 1)
                        rowoff = {(0, 0): p0, (0, 1): p0 + ln, (0, -1): p0 - (ln + 1),
                                  (1, 0): pp, (1, -1): pp - ln, (-1, 0): pm, (-1, 1): pm + ln + 1}
                        pl_of = {(0, 0): 0, (0, 1): 0, (0, -1): 0, (1, 0): 1, (1, -1): 1,
                                 (-1, 0): -1, (-1, 1): -1}
                        for (di, dj, dk) in DIRS:
                            a, b, cc = i + di, j + dj, k + dk
                            inc = (a >= 0) & (b >= 0) & (cc >= 0) & (a + b + cc <= n)
                            check = valid & inc          # interior points: all 15 in the cell
                            assert np.all(inc[interior])
                            if not check.any():
                                continue
                            pl = pl_of[(dk, dj)]
                            ridx = rowoff[(dk, dj)] + a[check]
                            got = gaof[pl] + (ridx - base[pl])
                            exp = TW[a[check], b, cc]
                            assert np.array_equal(got, exp), (level, k, j, (di, dj, dk))
    assert np.all(visits == 1), np.argwhere(visits != 1)[:5]


@pytest.mark.parametrize("level", [0, 1, 2, 3, 4, 5, 6])
@pytest.mark.parametrize("dtype_code", [hg.HG_F32, hg.HG_F64])
def test_stream_single_cell_all_ctas(level, dtype_code):
    for nctas in (1, 3, 152):
        _emulate(level, 1, nctas, dtype_code)


@pytest.mark.parametrize("level,ncells,nctas", [(3, 6, 152), (4, 6, 7), (4, 48, 152), (7, 1, 152)])
def test_stream_multi_cell(level, ncells, nctas):
    _emulate(level, ncells, nctas, hg.HG_F32)


def test_stream_schedule_balances_cost():
    """The level-7 six-cell schedule over 152 CTAs: no CTA gets more than 1.3x
    the mean number of lattice points."""
    level, ncells, nctas = 7, 6, 152
    w = (1 << level) + 1
    units, begin = hg.stream_schedule(level, ncells, nctas)
    pts = np.zeros(nctas)
    for g in range(nctas):
        for u in range(begin[g], begin[g + 1]):
            _, yy, zz, _ = units[u]
            j0, rows, k0, k1 = yy & 0xffff, yy >> 16, zz & 0xffff, zz >> 16
            for k in range(k0, k1):
                for j in range(j0, min(j0 + rows, w - k)):
                    pts[g] += w - k - j
    assert pts.sum() == ncells * ix.n_tet(w)
    assert pts.max() <= 1.3 * pts.mean()
