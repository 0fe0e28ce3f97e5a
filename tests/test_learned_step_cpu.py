"""The learned smoothing step's row windows (learned_step_kernel), emulated on
the CPU (no GPU).

One warp per lattice row (j, k) of a cell, windows of 30 points: lane l holds
column i = i0 - 1 + l (i0 = 0, 30, ...), its load column max(i, 0); in rows
with cell-interior points (j, k >= 1, row length >= 3) every lane loads r and
1/D at its column on the seven neighbour rows (plane k rows j, j+1, j-1; plane
k+1 rows j, j-1; plane k-1 rows j, j+1) and the i -/+ 1 neighbours come from
lanes l -/+ 1.  The emulation checks, for every level up to 7, that every load
index stays inside the padded cell (cell stride = roundup(N_tet + 32, 32)),
that each interior point (i, j, k >= 1, i + j + k <= n - 1) is produced by
exactly one lane with all 15 features equal to its lattice neighbours in the
15-point order of Sec. 5.2 (t_w of Sec. 4, through the oracle's index
function), and that every lattice point is written exactly once."""
import numpy as np
import pytest

from oracle import indexing as ix

DIRS = [(0, 0, 0), (1, 0, 0), (-1, 0, 0), (0, 1, 0), (0, -1, 0), (0, 0, 1), (0, 0, -1),
        (-1, 1, 0), (1, -1, 0), (-1, 0, 1), (1, 0, -1), (0, -1, 1), (0, 1, -1), (1, -1, 1),
        (-1, 1, -1)]
# direction d: (row of the seven, lane shift): row 0 c, 1 j+1, 2 j-1, 3 (k+1, j),
# 4 (k+1, j-1), 5 (k-1, j), 6 (k-1, j+1); shift -1 = lane l-1 (i-1), +1 = lane l+1
SRC = [(0, 0), (0, +1), (0, -1), (1, 0), (2, 0), (3, 0), (5, 0), (1, -1), (2, +1), (3, -1),
       (5, +1), (4, 0), (6, 0), (4, +1), (6, -1)]


def _ntri(m):
    return m * (m + 1) // 2 if m > 0 else 0


@pytest.mark.parametrize("level", [1, 2, 3, 4, 5, 6, 7])
def test_learned_step_windows_load_in_bounds_and_gather_the_neighbourhood(level):
    n = 1 << level
    w = n + 1
    ntet = ix.n_tet(w)
    stride = (ntet + 32 + 31) // 32 * 32
    lanes = np.arange(32)
    written = np.zeros(ntet, dtype=np.int64)
    interior_seen = np.zeros(ntet, dtype=np.int64)
    for k in range(w):
        for j in range(w - k):
            ln = w - k - j
            r0 = ix.tw(w, 0, j, k)
            nbr = j >= 1 and k >= 1 and ln >= 3
            rows = [r0, r0 + ln, r0 - (ln + 1), r0 + _ntri(w - k - 1) + ln,
                    r0 + _ntri(w - k - 1), r0 - _ntri(w - k) - (ln + 1), r0 - _ntri(w - k)]
            for i0 in range(0, ln, 30):
                i = i0 - 1 + lanes
                il = np.maximum(i, 0)
                used = [0] + (list(range(1, 7)) if nbr else [])
                for m in used:
                    idx = rows[m] + il
                    assert idx.min() >= 0 and idx.max() < stride, (level, j, k, m)
                out = (lanes >= 1) & (lanes <= 30) & (i <= ln - 1)
                written[r0 + i[out]] += 1
                if not nbr:
                    continue
                interior = out & (i >= 1) & (i <= ln - 2)
                for lane in np.flatnonzero(interior):
                    ii = int(i[lane])
                    assert ii + j + k <= n - 1
                    interior_seen[ix.tw(w, ii, j, k)] += 1
                    for d, (m, sh) in enumerate(SRC):
                        src_lane = lane + sh
                        assert 0 <= src_lane < 32
                        got = rows[m] + int(il[src_lane])
                        di, dj, dk = DIRS[d]
                        assert got == ix.tw(w, ii + di, j + dj, k + dk), (level, ii, j, k, d)
    assert np.all(written == 1)
    want = np.zeros(ntet, dtype=np.int64)
    for k in range(1, n):
        for j in range(1, n - k):
            for i in range(1, n - k - j):
                want[ix.tw(w, i, j, k)] = 1
    assert np.array_equal(interior_seen, want)
