"""Parity at the full workload sizes on sampled outputs the oracle computes one
by one (through the C ABI, in the launch configuration the bench times).

For a sample of points well inside random macro cells, the oracle forms the
element matrices (oracle.fem) of every micro-cell incident to the point and
sums its row: y_i = sum_T K_T[a_i, :] x_T.  The GPU output at the same
point must agree to 1e-12 of the row's term magnitudes (FP64).  Workloads:
- P2 -div(k grad), k = 1 + 0.5 sin sin sin, unit cube as 48 Kuhn cells,
  P2 level 6 (16 974 593 DoFs);
- P1 -div(k grad), log-normal k (seed 1000), 384 Kuhn cells, level 6
  (16 974 593 DoFs), on-the-fly and stored-stencil forms;
plus the closed-form 7-point identity of the P1 Laplacian on 384 cells."""
import numpy as np
import pytest

import synthgen as sg
from oracle import fem
from oracle import indexing as ix

from helpers import rel_err

torch = pytest.importorskip("torch")
pytestmark = [pytest.mark.gpu, pytest.mark.slow]

import paper_2308_01792_gb300 as hg

TYPES = [[(0, 0, 0), (1, 0, 0), (0, 1, 0), (0, 0, 1)], [(1, 1, 0), (1, 0, 1), (0, 1, 1), (1, 1, 1)],
         [(0, 1, 0), (1, 0, 1), (1, 0, 0), (0, 0, 1)], [(0, 1, 0), (1, 0, 1), (0, 0, 1), (0, 1, 1)],
         [(0, 1, 0), (1, 0, 1), (0, 1, 1), (1, 1, 0)], [(0, 1, 0), (1, 0, 1), (1, 1, 0), (1, 0, 0)]]
DELTA = [0, 2, 1, 1, 1, 1]
EDGES = [(0, 1), (0, 2), (0, 3), (1, 2), (1, 3), (2, 3)]


def _cell_xyz(macro, c):
    V = macro.xyz[macro.cells[c]]
    return V[0], V[1] - V[0], V[2] - V[0], V[3] - V[0]


def _micro_cells_at(n, pt, scale):
    """Micro-cells (type, anchor) of level n whose DoF points (in `scale` units
    per level unit: 1 for P1 vertices, 2 for the doubled P2 lattice) include
    pt, with the point's local DoF index."""
    out = []
    lo = [max(0, (pt[d] - scale) // scale) for d in range(3)]
    hi = [pt[d] // scale for d in range(3)]
    for i in range(lo[0], hi[0] + 1):
        for j in range(lo[1], hi[1] + 1):
            for k in range(lo[2], hi[2] + 1):
                for t in range(6):
                    if i + j + k > n - 1 - DELTA[t]:
                        continue
                    o = [np.array(v) for v in TYPES[t]]
                    p = np.array([i, j, k])
                    dofs = [scale * p + scale * v for v in o]
                    if scale == 2:
                        dofs += [2 * p + o[a] + o[b] for a, b in EDGES]
                    for a, q in enumerate(dofs):
                        if tuple(q) == tuple(pt):
                            out.append((t, p, a))
    return out


def _sample_points(rng, n_lat, margin, count):
    pts = []
    while len(pts) < count:
        p = rng.integers(margin, n_lat - 2 * margin + 1, size=3)
        if p.sum() <= n_lat - margin:
            pts.append(tuple(int(v) for v in p))
    return pts


def test_p2_stiffness_full_size_sampled_rows():
    macro, L = sg.kuhn_cube(2), 6
    n, N = 1 << L, 2 << L                         # level-6 intervals, doubled lattice
    P2 = hg.HG_SPACE_P2
    H = hg.Hierarchy(hg.Mesh(macro.xyz, macro.cells), L - 1, L + 1)
    op = hg.Operator(H, hg.HG_OP_P2_DIVKGRAD, coeff=sg.SINPROD_AB)
    ns, nu, _, stride = H.size(L, space=P2)
    assert nu == 257 ** 3
    s2c, _, _ = H.canonical_info(L, space=P2)
    xc = sg.uniform_vector(61, nu)
    x = H.from_canonical(L, torch.tensor(xc, device="cuda"), space=P2)
    y = H.zeros(L, torch.float64, space=P2)
    op.apply(L, x, y, mask=hg.HG_MASK_ALL)
    yc = H.to_canonical(L, y, space=P2).cpu().numpy()
    kfun = sg.sinprod_coefficient(*sg.SINPROD_AB)
    rng = np.random.Generator(np.random.PCG64(62))
    w2 = N + 1
    for s in range(96):
        c = int(rng.integers(0, len(macro.cells)))
        pt = _sample_points(rng, N, 3, 1)[0]
        v0, e1, e2, e3 = _cell_xyz(macro, c)
        inc = _micro_cells_at(n, pt, 2)
        assert 1 <= len(inc) <= 64
        acc, scale = 0.0, 0.0
        for t, p, a in inc:
            o = [np.array(v) for v in TYPES[t]]
            X = np.array([v0 + ((p + ov) @ np.stack([e1, e2, e3])) / n for ov in o])
            Ke = fem.p2_stiffness(X[None], kfun)[0]
            dof_pts = [2 * p + 2 * ov for ov in o] + [2 * p + o[u] + o[v] for u, v in EDGES]
            xv = np.array([xc[s2c[c * stride + ix.tw(w2, *q)]] for q in dof_pts])
            acc += Ke[a] @ xv
            scale += np.abs(Ke[a] * xv).sum()
        got = yc[s2c[c * stride + ix.tw(w2, *pt)]]
        assert abs(got - acc) <= 1e-12 * scale, (s, c, pt, got, acc)


@pytest.mark.parametrize("kind", [hg.HG_OP_P1_DIVKGRAD, hg.HG_OP_P1_DIVKGRAD_STORED],
                         ids=["onthefly", "stored"])
def test_p1_divkgrad_full_size_sampled_rows(kind):
    macro, L = sg.kuhn_cube(4), 6
    n = 1 << L
    H = hg.Hierarchy(hg.Mesh(macro.xyz, macro.cells), L, L)
    s2c, xyz, _ = H.canonical_info(L)
    ns, nu, _, stride = H.size(L)
    assert nu == 257 ** 3
    k = sg.rff_eval_torch(sg.rff_params(1000), xyz)          # the workload's field, FP64
    op = hg.Operator(H, kind, coeff=k)
    xc = sg.uniform_vector(63, nu)
    x = H.from_canonical(L, torch.tensor(xc, device="cuda"))
    y = H.zeros(L, torch.float64)
    op.apply(L, x, y, mask=hg.HG_MASK_ALL)
    yc = H.to_canonical(L, y).cpu().numpy()
    rng = np.random.Generator(np.random.PCG64(64))
    w = n + 1
    for s in range(128):
        c = int(rng.integers(0, len(macro.cells)))
        pt = _sample_points(rng, n, 2, 1)[0]
        v0, e1, e2, e3 = _cell_xyz(macro, c)
        inc = _micro_cells_at(n, pt, 1)
        assert len(inc) == 24                            # interior vertex: 4 per subgroup
        acc, scale = 0.0, 0.0
        for t, p, a in inc:
            o = [np.array(v) for v in TYPES[t]]
            X = np.array([v0 + ((p + ov) @ np.stack([e1, e2, e3])) / n for ov in o])
            idx = [s2c[c * stride + ix.tw(w, *(p + ov))] for ov in o]
            Ke = fem.p1_divkgrad(X[None], k[idx][None])[0]
            xv = xc[idx]
            acc += Ke[a] @ xv
            scale += np.abs(Ke[a] * xv).sum()
        got = yc[s2c[c * stride + ix.tw(w, *pt)]]
        assert abs(got - acc) <= 1e-12 * scale, (s, c, pt, got, acc)


def test_p1_laplace_384_cells_is_seven_point():
    """Kuhn cube with 4^3 sub-cubes, level 6 (257^3 DoFs): the P1 Laplacian is
    h times the 7-point stencil (closed form) in FP64 and FP32."""
    macro, L = sg.kuhn_cube(4), 6
    N = 4 << L
    h = 1.0 / N
    H = hg.Hierarchy(hg.Mesh(macro.xyz, macro.cells), L, L)
    op = hg.Operator(H)
    for dtype, tol in ((torch.float64, 1e-12), (torch.float32, 1e-5)):
        xc = sg.uniform_vector(65, (N + 1) ** 3)
        x3 = xc.reshape(N + 1, N + 1, N + 1).copy()
        x3[0], x3[-1], x3[:, 0], x3[:, -1], x3[:, :, 0], x3[:, :, -1] = 0, 0, 0, 0, 0, 0
        x = H.from_canonical(L, torch.tensor(x3.ravel(), dtype=dtype, device="cuda"))
        y = H.zeros(L, dtype)
        op.apply(L, x, y)
        yc = H.to_canonical(L, y).cpu().double().numpy().reshape(N + 1, N + 1, N + 1)
        ref = np.zeros_like(x3)
        c = x3[1:-1, 1:-1, 1:-1]
        ref[1:-1, 1:-1, 1:-1] = h * (6 * c - x3[:-2, 1:-1, 1:-1] - x3[2:, 1:-1, 1:-1]
                                     - x3[1:-1, :-2, 1:-1] - x3[1:-1, 2:, 1:-1]
                                     - x3[1:-1, 1:-1, :-2] - x3[1:-1, 1:-1, 2:])
        assert rel_err(yc, ref) <= tol
