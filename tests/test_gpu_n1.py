"""Lowest-order Nedelec operator alpha curl curl + beta I through the C ABI
against the oracle's assembled matrices (oracle.nedelec).

N1 DoFs are stored as P2-space vectors at the edge-midpoint points; in the
P2 canonical order the edge points must be exactly the oracle's N1 DoFs (same
keys, same order) with the same boundary set.  Bars: apply (ALL and INNER
masks), residual and Jacobi within 1e-12 (FP64) / 1e-5 (FP32) relative,
vertex points 0, interface copies bit-identical."""
import numpy as np
import pytest

import synthgen as sg
from oracle import fem
from oracle import nedelec as ne
from oracle.mesh import coord_key

from helpers import rel_err

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

import paper_2308_01792_gb300 as hg

P2 = hg.HG_SPACE_P2
AB = (1.0, 0.3)
TOL = {torch.float64: 1e-12, torch.float32: 1e-5}
CASES = [(sg.kuhn_cube(1), 2), (sg.reference_tet(), 3), (sg.permuted_cells(sg.kuhn_cube(1), 3), 2),
         (sg.kuhn_cube(2), 2)]
IDS = ["cube1_L2", "tet_L3", "cube1perm_L2", "cube2_L2"]


@pytest.fixture(scope="module", params=range(len(CASES)), ids=IDS)
def case(request):
    macro, L = CASES[request.param]
    H = hg.Hierarchy(hg.Mesh(macro.xyz, macro.cells), 0, L + 1)
    op = hg.Operator(H, hg.HG_OP_N1_CURLCURL, coeff=AB)
    lev = ne.NedelecLevel(macro, L, *AB)
    num = fem.P2Numbering(lev.rm)
    edge = np.flatnonzero(np.any(num.coords2 % 2 == 1, axis=1))
    return macro, L, H, op, lev, num, edge


def _stored(H, L, n_p2, edge, vals, dtype):
    full = np.zeros(n_p2)
    full[edge] = vals
    return H.from_canonical(L, torch.tensor(full, dtype=dtype, device="cuda"), space=P2)


def _canon(H, L, y):
    return H.to_canonical(L, y, space=P2).cpu().double().numpy()


def test_n1_dofs_are_the_p2_edge_points(case):
    macro, L, H, op, lev, num, edge = case
    assert np.array_equal(coord_key(num.coords2[edge], 2 * lev.rm.side), lev.keys)
    _, _, dirich = H.canonical_info(L, space=P2)
    assert np.array_equal(dirich[edge], lev.boundary)


@pytest.mark.parametrize("dtype", [torch.float64, torch.float32])
def test_n1_apply_matches_oracle(case, dtype):
    macro, L, H, op, lev, num, edge = case
    xe = sg.uniform_vector(50, lev.n)
    if dtype == torch.float32:
        xe = xe.astype(np.float32).astype(np.float64)
    x = _stored(H, L, num.n, edge, xe, dtype)
    y = H.zeros(L, dtype, space=P2)
    op.apply(L, x, y, mask=hg.HG_MASK_ALL)
    got = _canon(H, L, y)
    assert rel_err(got[edge], lev.A_full @ xe) <= TOL[dtype]
    vert = np.setdiff1d(np.arange(num.n), edge)
    assert np.all(got[vert] == 0)
    # INNER mask on a vector with zero tangential boundary values
    xi = xe.copy()
    xi[lev.boundary] = 0
    x = _stored(H, L, num.n, edge, xi, dtype)
    y = H.zeros(L, dtype, space=P2)
    op.apply(L, x, y)
    got = _canon(H, L, y)
    ii = lev.interior
    assert rel_err(got[edge][ii], (lev.A_full @ xi)[ii]) <= TOL[dtype]
    assert np.all(got[edge][lev.boundary] == 0)
    # INNER on a nonzero destination (edge points), both modes: Dirichlet
    # edges 0, vertex points keep 0
    y0 = sg.uniform_vector(54, lev.n)
    y0r = torch.tensor(y0, dtype=dtype).double().numpy()
    for mode, base in ((hg.HG_REPLACE, 0.0), (hg.HG_ADD, y0r)):
        y = _stored(H, L, num.n, edge, y0, dtype)
        op.apply(L, x, y, mode=mode)
        got = _canon(H, L, y)
        assert rel_err(got[edge][ii], (base + lev.A_full @ xi)[ii]) <= 2 * TOL[dtype]
        assert np.all(got[edge][lev.boundary] == 0)
        assert np.all(got[vert] == 0)


def test_n1_copies_bit_identical(case):
    macro, L, H, op, lev, num, edge = case
    s2c, _, _ = H.canonical_info(L, space=P2)
    x = _stored(H, L, num.n, edge, sg.uniform_vector(51, lev.n), torch.float64)
    y = H.zeros(L, torch.float64, space=P2)
    op.apply(L, x, y, mask=hg.HG_MASK_ALL)
    ys = y.cpu().numpy()
    yc = _canon(H, L, y)
    m = s2c >= 0
    assert np.array_equal(ys[m], yc[s2c[m]])


@pytest.mark.parametrize("dtype", [torch.float64, torch.float32])
def test_n1_residual_and_jacobi_match_oracle(case, dtype):
    macro, L, H, op, lev, num, edge = case
    ii = lev.interior
    xe = np.zeros(lev.n)
    be = np.zeros(lev.n)
    xe[ii] = sg.uniform_vector(52, len(ii))
    be[ii] = sg.uniform_vector(53, len(ii))
    if dtype == torch.float32:
        xe, be = xe.astype(np.float32).astype(np.float64), be.astype(np.float32).astype(np.float64)
    x = _stored(H, L, num.n, edge, xe, dtype)
    b = _stored(H, L, num.n, edge, be, dtype)
    r = H.zeros(L, dtype, space=P2)
    op.residual(L, x, b, r)
    got = _canon(H, L, r)[edge]
    assert rel_err(got[ii], be[ii] - lev.A @ xe[ii]) <= TOL[dtype] * 4
    xo = H.zeros(L, dtype, space=P2)
    op.jacobi(L, x, b, xo, omega=0.5)
    got = _canon(H, L, xo)[edge]
    ref = xe[ii] + 0.5 * (be[ii] - lev.A @ xe[ii]) / lev.D
    assert rel_err(got[ii], ref) <= TOL[dtype] * 4
    assert np.all(got[lev.boundary] == 0)


def test_n1_rejects_bad_coefficients():
    macro = sg.kuhn_cube(1)
    H = hg.Hierarchy(hg.Mesh(macro.xyz, macro.cells), 0, 3)
    with pytest.raises(hg.HGError):
        hg.Operator(H, hg.HG_OP_N1_CURLCURL, coeff=(1.0, 0.0))
