"""P2 (vertex + edge DoFs) parity against the oracle through the C ABI.

The GPU stores a P2 function of level L on the vertex lattice of level L+1;
its canonical numbering and Dirichlet set must be the oracle's P2 numbering
(doubled-lattice keys).  Operators are element-wise with on-the-fly element
matrices (stiffness with k = a + b sin 2 pi x sin 2 pi y sin 2 pi z by the
14-point rule, mass); the oracle assembles the same element matrices into
CSR.  Bars: FP64 1e-12 relative, FP32 1e-5 relative, copies bit-identical,
transfers equal to the oracle's quadratic interpolation and its transpose,
V-cycle iterates within 1e-12 of the oracle's, solves to the same discrete
solution."""
import numpy as np
import pytest
import scipy.sparse.linalg as spla

import synthgen as sg
from oracle import gmg as og

from helpers import rel_err

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

import paper_2308_01792_gb300 as hg

P2 = hg.HG_SPACE_P2
AB = sg.SINPROD_AB
KFUN = sg.sinprod_coefficient(*AB)
CASES = [(sg.kuhn_cube(1), 2), (sg.kuhn_cube(1), 3), (sg.kuhn_cube(2), 2), (sg.reference_tet(), 3),
         (sg.permuted_cells(sg.kuhn_cube(1), 3), 2)]
IDS = ["cube1_L2", "cube1_L3", "cube2_L2", "tet_L3", "cube1perm_L2"]


@pytest.fixture(scope="module", params=range(len(CASES)), ids=IDS)
def setup(request):
    macro, L = CASES[request.param]
    H = hg.Hierarchy(hg.Mesh(macro.xyz, macro.cells), 0, L + 1)
    ops = {"stiff": hg.Operator(H, hg.HG_OP_P2_DIVKGRAD, coeff=AB),
           "mass": hg.Operator(H, hg.HG_OP_P2_MASS)}
    lev = og.Level(macro, L, space="P2", coeff=KFUN)
    return macro, L, H, ops, lev


def _stored(H, L, c, dtype=torch.float64):
    return H.from_canonical(L, torch.tensor(c, dtype=dtype, device="cuda"), space=P2)


def _canon(H, L, x):
    return H.to_canonical(L, x, space=P2).cpu().double().numpy()


def test_p2_numbering_matches_oracle(setup):
    macro, L, H, ops, lev = setup
    s2c, xyz, dirich = H.canonical_info(L, space=P2)
    assert len(xyz) == lev.n
    assert np.array_equal(xyz, lev.xyz)
    assert np.array_equal(dirich, lev.boundary)
    ns, nu, ni, stride = H.size(L, space=P2)
    assert nu == lev.n and ni == len(lev.interior)


@pytest.mark.parametrize("which", ["stiff", "mass"])
@pytest.mark.parametrize("dtype,tol", [(torch.float64, 1e-12), (torch.float32, 1e-5)])
def test_p2_apply_matches_oracle(setup, which, dtype, tol):
    macro, L, H, ops, lev = setup
    A = lev.A_full if which == "stiff" else lev.M_full
    xc = sg.uniform_vector(21, lev.n)
    x = _stored(H, L, xc, dtype)
    ref = A @ (xc.astype(np.float32).astype(np.float64) if dtype == torch.float32 else xc)
    y = H.zeros(L, dtype, space=P2)
    ops[which].apply(L, x, y, mask=hg.HG_MASK_ALL)
    got = _canon(H, L, y)
    assert rel_err(got, ref) <= tol
    # INNER on a nonzero destination: interior rows, Dirichlet rows set to 0
    # (REPLACE), and y + A x on the interior rows (ADD)
    y0 = sg.uniform_vector(23, lev.n)
    y0r = torch.tensor(y0, dtype=dtype).double().numpy()
    y2 = _stored(H, L, y0, dtype)
    ops[which].apply(L, x, y2)
    got2 = _canon(H, L, y2)
    assert rel_err(got2[lev.interior], ref[lev.interior]) <= tol
    assert np.all(got2[lev.boundary] == 0)
    y3 = _stored(H, L, y0, dtype)
    ops[which].apply(L, x, y3, mode=hg.HG_ADD)
    got3 = _canon(H, L, y3)
    assert rel_err(got3[lev.interior], (y0r + ref)[lev.interior]) <= 2 * tol
    assert np.all(got3[lev.boundary] == 0)


def test_p2_copies_bit_identical(setup):
    macro, L, H, ops, lev = setup
    s2c, _, _ = H.canonical_info(L, space=P2)
    x = _stored(H, L, sg.uniform_vector(22, lev.n))
    y = H.zeros(L, torch.float64, space=P2)
    ops["stiff"].apply(L, x, y, mask=hg.HG_MASK_ALL)
    ys = y.cpu().numpy()
    yc = _canon(H, L, y)
    m = s2c >= 0
    assert np.array_equal(ys[m], yc[s2c[m]])


def test_p2_residual_and_jacobi(setup):
    macro, L, H, ops, lev = setup
    xc = sg.uniform_vector(23, lev.n)
    bc = sg.uniform_vector(24, lev.n)
    xc[lev.boundary] = 0.0
    x, b = _stored(H, L, xc), _stored(H, L, bc)
    r = H.zeros(L, torch.float64, space=P2)
    ops["stiff"].residual(L, x, b, r)
    rc = _canon(H, L, r)
    ii = lev.interior
    ref = bc[ii] - lev.A @ xc[ii]
    assert rel_err(rc[ii], ref) <= 1e-12 and np.all(rc[lev.boundary] == 0)
    xo = H.zeros(L, torch.float64, space=P2)
    ops["stiff"].jacobi(L, x, b, xo, omega=2.0 / 3.0)
    xj = _canon(H, L, xo)
    refj = og.jacobi(lev.A, lev.D, xc[ii], bc[ii], 2.0 / 3.0)
    assert rel_err(xj[ii], refj) <= 1e-12
    assert np.all(xj[lev.boundary] == xc[lev.boundary])


def test_p2_transfers_match_oracle(setup):
    macro, L, H, ops, lev = setup
    co = og.Level(macro, L - 1, space="P2")
    P = og.p2_prolongation(lev, co)
    ec = sg.uniform_vector(25, co.n)
    ec[co.boundary] = 0.0
    xf = H.zeros(L, torch.float64, space=P2)
    H.prolong_add(L, _stored(H, L - 1, ec), xf, space=P2)
    got = _canon(H, L, xf)
    ref = P @ ec
    assert rel_err(got[lev.interior], ref[lev.interior]) <= 1e-14
    assert np.all(got[lev.boundary] == 0)
    rf = sg.uniform_vector(26, lev.n)
    rf[lev.boundary] = 0.0
    rc = H.zeros(L - 1, torch.float64, space=P2)
    H.restrict(L, _stored(H, L, rf), rc, space=P2)
    gc = _canon(H, L - 1, rc)
    refr = P.T @ rf
    assert rel_err(gc[co.interior], refr[co.interior]) <= 1e-13
    assert np.all(gc[co.boundary] == 0)


def test_p2_vcycle_iterates_match_oracle(setup):
    macro, L, H, ops, lev = setup
    G = hg.GMG(ops["stiff"], lmin=0)
    Ho = og.Hierarchy(macro, 0, L, space="P2", coeff=KFUN)
    bc = np.zeros(lev.n)
    bc[lev.interior] = sg.uniform_vector(27, len(lev.interior))
    b = _stored(H, L, bc)
    x = H.zeros(L, torch.float64, space=P2)
    xo = np.zeros(len(lev.interior))
    for cyc in range(3):
        G.vcycle(L, x, b)
        xo = og.vcycle(Ho, L, xo, bc[lev.interior])
        got = _canon(H, L, x)
        assert rel_err(got[lev.interior], xo) <= 1e-12, cyc
        assert np.all(got[lev.boundary] == 0)


@pytest.mark.parametrize("precision", [hg.HG_PREC_F64, hg.HG_PREC_MIXED])
def test_p2_solve_manufactured(setup, precision):
    macro, L, H, ops, lev = setup
    tol = 1e-10
    _, xyz, dirich = H.canonical_info(L, space=P2)
    _, f = sg.sinprod_manufactured(xyz, *AB)
    b = H.zeros(L, torch.float64, space=P2)
    ops["mass"].apply(L, _stored(H, L, f), b)
    bo = (lev.M_full @ f)[lev.interior]
    bg = _canon(H, L, b)
    assert rel_err(bg[lev.interior], bo) <= 1e-12
    G = hg.GMG(ops["stiff"], lmin=0)
    x = H.zeros(L, torch.float64, space=P2)
    it, rel = G.solve(x, b, tol=tol, max_iter=80, precision=precision)
    xg = _canon(H, L, x)[lev.interior]
    ro = np.linalg.norm(bo - lev.A @ xg) / np.linalg.norm(bo)
    assert rel <= tol and ro <= tol * 1.01
    xd = spla.spsolve(lev.A.tocsc(), bo)
    assert np.linalg.norm(xg - xd) <= 1e3 * tol * np.linalg.norm(xd)


def test_p2_divkgrad_rejects_a_coefficient_that_is_not_positive():
    """k = a + b sin(2 pi x) sin(2 pi y) sin(2 pi z) ranges over [a - |b|,
    a + |b|], so creation needs finite a > |b|; {a, b} must be two values."""
    macro = sg.kuhn_cube(1)
    H = hg.Hierarchy(hg.Mesh(macro.xyz, macro.cells), 0, 3)
    for bad in ((0.5, 0.5), (1.0, -1.5), (-1.0, 0.0), (np.nan, 0.0), (1.0, np.inf)):
        with pytest.raises(hg.HGError) as e:
            hg.Operator(H, hg.HG_OP_P2_DIVKGRAD, coeff=bad)
        assert e.value.code == -1 and "a > |b|" in str(e.value)
    with pytest.raises(ValueError):
        hg.Operator(H, hg.HG_OP_P2_DIVKGRAD, coeff=(1.0,))
    hg.Operator(H, hg.HG_OP_P2_DIVKGRAD, coeff=(1.0, 0.99))
