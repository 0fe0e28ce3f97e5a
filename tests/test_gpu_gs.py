"""4-colour Gauss-Seidel (smoother option of the P1 multigrid) through the C ABI.

The colouring is not unique; what is checked is that it is a proper
colouring of the oracle's assembled matrix graph (no nonzero couples two
DoFs of one colour) with 4 colours.  Given that colouring, one sweep
(colours 0..3 in turn) must equal the oracle's colour-ordered Gauss-Seidel
sweep, V-cycles with it must follow the oracle's, and GS-smoothed GMG must
converge in fewer steps than Jacobi."""
import numpy as np
import pytest

import synthgen as sg
from oracle import gmg as og

from helpers import rel_err

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

import paper_2308_01792_gb300 as hg

CASES = [(sg.reference_tet(), 2, 4), (sg.kuhn_cube(1), 1, 4), (sg.kuhn_cube(2), 1, 3)]
IDS = ["tet_L2-4", "cube1_L1-4", "cube2_L1-3"]


@pytest.fixture(scope="module", params=range(len(CASES)), ids=IDS)
def setup(request):
    macro, lmin, lmax = CASES[request.param]
    H = hg.Hierarchy(hg.Mesh(macro.xyz, macro.cells), lmin, lmax)
    Ho = og.Hierarchy(macro, lmin, lmax)
    return macro, H, Ho


def _sweep(op, H, L, x, b):
    t = torch.zeros_like(x)
    for c in range(4):
        src, dst = (x, t) if c % 2 == 0 else (t, x)
        op.gauss_seidel(L, src, b, dst, c)
    return x


def test_colouring_is_proper(setup):
    macro, H, Ho = setup
    for L in range(H.lmin, H.lmax + 1):
        col = H.gs_colours(L)
        A = Ho.levels[L].A_full.tocoo()
        off = A.row != A.col
        assert np.all(col[A.row[off]] != col[A.col[off]]), L
        assert set(np.unique(col)) <= {0, 1, 2, 3}
        if L >= 2:
            assert len(np.unique(col)) == 4


@pytest.mark.parametrize("dtype,tol", [(torch.float64, 1e-12), (torch.float32, 1e-5)])
def test_sweep_matches_oracle(setup, dtype, tol):
    macro, H, Ho = setup
    L = H.lmax
    lev = Ho.levels[L]
    op = hg.Operator(H)
    col = H.gs_colours(L)
    ii = lev.interior
    xc = np.zeros(lev.n)
    xc[ii] = sg.uniform_vector(41, len(ii))
    bc = np.zeros(lev.n)
    bc[ii] = sg.uniform_vector(42, len(ii))
    if dtype == torch.float32:
        xc, bc = xc.astype(np.float32).astype(np.float64), bc.astype(np.float32).astype(np.float64)
    x = H.from_canonical(L, torch.tensor(xc, dtype=dtype, device="cuda"))
    b = H.from_canonical(L, torch.tensor(bc, dtype=dtype, device="cuda"))
    _sweep(op, H, L, x, b)
    got = H.to_canonical(L, x).cpu().double().numpy()
    ref = og.gauss_seidel_colours(lev.A, lev.D, xc[ii], bc[ii], col[ii])
    assert rel_err(got[ii], ref) <= tol
    assert np.all(got[lev.boundary] == 0)


def test_divkgrad_sweep_matches_oracle():
    macro, L = sg.kuhn_cube(1), 3
    H = hg.Hierarchy(hg.Mesh(macro.xyz, macro.cells), L, L)
    _, xyz, _ = H.canonical_info(L)
    k = sg.rff_eval(sg.rff_params(5), xyz)
    op = hg.Operator(H, hg.HG_OP_P1_DIVKGRAD, coeff=k)
    lev = og.Level(macro, L, kind="divkgrad", coeff=lambda X: sg.rff_eval(sg.rff_params(5), X))
    col = H.gs_colours(L)
    ii = lev.interior
    xc = np.zeros(lev.n)
    xc[ii] = sg.uniform_vector(43, len(ii))
    bc = np.zeros(lev.n)
    bc[ii] = sg.uniform_vector(44, len(ii))
    x = H.from_canonical(L, torch.tensor(xc, device="cuda"))
    b = H.from_canonical(L, torch.tensor(bc, device="cuda"))
    _sweep(op, H, L, x, b)
    got = H.to_canonical(L, x).cpu().numpy()
    ref = og.gauss_seidel_colours(lev.A, lev.D, xc[ii], bc[ii], col[ii])
    assert rel_err(got[ii], ref) <= 1e-12


def test_gs_vcycles_match_oracle_and_beat_jacobi(setup):
    macro, H, Ho = setup
    L = H.lmax
    lev = Ho.levels[L]
    op = hg.Operator(H)
    cols = {len(Ho.levels[l].interior): H.gs_colours(l)[Ho.levels[l].interior]
            for l in range(H.lmin, H.lmax + 1)}

    def gs(A, D, x, b):
        return og.gauss_seidel_colours(A, D, x, b, cols[len(x)])

    G = hg.GMG(op, smoother=hg.HG_SMOOTH_GS)
    bc = np.zeros(lev.n)
    bc[lev.interior] = sg.uniform_vector(45, len(lev.interior))
    b = H.from_canonical(L, torch.tensor(bc, device="cuda"))
    x = H.zeros(L, torch.float64)
    xo = np.zeros(len(lev.interior))
    for cyc in range(2):
        G.vcycle(L, x, b)
        xo = og.vcycle(Ho, L, xo, bc[lev.interior], smoother=gs)
        got = H.to_canonical(L, x).cpu().numpy()
        assert rel_err(got[lev.interior], xo) <= 1e-12, cyc
    it_gs, rel_gs = G.solve(H.zeros(L, torch.float64), b, tol=1e-10, max_iter=60)
    it_j, rel_j = hg.GMG(op).solve(H.zeros(L, torch.float64), b, tol=1e-10, max_iter=60)
    assert rel_gs <= 1e-10 and rel_j <= 1e-10 and it_gs < it_j
    xs = H.zeros(L, torch.float64)
    G.solve(xs, b, tol=1e-10, max_iter=60, precision=hg.HG_PREC_MIXED)
    xg = H.to_canonical(L, xs).cpu().numpy()[lev.interior]
    bi = bc[lev.interior]
    assert np.linalg.norm(bi - lev.A @ xg) / np.linalg.norm(bi) <= 1.01e-10


def test_gs_rejected_for_p2():
    macro = sg.kuhn_cube(1)
    H = hg.Hierarchy(hg.Mesh(macro.xyz, macro.cells), 0, 3)
    op2 = hg.Operator(H, hg.HG_OP_P2_LAPLACE)
    x = H.zeros(2, torch.float64, space=hg.HG_SPACE_P2)
    with pytest.raises(hg.HGError) as e:
        op2.gauss_seidel(2, x, x.clone(), torch.zeros_like(x), 0)
    assert e.value.code == -7
    with pytest.raises(hg.HGError):
        hg.GMG(op2, smoother=hg.HG_SMOOTH_GS)
