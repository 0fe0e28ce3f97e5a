"""Nedelec multigrid with Hiptmair's hybrid smoother through the C ABI
against the oracle (oracle.nedelec): V(1,1) iterates with weighted Jacobi
(omega = 1/2) or order-2 Chebyshev smoothing (the paper's choice, Sec. 6)
in the edge and the potential space, FMG, and solves to 1e-8 in FP64 and
mixed precision, on a Kuhn cube, a permuted-cell cube and the 48-cell cube
(2 x 2 x 2 sub-cubes).  For the Chebyshev iterates the GPU takes the
oracle's lambda_max estimates of both spaces, so the same polynomials act."""
import numpy as np
import pytest

import synthgen as sg
from oracle import fem
from oracle import gmg as og
from oracle import nedelec as ne

from helpers import rel_err

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

import paper_2308_01792_gb300 as hg

P2 = hg.HG_SPACE_P2
AB = (1.0, 0.3)
L = 3
CASES = [sg.kuhn_cube(1), sg.permuted_cells(sg.kuhn_cube(1), 3), sg.kuhn_cube(2)]
IDS = ["cube1", "cube1perm", "cube2"]


@pytest.fixture(scope="module", params=range(len(CASES)), ids=IDS)
def case(request):
    macro = CASES[request.param]
    H = hg.Hierarchy(hg.Mesh(macro.xyz, macro.cells), 0, L + 1)
    op = hg.Operator(H, hg.HG_OP_N1_CURLCURL, coeff=AB)
    Ho = ne.NedelecHierarchy(macro, 1, L, *AB)
    lev = Ho.levels[L]
    num = fem.P2Numbering(lev.rm)
    edge = np.flatnonzero(np.any(num.coords2 % 2 == 1, axis=1))
    return macro, H, op, Ho, lev, num.n, edge


def _stored(H, n, edge, lev, vals_interior, dtype=torch.float64):
    full = np.zeros(n)
    e = np.zeros(lev.n)
    e[lev.interior] = vals_interior
    full[edge] = e
    return H.from_canonical(L, torch.tensor(full, dtype=dtype, device="cuda"), space=P2)


def _interior(H, edge, lev, x):
    got = H.to_canonical(L, x, space=P2).cpu().double().numpy()[edge]
    assert np.all(got[lev.boundary] == 0)
    return got[lev.interior]


def test_hiptmair_vcycles_match_oracle(case):
    macro, H, op, Ho, lev, n, edge = case
    G = hg.GMG(op, nu1=1, nu2=1, omega=0.5, lmin=1)
    b = sg.uniform_vector(60, len(lev.interior))
    bs = _stored(H, n, edge, lev, b)
    x = H.zeros(L, torch.float64, space=P2)
    xo = np.zeros_like(b)
    for cyc in range(2):
        G.vcycle(L, x, bs)
        xo = ne.vcycle(Ho, L, xo, b, 1, 1)
        assert rel_err(_interior(H, edge, lev, x), xo) <= 1e-11, cyc


def test_hiptmair_fmg_matches_oracle(case):
    macro, H, op, Ho, lev, n, edge = case
    G = hg.GMG(op, nu1=1, nu2=1, omega=0.5, lmin=1)
    b = sg.uniform_vector(61, len(lev.interior))
    x = H.zeros(L, torch.float64, space=P2)
    G.fmg(L, x, _stored(H, n, edge, lev, b), cycles=3)
    xo = ne.fmg(Ho, b, cycles=3)
    assert rel_err(_interior(H, edge, lev, x), xo) <= 1e-11


@pytest.mark.parametrize("precision", [hg.HG_PREC_F64, hg.HG_PREC_MIXED])
def test_hiptmair_solve_converges(case, precision):
    macro, H, op, Ho, lev, n, edge = case
    G = hg.GMG(op, nu1=2, nu2=2, omega=0.5, lmin=1)
    b = sg.uniform_vector(62, len(lev.interior))
    x = H.zeros(L, torch.float64, space=P2)
    it, rel = G.solve(x, _stored(H, n, edge, lev, b), tol=1e-8, max_iter=200, precision=precision)
    xi = _interior(H, edge, lev, x)
    assert rel <= 1e-8 and np.linalg.norm(b - lev.A @ xi) <= 1.01e-8 * np.linalg.norm(b)
    assert it <= 120


def _cheb_setup(G, Ho):
    """The oracle's lambda_max of both spaces on every smoothed level, given to
    the GPU; returns the oracle's two smoothers."""
    lam = {}
    for l in range(Ho.lmin + 1, Ho.lmax + 1):
        lev = Ho.levels[l]
        le = og.power_lambda_max(lev.A, lev.D, sg.uniform_vector(3, len(lev.D)))
        lp = og.power_lambda_max(lev.Ap, lev.Dp, sg.uniform_vector(4, len(lev.Dp)))
        lam["e", len(lev.D)], lam["p", len(lev.Dp)] = le, lp
        G.set_lam(l, le)
        G.set_lam_potential(l, lp)
    es = lambda A, D, x, b: og.chebyshev(A, D, x, b, lam["e", len(x)])  # noqa: E731
    ps = lambda A, D, x, b: og.chebyshev(A, D, x, b, lam["p", len(x)])  # noqa: E731
    return es, ps


def test_hiptmair_chebyshev_vcycles_match_oracle(case):
    macro, H, op, Ho, lev, n, edge = case
    G = hg.GMG(op, nu1=1, nu2=1, lmin=1, smoother=hg.HG_SMOOTH_CHEB)
    es, ps = _cheb_setup(G, Ho)
    b = sg.uniform_vector(63, len(lev.interior))
    bs = _stored(H, n, edge, lev, b)
    x = H.zeros(L, torch.float64, space=P2)
    xo = np.zeros_like(b)
    for cyc in range(2):
        G.vcycle(L, x, bs)
        xo = ne.vcycle(Ho, L, xo, b, 1, 1, edge_smoother=es, potential_smoother=ps)
        assert rel_err(_interior(H, edge, lev, x), xo) <= 1e-11, cyc


def test_hiptmair_chebyshev_fmg_matches_oracle(case):
    macro, H, op, Ho, lev, n, edge = case
    G = hg.GMG(op, nu1=1, nu2=1, lmin=1, smoother=hg.HG_SMOOTH_CHEB)
    es, ps = _cheb_setup(G, Ho)
    b = sg.uniform_vector(64, len(lev.interior))
    x = H.zeros(L, torch.float64, space=P2)
    G.fmg(L, x, _stored(H, n, edge, lev, b), cycles=3)
    xo = ne.fmg(Ho, b, cycles=3, edge_smoother=es, potential_smoother=ps)
    assert rel_err(_interior(H, edge, lev, x), xo) <= 1e-11


@pytest.mark.parametrize("precision", [hg.HG_PREC_F64, hg.HG_PREC_MIXED])
def test_hiptmair_chebyshev_solve_converges_faster_than_jacobi(case, precision):
    """With its own lambda estimates, Chebyshev V(1,1) reaches 1e-8 in fewer
    cycles than Jacobi V(1,1) (the oracle pins the same ordering of rates)."""
    macro, H, op, Ho, lev, n, edge = case
    b = sg.uniform_vector(65, len(lev.interior))
    its = {}
    for sm in (hg.HG_SMOOTH_JACOBI, hg.HG_SMOOTH_CHEB):
        G = hg.GMG(op, nu1=1, nu2=1, omega=0.5, lmin=1, smoother=sm)
        x = H.zeros(L, torch.float64, space=P2)
        it, rel = G.solve(x, _stored(H, n, edge, lev, b), tol=1e-8, max_iter=200,
                          precision=precision)
        xi = _interior(H, edge, lev, x)
        assert rel <= 1e-8 and np.linalg.norm(b - lev.A @ xi) <= 1.01e-8 * np.linalg.norm(b)
        its[sm] = it
    assert its[hg.HG_SMOOTH_CHEB] < its[hg.HG_SMOOTH_JACOBI], its


def test_hiptmair_default_lambdas_near_the_dense_eigenvalues():
    macro = sg.kuhn_cube(1)
    H = hg.Hierarchy(hg.Mesh(macro.xyz, macro.cells), 0, 3)
    op = hg.Operator(H, hg.HG_OP_N1_CURLCURL, coeff=AB)
    G = hg.GMG(op, lmin=1, smoother=hg.HG_SMOOTH_CHEB)
    Ho = ne.NedelecHierarchy(macro, 1, 2, *AB)
    lev = Ho.levels[2]
    le = np.max(np.linalg.eigvals(lev.A.toarray() / lev.D[:, None]).real)
    lp = np.max(np.linalg.eigvals(lev.Ap.toarray() / lev.Dp[:, None]).real)
    assert 0.85 * le <= G.lam(2) <= 1.05 * le, (G.lam(2), le)
    assert 0.85 * lp <= G.lam_potential(2) <= 1.05 * lp, (G.lam_potential(2), lp)


def test_n1_gmg_rejects_gauss_seidel():
    macro = sg.kuhn_cube(1)
    H = hg.Hierarchy(hg.Mesh(macro.xyz, macro.cells), 0, 3)
    op = hg.Operator(H, hg.HG_OP_N1_CURLCURL, coeff=AB)
    with pytest.raises(hg.HGError) as e:
        hg.GMG(op, smoother=hg.HG_SMOOTH_GS)
    assert e.value.code == -7
