"""GPU parity of the polynomial surrogate operator (Sec. 5.2, surrogate
operators) against the oracle's surrogate matrix (oracle.surrogate), through
the C ABI.

The oracle fits the exact weights by numpy.linalg.lstsq in the monomials of
(i/n, j/n, k/n); the library by a QR factorisation in shifted monomials.  Both
are the same least-squares projection, so the fitted weights agree up to
rounding amplified by the conditioning of the basis (below 1e4 for these
degrees on the interior lattice): the FP64 apply is held to 1e-11 relative
(max norm), the FP32 apply to 1e-5.  Independent of the oracle: a degree-1
surrogate of a coefficient linear in x is the exact operator."""
import numpy as np
import pytest

import synthgen as sg
from oracle import surrogate as su

from helpers import rel_err

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

import paper_2308_01792_gb300 as hg

SUR = hg.HG_OP_P1_DIVKGRAD_SURROGATE
CASES = [(sg.kuhn_cube(1), 1, 4), (sg.permuted_cells(sg.kuhn_cube(1), 3), 1, 4),
         (sg.kuhn_cube(2), 1, 3), (sg.reference_tet(), 2, 5)]
IDS = ["cube1_L1-4", "cube1perm_L1-4", "cube2_L1-3", "tet_L2-5"]
KFUN = sg.sinprod_coefficient(*sg.SINPROD_AB)


@pytest.fixture(scope="module", params=range(len(CASES)), ids=IDS)
def case(request):
    macro, lmin, lmax = CASES[request.param]
    H = hg.Hierarchy(hg.Mesh(macro.xyz, macro.cells), lmin, lmax)
    _, xyz, _ = H.canonical_info(lmax)
    return macro, H, KFUN(xyz)


@pytest.mark.parametrize("degree", [0, 1, 2, 3, 4])
@pytest.mark.parametrize("dtype", [torch.float64, torch.float32])
def test_surrogate_apply_matches_oracle(case, degree, dtype):
    macro, H, k = case
    op = hg.Operator(H, SUR, coeff=k, degree=degree)
    for L in range(max(H.lmin, 2), H.lmax + 1):
        S = su.SurrogateLevel(macro, L, KFUN)
        A = S.surrogate(degree)
        nu = S.rm.n_vertices
        xc = sg.uniform_vector(50 + L, nu)
        x = H.from_canonical(L, torch.tensor(xc, dtype=dtype, device="cuda"))
        y = H.zeros(L, dtype)
        op.apply(L, x, y, mask=hg.HG_MASK_ALL)
        got = H.to_canonical(L, y).cpu().double().numpy()
        ref = A @ xc.astype(np.float32 if dtype == torch.float32 else np.float64).astype(np.float64)
        tol = 1e-11 if dtype == torch.float64 else 1e-5
        assert rel_err(got, ref) <= tol, (L, degree, rel_err(got, ref))
        # Dirichlet rows: interior rows as given x, boundary rows 0
        y.fill_(3.0)
        op.apply(L, x, y)
        got = H.to_canonical(L, y).cpu().double().numpy()
        ii, bd = S.rm.interior, S.rm.boundary
        if len(ii):
            assert rel_err(got[ii], ref[ii]) <= tol, (L, degree)
        assert np.all(got[bd] == 0.0)


def test_degree1_reproduces_a_linear_coefficient():
    """k linear in x makes every stencil weight affine in the position: the
    degree-1 surrogate is then the exact operator (element-wise apply)."""
    macro = sg.permuted_cells(sg.kuhn_cube(2), 7)
    H = hg.Hierarchy(hg.Mesh(macro.xyz, macro.cells), 1, 4)
    _, xyz, _ = H.canonical_info(4)
    k = 1.0 + xyz @ np.array([1.0, 2.0, 3.0])
    sur = hg.Operator(H, SUR, coeff=k, degree=1)
    ex = hg.Operator(H, hg.HG_OP_P1_DIVKGRAD, coeff=k)
    for L in range(1, 5):
        nu = H.size(L)[1]
        x = H.from_canonical(L, torch.tensor(sg.uniform_vector(7, nu), device="cuda"))
        ys, ye = H.zeros(L, torch.float64), H.zeros(L, torch.float64)
        sur.apply(L, x, ys, mask=hg.HG_MASK_ALL)
        ex.apply(L, x, ye, mask=hg.HG_MASK_ALL)
        assert rel_err(H.to_canonical(L, ys).cpu().numpy(),
                       H.to_canonical(L, ye).cpu().numpy()) <= 1e-12, L


@pytest.mark.parametrize("dtype", [torch.float64, torch.float32])
def test_surrogate_jacobi_uses_its_own_diagonal(case, dtype):
    macro, H, k = case
    op = hg.Operator(H, SUR, coeff=k, degree=2)
    L = H.lmax
    S = su.SurrogateLevel(macro, L, KFUN)
    A = S.surrogate(2)
    ii = S.rm.interior
    if not len(ii):
        pytest.skip("no interior DoFs")
    nu = S.rm.n_vertices
    xc = sg.uniform_vector(60, nu)
    bc = sg.uniform_vector(61, nu)
    xc[S.rm.boundary] = 0.0
    bc[S.rm.boundary] = 0.0
    npd = np.float32 if dtype == torch.float32 else np.float64
    xc, bc = xc.astype(npd).astype(np.float64), bc.astype(npd).astype(np.float64)
    x = H.from_canonical(L, torch.tensor(xc, dtype=dtype, device="cuda"))
    b = H.from_canonical(L, torch.tensor(bc, dtype=dtype, device="cuda"))
    xo = H.zeros(L, dtype)
    op.jacobi(L, x, b, xo, omega=2.0 / 3.0)
    got = H.to_canonical(L, xo).cpu().double().numpy()
    D = A.diagonal()
    ref = xc + (2.0 / 3.0) * (bc - A @ xc) / D
    tol = 1e-11 if dtype == torch.float64 else 1e-5
    assert rel_err(got[ii], ref[ii]) <= tol


@pytest.mark.parametrize("precision", [hg.HG_PREC_F64, hg.HG_PREC_MIXED])
def test_surrogate_gmg_solves_the_surrogate_system(precision):
    """GMG on the surrogate operator reaches 1e-10; the oracle's surrogate
    matrix measures the residual of the GPU solution in FP64."""
    macro = sg.kuhn_cube(1)
    H = hg.Hierarchy(hg.Mesh(macro.xyz, macro.cells), 1, 4)
    _, xyz, dirich = H.canonical_info(4)
    op = hg.Operator(H, SUR, coeff=KFUN(xyz), degree=3)
    G = hg.GMG(op)
    bc = sg.uniform_vector(9, len(xyz))
    bc[dirich] = 0.0
    b = H.from_canonical(4, torch.tensor(bc, device="cuda"))
    x = H.zeros(4, torch.float64)
    it, rel = G.solve(x, b, tol=1e-10, max_iter=60, precision=precision)
    assert rel <= 1e-10
    S = su.SurrogateLevel(macro, 4, KFUN)
    A = S.surrogate(3)
    ii = S.rm.interior
    xg = H.to_canonical(4, x).cpu().numpy()
    r = bc[ii] - (A @ xg)[ii]
    assert np.linalg.norm(r) <= 1.01e-10 * np.linalg.norm(bc[ii])


def test_surrogate_rejects_bad_degree():
    macro = sg.kuhn_cube(1)
    H = hg.Hierarchy(hg.Mesh(macro.xyz, macro.cells), 1, 2)
    k = np.ones(H.size(2)[1])
    for q in (-1, 5):
        with pytest.raises(hg.HGError):
            hg.Operator(H, SUR, coeff=k, degree=q)
