"""GPU parity of the variable-coefficient P1 operator -div(k grad) (element-wise,
k_T = mean of the vertex values) and of multigrid built on it, against the
oracle's assembled matrices (through the C ABI).  Every test runs for the
on-the-fly form and for the stored-stencil form (grid-aware precomputation:
the partial stencil of every stored point kept in HBM)."""
import numpy as np
import pytest

import synthgen as sg
from oracle import fem
from oracle import gmg as og
from oracle.mesh import RefinedMesh

from helpers import rel_err

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

import paper_2308_01792_gb300 as hg

TOL = {torch.float64: 1e-12, torch.float32: 1e-5}


def kfun_smooth(xyz):
    return np.exp(np.sin(2.0 * xyz[:, 0] + xyz[:, 1]) * np.cos(3.0 * xyz[:, 2]))


def kfun_lognormal(xyz, _p=sg.rff_params(1000)):
    return sg.rff_eval(_p, xyz)


CASES = [(sg.reference_tet(), 2, 4, kfun_smooth), (sg.kuhn_cube(2), 1, 4, kfun_lognormal),
         (sg.kuhn_cube(1), 1, 5, kfun_smooth)]
IDS = ["tet_smooth", "cube2_lognormal", "cube1_smooth"]


KINDS = [hg.HG_OP_P1_DIVKGRAD, hg.HG_OP_P1_DIVKGRAD_STORED]


@pytest.fixture(scope="module", params=[(c, k) for c in range(len(CASES)) for k in KINDS],
                ids=[f"{i}-{k}" for i in IDS for k in ("onthefly", "stored")])
def case(request):
    c, kind = request.param
    macro, lmin, lmax, kf = CASES[c]
    H = hg.Hierarchy(hg.Mesh(macro.xyz, macro.cells), lmin, lmax)
    _, xyz, _ = H.canonical_info(lmax)
    op = hg.Operator(H, kind, coeff=kf(xyz))
    return macro, H, op, kf


@pytest.mark.parametrize("dtype", [torch.float64, torch.float32])
def test_divkgrad_apply_matches_assembled(case, dtype):
    macro, H, op, kf = case
    for L in range(H.lmin, H.lmax + 1):
        rm = RefinedMesh(macro, L)
        kv = kf(rm.xyz)[rm.cells]
        A = fem.assemble(rm.cells, fem.p1_divkgrad(rm.cell_xyz, kv), rm.n_vertices)
        xc = sg.uniform_vector(30 + L, rm.n_vertices)
        x = H.from_canonical(L, torch.tensor(xc, dtype=dtype, device="cuda"))
        y = H.zeros(L, dtype)
        op.apply(L, x, y, mask=hg.HG_MASK_ALL)
        got = H.to_canonical(L, y).cpu().double().numpy()
        assert rel_err(got, A @ xc) <= TOL[dtype] * 4, L
        xi = xc.copy()
        xi[rm.boundary] = 0
        x = H.from_canonical(L, torch.tensor(xi, dtype=dtype, device="cuda"))
        y = H.zeros(L, dtype)
        op.apply(L, x, y)
        got = H.to_canonical(L, y).cpu().double().numpy()
        ii = rm.interior
        if len(ii):
            assert rel_err(got[ii], (A @ xi)[ii]) <= TOL[dtype] * 4
        assert np.all(got[rm.boundary] == 0)
        # INNER on a nonzero destination, both modes: Dirichlet entries 0
        y0 = sg.uniform_vector(60 + L, rm.n_vertices)
        y0r = torch.tensor(y0, dtype=dtype).double().numpy()
        for mode, base in ((hg.HG_REPLACE, 0.0), (hg.HG_ADD, y0r)):
            y = H.from_canonical(L, torch.tensor(y0, dtype=dtype, device="cuda"))
            op.apply(L, x, y, mode=mode)
            got = H.to_canonical(L, y).cpu().double().numpy()
            if len(ii):
                assert rel_err(got[ii], (base + A @ xi)[ii]) <= TOL[dtype] * 4
            assert np.all(got[rm.boundary] == 0)


@pytest.mark.parametrize("dtype", [torch.float64, torch.float32])
def test_divkgrad_jacobi_uses_exact_diagonal(case, dtype):
    macro, H, op, kf = case
    L = H.lmax
    Ho = og.Hierarchy(macro, L, L, kind="divkgrad", coeff=kf)
    lev = Ho.levels[L]
    xc = sg.uniform_vector(40, lev.n)
    bc = sg.uniform_vector(41, lev.n)
    xc[lev.boundary] = 0
    bc[lev.boundary] = 0
    x = H.from_canonical(L, torch.tensor(xc, dtype=dtype, device="cuda"))
    b = H.from_canonical(L, torch.tensor(bc, dtype=dtype, device="cuda"))
    xo = H.zeros(L, dtype)
    op.jacobi(L, x, b, xo, omega=0.7)
    got = H.to_canonical(L, xo).cpu().double().numpy()
    ref = og.jacobi(lev.A, lev.D, xc[lev.interior], bc[lev.interior], 0.7)
    assert rel_err(got[lev.interior], ref) <= TOL[dtype] * 8
    r = H.zeros(L, dtype)
    op.residual(L, x, b, r)
    got = H.to_canonical(L, r).cpu().double().numpy()
    assert rel_err(got[lev.interior], bc[lev.interior] - lev.A @ xc[lev.interior]) <= TOL[dtype] * 8


@pytest.mark.parametrize("precision", [hg.HG_PREC_F64, hg.HG_PREC_MIXED])
def test_divkgrad_gmg_matches_oracle(case, precision):
    macro, H, op, kf = case
    L = H.lmax
    Ho = og.Hierarchy(macro, H.lmin, L, kind="divkgrad", coeff=kf)
    lev = Ho.levels[L]
    G = hg.GMG(op)
    bc = np.zeros(lev.n)
    bc[lev.interior] = sg.uniform_vector(42, len(lev.interior))
    b = H.from_canonical(L, torch.tensor(bc, device="cuda"))
    x = H.zeros(L, torch.float64)
    if precision == hg.HG_PREC_F64:
        G.vcycle(L, x, b)
        xo = og.vcycle(Ho, L, np.zeros(len(lev.interior)), bc[lev.interior])
        got = H.to_canonical(L, x).cpu().numpy()
        assert rel_err(got[lev.interior], xo) <= 1e-11
    it, rel = G.solve(x, b, tol=1e-8, max_iter=80, precision=precision)
    xg = H.to_canonical(L, x).cpu().numpy()[lev.interior]
    ro = np.linalg.norm(bc[lev.interior] - lev.A @ xg) / np.linalg.norm(bc[lev.interior])
    assert rel <= 1e-8 and ro <= 1.01e-8
    _, ito, _ = og.solve(Ho, bc[lev.interior], tol=1e-8)
    assert abs(it - ito) <= (1 if precision == hg.HG_PREC_F64 else 3)


def test_divkgrad_rejects_coefficients_that_are_not_positive_and_finite():
    """-div(k grad) is elliptic only for k > 0: a zero, negative, NaN or
    infinite vertex value is refused at creation (both forms), and so is a
    coefficient array of the wrong length; a positive constant is accepted."""
    macro = sg.kuhn_cube(1)
    H = hg.Hierarchy(hg.Mesh(macro.xyz, macro.cells), 1, 3)
    n = H.size(3)[1]
    for kind in (hg.HG_OP_P1_DIVKGRAD, hg.HG_OP_P1_DIVKGRAD_STORED):
        for bad in (0.0, -1.0, np.nan, np.inf):
            k = np.ones(n)
            k[n // 2] = bad
            with pytest.raises(hg.HGError) as e:
                hg.Operator(H, kind, coeff=k)
            assert e.value.code == -1 and "positive and finite" in str(e.value)
        with pytest.raises(ValueError):
            hg.Operator(H, kind, coeff=np.ones(n - 1))
        hg.Operator(H, kind, coeff=np.full(n, 2.0))
