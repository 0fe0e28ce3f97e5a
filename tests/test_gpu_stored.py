"""Stored-stencil form of P1 -div(k grad) (grid-aware precomputation, Sec. 5.2:
the operator's stencil entries laid out in the order of the iteration pattern
instead of a sparse format) through the C ABI.

The general parity (apply, Jacobi, residual, V-cycles and solves against the
oracle's assembled matrices) runs in test_gpu_divkgrad.py for both forms.
Here: the stored form equals the on-the-fly form to rounding on every level
(FP64 1e-13, FP32 1e-6) and keeps interface copies bit-identical; constants
are in the kernel of the operator (ALL mask, row sums zero); Chebyshev
V-cycles, Gauss-Seidel sweeps and FMG through the stored form match the
oracle."""
import numpy as np
import pytest

import synthgen as sg
from oracle import gmg as og

from helpers import rel_err

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

import paper_2308_01792_gb300 as hg


def _kf(xyz, _p=sg.rff_params(1000)):
    return sg.rff_eval(_p, xyz)


CASES = [(sg.kuhn_cube(2), 1, 4), (sg.reference_tet(), 2, 5)]


@pytest.fixture(scope="module", params=range(len(CASES)), ids=["cube2_L1-4", "tet_L2-5"])
def pair(request):
    macro, lmin, lmax = CASES[request.param]
    H = hg.Hierarchy(hg.Mesh(macro.xyz, macro.cells), lmin, lmax)
    _, xyz, _ = H.canonical_info(lmax)
    k = _kf(xyz)
    fly = hg.Operator(H, hg.HG_OP_P1_DIVKGRAD, coeff=k)
    st = hg.Operator(H, hg.HG_OP_P1_DIVKGRAD_STORED, coeff=k)
    return macro, H, fly, st


@pytest.mark.parametrize("dtype,tol", [(torch.float64, 1e-13), (torch.float32, 1e-6)])
def test_stored_equals_on_the_fly(pair, dtype, tol):
    macro, H, fly, st = pair
    for L in range(H.lmin, H.lmax + 1):
        s2c, _, _ = H.canonical_info(L)
        nu = H.size(L)[1]
        x = H.from_canonical(L, torch.tensor(sg.uniform_vector(90 + L, nu), dtype=dtype,
                                             device="cuda"))
        for mask in (hg.HG_MASK_ALL, hg.HG_MASK_INNER):
            y1, y2 = H.zeros(L, dtype), H.zeros(L, dtype)
            fly.apply(L, x, y1, mask=mask)
            st.apply(L, x, y2, mask=mask)
            a = H.to_canonical(L, y1).cpu().double().numpy()
            b = H.to_canonical(L, y2).cpu().double().numpy()
            assert rel_err(b, a) <= tol, (L, mask)
        ys = y2.cpu().numpy()
        m = s2c >= 0
        assert np.array_equal(ys[m], H.to_canonical(L, y2).cpu().numpy()[s2c[m]])


def test_constants_in_the_kernel(pair):
    macro, H, fly, st = pair
    L = H.lmax
    x = torch.ones(H.size(L)[0], dtype=torch.float64, device="cuda")
    y = H.zeros(L, torch.float64)
    st.apply(L, x, y, mask=hg.HG_MASK_ALL)
    yref = H.zeros(L, torch.float64)
    fly.apply(L, torch.tensor(sg.uniform_vector(3, H.size(L)[0]), device="cuda").abs(), yref,
              mask=hg.HG_MASK_ALL)
    assert torch.abs(y).max().item() <= 1e-12 * torch.abs(yref).max().item()


def test_stored_chebyshev_gs_and_fmg_match_oracle(pair):
    macro, H, fly, st = pair
    L = H.lmax
    Ho = og.Hierarchy(macro, H.lmin, L, kind="divkgrad", coeff=_kf)
    lev = Ho.levels[L]
    lam = {l: og.power_lambda_max(Ho.levels[l].A, Ho.levels[l].D,
                                  sg.uniform_vector(95 + l, len(Ho.levels[l].interior)))
           for l in range(H.lmin + 1, L + 1)}
    lam_by_n = {len(Ho.levels[l].interior): v for l, v in lam.items()}

    def cheb(A, D, x, b):
        return og.chebyshev(A, D, x, b, lam_by_n[len(x)])

    G = hg.GMG(st, nu1=1, nu2=1, smoother=hg.HG_SMOOTH_CHEB)
    for l, v in lam.items():
        G.set_lam(l, v)
    bc = np.zeros(lev.n)
    bc[lev.interior] = sg.uniform_vector(96, len(lev.interior))
    b = H.from_canonical(L, torch.tensor(bc, device="cuda"))
    x = H.zeros(L, torch.float64)
    xo = np.zeros(len(lev.interior))
    for cyc in range(2):
        G.vcycle(L, x, b)
        xo = og.vcycle(Ho, L, xo, bc[lev.interior], 1, 1, smoother=cheb)
        got = H.to_canonical(L, x).cpu().numpy()
        assert rel_err(got[lev.interior], xo) <= 1e-11, cyc
    xf = H.zeros(L, torch.float64)
    G.fmg(L, xf, b, cycles=5)
    xo = og.fmg(Ho, bc[lev.interior], cycles=5, smoother=cheb)
    assert rel_err(H.to_canonical(L, xf).cpu().numpy()[lev.interior], xo) <= 1e-11
    # one 4-colour Gauss-Seidel sweep
    col = H.gs_colours(L)
    xc = np.zeros(lev.n)
    xc[lev.interior] = sg.uniform_vector(97, len(lev.interior))
    xg = H.from_canonical(L, torch.tensor(xc, device="cuda"))
    t = torch.zeros_like(xg)
    for c in range(4):
        src, dst = (xg, t) if c % 2 == 0 else (t, xg)
        st.gauss_seidel(L, src, b, dst, c)
    got = H.to_canonical(L, xg).cpu().numpy()
    ref = og.gauss_seidel_colours(lev.A, lev.D, xc[lev.interior], bc[lev.interior],
                                  col[lev.interior])
    assert rel_err(got[lev.interior], ref) <= 1e-12
