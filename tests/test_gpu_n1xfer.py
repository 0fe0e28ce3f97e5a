"""Nedelec transfers and discrete gradient through the C ABI against the
oracle (oracle.nedelec): prolongation P (tangential line integrals of the
coarse function), restriction P^T, the discrete gradient G and G^T, on meshes
with Kuhn-ordered and permuted cells (other local orientations) and on the
48-cell cube (interior macro vertices and edges).  Bars: FP64
1e-13, FP32 1e-6 relative; boundary entries as documented."""
import numpy as np
import pytest

import synthgen as sg
from oracle import fem
from oracle import nedelec as ne

from helpers import rel_err

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

import paper_2308_01792_gb300 as hg

P2 = hg.HG_SPACE_P2
TOL = {torch.float64: 1e-13, torch.float32: 1e-6}
CASES = [sg.kuhn_cube(1), sg.permuted_cells(sg.kuhn_cube(1), 3), sg.reference_tet(), sg.kuhn_cube(2)]
IDS = ["cube1", "cube1perm", "tet", "cube2"]
L = 2


@pytest.fixture(scope="module", params=range(len(CASES)), ids=IDS)
def case(request):
    macro = CASES[request.param]
    H = hg.Hierarchy(hg.Mesh(macro.xyz, macro.cells), 0, L + 1)
    op = hg.Operator(H, hg.HG_OP_N1_CURLCURL, coeff=(1.0, 0.5))
    fine, coarse = ne.NedelecLevel(macro, L), ne.NedelecLevel(macro, L - 1)
    ef = np.flatnonzero(np.any(fem.P2Numbering(fine.rm).coords2 % 2 == 1, axis=1))
    ec = np.flatnonzero(np.any(fem.P2Numbering(coarse.rm).coords2 % 2 == 1, axis=1))
    nf = fem.P2Numbering(fine.rm).n
    nc = fem.P2Numbering(coarse.rm).n
    return macro, H, op, fine, coarse, (ef, nf), (ec, nc)


def _n1_stored(H, level, sub, vals, dtype):
    idx, n = sub
    full = np.zeros(n)
    full[idx] = vals
    return H.from_canonical(level, torch.tensor(full, dtype=dtype, device="cuda"), space=P2)


def _n1_canon(H, level, sub, y):
    return H.to_canonical(level, y, space=P2).cpu().double().numpy()[sub[0]]


def _interior_vec(lev, seed, dtype):
    v = np.zeros(lev.n)
    v[lev.interior] = sg.uniform_vector(seed, len(lev.interior))
    if dtype == torch.float32:
        v = v.astype(np.float32).astype(np.float64)
    return v


@pytest.mark.parametrize("dtype", [torch.float64, torch.float32])
def test_n1_prolongation_matches_oracle(case, dtype):
    macro, H, op, fine, coarse, fsub, csub = case
    uc = _interior_vec(coarse, 40, dtype)
    ecv = _n1_stored(H, L - 1, csub, uc, dtype)
    xf = H.zeros(L, dtype, space=P2)
    op.n1_prolong_add(L, ecv, xf)
    got = _n1_canon(H, L, fsub, xf)
    ref = ne.nedelec_prolongation(fine, coarse) @ uc
    assert rel_err(got, ref) <= TOL[dtype]


@pytest.mark.parametrize("dtype", [torch.float64, torch.float32])
def test_n1_restriction_is_the_transpose(case, dtype):
    macro, H, op, fine, coarse, fsub, csub = case
    rf = _interior_vec(fine, 41, dtype)
    rc = H.zeros(L - 1, dtype, space=P2)
    op.n1_restrict(L, _n1_stored(H, L, fsub, rf, dtype), rc)
    got = _n1_canon(H, L - 1, csub, rc)
    ref = ne.nedelec_prolongation(fine, coarse).T @ rf
    ii = coarse.interior
    assert rel_err(got[ii], ref[ii]) <= TOL[dtype]
    assert np.all(got[coarse.boundary] == 0)


@pytest.mark.parametrize("dtype", [torch.float64, torch.float32])
def test_n1_gradient_and_transpose_match_oracle(case, dtype):
    macro, H, op, fine, coarse, fsub, csub = case
    rm = fine.rm
    phi = np.zeros(rm.n_vertices)
    phi[rm.interior] = sg.uniform_vector(42, len(rm.interior))
    if dtype == torch.float32:
        phi = phi.astype(np.float32).astype(np.float64)
    u = H.zeros(L, dtype, space=P2)
    op.n1_gradient(L, H.from_canonical(L, torch.tensor(phi, dtype=dtype, device="cuda")), u)
    got = _n1_canon(H, L, fsub, u)
    assert rel_err(got, fine.G_full @ phi) <= TOL[dtype]
    r = _interior_vec(fine, 43, dtype)
    rp = H.zeros(L, dtype)
    op.n1_gradient_t(L, _n1_stored(H, L, fsub, r, dtype), rp)
    gp = H.to_canonical(L, rp).cpu().double().numpy()
    ref = fine.G_full.T @ r
    assert rel_err(gp[rm.interior], ref[rm.interior]) <= TOL[dtype]
    assert np.all(gp[rm.boundary] == 0)


def test_n1_transfers_reject_other_operators():
    macro = sg.kuhn_cube(1)
    H = hg.Hierarchy(hg.Mesh(macro.xyz, macro.cells), 0, 3)
    op = hg.Operator(H, hg.HG_OP_P2_LAPLACE)
    x = H.zeros(2, torch.float64, space=P2)
    with pytest.raises(hg.HGError):
        op.n1_prolong_add(2, H.zeros(1, torch.float64, space=P2), x)
