"""Chebyshev-accelerated Jacobi smoothing and full multigrid through the C ABI.

The paper's solver (Sec. 6) is full multigrid with five V(1,1) cycles per
level and Chebyshev smoothers of order 2.  Checked against the oracle:
- the power-iteration estimate of lambda_max(D^-1 A) from the same start
  vector (1e-12 relative, FP64);
- V-cycle iterates with Chebyshev smoothing, the GPU given the oracle's
  lambda per level (FP64 1e-12, FP32 1e-5);
- FMG results (FP64 1e-11), for the P1 Laplacian on three meshes, the P1
  -div(k grad) operator and the P2 operator;
plus properties: the default estimate (fixed SplitMix64 start vector) lies
within a few percent of the dense largest eigenvalue, Chebyshev-smoothed
solves converge in FP64 and mixed precision, FMG on a manufactured problem
ends with an algebraic error far below the discretization error, and bad
parameters are rejected."""
import numpy as np
import pytest
import scipy.sparse as sp

import synthgen as sg
from oracle import gmg as og

from helpers import rel_err

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

import paper_2308_01792_gb300 as hg

P2 = hg.HG_SPACE_P2


def _kf(xyz, _p=sg.rff_params(5)):
    return sg.rff_eval(_p, xyz)


# (id, macro, lmin, lmax, kind)
CASES = [("tet_L2-4", sg.reference_tet(), 2, 4, "laplace"),
         ("cube1_L1-4", sg.kuhn_cube(1), 1, 4, "laplace"),
         ("cube2_L1-3", sg.kuhn_cube(2), 1, 3, "laplace"),
         ("cube1_divkgrad_L1-4", sg.kuhn_cube(1), 1, 4, "divkgrad"),
         ("cube1_P2_L0-3", sg.kuhn_cube(1), 0, 3, "p2"),
         ("tet_P2_L0-3", sg.reference_tet(), 0, 3, "p2")]


@pytest.fixture(scope="module", params=range(len(CASES)), ids=[c[0] for c in CASES])
def case(request):
    _, macro, lmin, lmax, kind = CASES[request.param]
    space = P2 if kind == "p2" else hg.HG_SPACE_P1
    if kind == "p2":
        H = hg.Hierarchy(hg.Mesh(macro.xyz, macro.cells), lmin, lmax + 1)
        op = hg.Operator(H, hg.HG_OP_P2_DIVKGRAD, coeff=sg.SINPROD_AB)
        Ho = og.Hierarchy(macro, lmin, lmax, space="P2", coeff=sg.sinprod_coefficient(*sg.SINPROD_AB))
    else:
        H = hg.Hierarchy(hg.Mesh(macro.xyz, macro.cells), lmin, lmax)
        if kind == "divkgrad":
            _, xyz, _ = H.canonical_info(lmax)
            op = hg.Operator(H, hg.HG_OP_P1_DIVKGRAD, coeff=_kf(xyz))
            Ho = og.Hierarchy(macro, lmin, lmax, kind="divkgrad", coeff=_kf)
        else:
            op = hg.Operator(H)
            Ho = og.Hierarchy(macro, lmin, lmax)
    # oracle lambda per level from a seeded start vector (20 power steps)
    v0 = {l: sg.uniform_vector(70 + l, len(Ho.levels[l].interior)) for l in range(lmin + 1, lmax + 1)}
    lam = {l: og.power_lambda_max(Ho.levels[l].A, Ho.levels[l].D, v0[l]) for l in v0}
    return dict(H=H, op=op, Ho=Ho, space=space, lmin=lmin, lmax=lmax, v0=v0, lam=lam, kind=kind)


def _stored(c, L, vec_interior, dtype=torch.float64):
    lev = c["Ho"].levels[L]
    full = np.zeros(lev.n)
    full[lev.interior] = vec_interior
    return c["H"].from_canonical(L, torch.tensor(full, dtype=dtype, device="cuda"), space=c["space"])


def _interior(c, L, x):
    lev = c["Ho"].levels[L]
    got = c["H"].to_canonical(L, x, space=c["space"]).cpu().double().numpy()
    assert np.all(got[lev.boundary] == 0)
    return got[lev.interior]


def _gmg(c, **kw):
    G = hg.GMG(c["op"], nu1=1, nu2=1, lmin=c["lmin"], smoother=hg.HG_SMOOTH_CHEB, **kw)
    for l, v in c["lam"].items():
        G.set_lam(l, v)
    return G


def _oracle_smoother(c):
    lam_by_n = {len(c["Ho"].levels[l].interior): v for l, v in c["lam"].items()}

    def cheb(A, D, x, b):
        return og.chebyshev(A, D, x, b, lam_by_n[len(x)])
    return cheb


def test_power_iteration_matches_oracle(case):
    G = _gmg(case)
    for l, v0 in case["v0"].items():
        got = G.power_lambda(l, _stored(case, l, v0), iters=20)
        assert abs(got - case["lam"][l]) <= 1e-12 * case["lam"][l], l
        assert G.lam(l) == case["lam"][l]            # estimate does not replace the value in use


def test_default_estimate_is_close_to_the_largest_eigenvalue(case):
    G = hg.GMG(case["op"], nu1=1, nu2=1, lmin=case["lmin"], smoother=hg.HG_SMOOTH_CHEB)
    for l in range(case["lmin"] + 1, case["lmax"] + 1):
        lev = case["Ho"].levels[l]
        if len(lev.interior) > 3000:
            continue
        Dm = sp.diags(1.0 / np.sqrt(lev.D))
        S = (Dm @ lev.A @ Dm).toarray()
        top = np.linalg.eigvalsh(S)[-1]                 # D^-1 A is similar to D^-1/2 A D^-1/2
        est = G.lam(l)
        assert 0.85 * top <= est <= 1.05 * top, (l, est, top)


@pytest.mark.parametrize("dtype,tol", [(torch.float64, 1e-12), (torch.float32, 1e-5)])
def test_chebyshev_vcycles_match_oracle(case, dtype, tol):
    L = case["lmax"]
    lev = case["Ho"].levels[L]
    G = _gmg(case)
    b_i = sg.uniform_vector(80, len(lev.interior))
    if dtype == torch.float32:
        b_i = b_i.astype(np.float32).astype(np.float64)
    b = _stored(case, L, b_i, dtype)
    x = case["H"].zeros(L, dtype, space=case["space"])
    xo = np.zeros(len(lev.interior))
    sm = _oracle_smoother(case)
    for cyc in range(2 if dtype == torch.float64 else 1):
        G.vcycle(L, x, b)
        xo = og.vcycle(case["Ho"], L, xo, b_i, 1, 1, smoother=sm)
        assert rel_err(_interior(case, L, x), xo) <= tol, cyc


def test_fmg_matches_oracle(case):
    L = case["lmax"]
    lev = case["Ho"].levels[L]
    G = _gmg(case)
    b_i = sg.uniform_vector(81, len(lev.interior))
    x = case["H"].zeros(L, torch.float64, space=case["space"])
    x.fill_(7.0)                                       # input ignored
    G.fmg(L, x, _stored(case, L, b_i), cycles=5)
    xo = og.fmg(case["Ho"], b_i, cycles=5, nu1=1, nu2=1, smoother=_oracle_smoother(case))
    assert rel_err(_interior(case, L, x), xo) <= 1e-11
    # FP32 FMG: same iterate to single precision
    x32 = case["H"].zeros(L, torch.float32, space=case["space"])
    G.fmg(L, x32, _stored(case, L, b_i, torch.float32), cycles=5)
    assert rel_err(_interior(case, L, x32), xo) <= 1e-4


@pytest.mark.parametrize("precision", [hg.HG_PREC_F64, hg.HG_PREC_MIXED])
def test_chebyshev_solve_converges(case, precision):
    L = case["lmax"]
    lev = case["Ho"].levels[L]
    G = hg.GMG(case["op"], nu1=1, nu2=1, lmin=case["lmin"], smoother=hg.HG_SMOOTH_CHEB)
    b_i = sg.uniform_vector(82, len(lev.interior))
    x = case["H"].zeros(L, torch.float64, space=case["space"])
    it, rel = G.solve(x, _stored(case, L, b_i), tol=1e-10, max_iter=60, precision=precision)
    xg = _interior(case, L, x)
    assert rel <= 1e-10 and np.linalg.norm(b_i - lev.A @ xg) <= 1.01e-10 * np.linalg.norm(b_i)
    assert it <= 30


def test_fmg_reaches_discretization_accuracy():
    """Poisson with u = sin(pi x) sin(pi y) sin(pi z) on the unit cube (6 Kuhn
    cells), P1 levels 1..6: FMG with 5 V(1,1) Chebyshev cycles per level ends
    with ||x - x_h|| far below the discretization error ||x_h - u||."""
    macro, L = sg.kuhn_cube(1), 6
    H = hg.Hierarchy(hg.Mesh(macro.xyz, macro.cells), 1, L)
    op = hg.Operator(H)
    mass = hg.Operator(H, hg.HG_OP_P1_MASS)
    _, xyz, dirich = H.canonical_info(L)
    u = np.prod(np.sin(np.pi * xyz), axis=1)
    f = 3 * np.pi ** 2 * u
    b = H.zeros(L, torch.float64)
    mass.apply(L, H.from_canonical(L, torch.tensor(f, device="cuda")), b)
    G = hg.GMG(op, nu1=1, nu2=1, smoother=hg.HG_SMOOTH_CHEB)
    x = H.zeros(L, torch.float64)
    G.fmg(L, x, b, cycles=5)
    xh = H.zeros(L, torch.float64)
    hg.GMG(op).solve(xh, b, tol=1e-13, max_iter=100)
    xf = H.to_canonical(L, x).cpu().numpy()
    xd = H.to_canonical(L, xh).cpu().numpy()
    inner = ~dirich.astype(bool)
    alg = np.linalg.norm((xf - xd)[inner])
    disc = np.linalg.norm((xd - u)[inner])
    assert alg < 0.02 * disc, (alg, disc)


def test_chebyshev_parameters_rejected():
    macro = sg.kuhn_cube(1)
    H = hg.Hierarchy(hg.Mesh(macro.xyz, macro.cells), 1, 3)
    op = hg.Operator(H)
    for kw in (dict(cheb_order=0), dict(cheb_iters=0), dict(cheb_interval=(0.0, 1.1)),
               dict(cheb_interval=(1.2, 1.1))):
        with pytest.raises(hg.HGError) as e:
            hg.GMG(op, smoother=hg.HG_SMOOTH_CHEB, **kw)
        assert e.value.code == -1
    G = hg.GMG(op, smoother=hg.HG_SMOOTH_CHEB)
    with pytest.raises(hg.HGError):
        G.set_lam(1, 1.0)                                # coarsest level is not smoothed
    with pytest.raises(hg.HGError):
        G.set_lam(3, -1.0)
    with pytest.raises(hg.HGError):
        G.power_lambda(3, H.zeros(3, torch.float64))     # zero start vector
