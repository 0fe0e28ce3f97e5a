"""Pins of the Nedelec (N1) curl-curl oracle against what the mathematics fixes.

Each check would catch a plausible mistake: a dropped or mis-signed term of
the basis (pointwise reproduction, finite-difference curls), a wrong mass
integral (quadrature), a wrong orientation or gradient map (curl grad = 0,
G^T M G = P1 stiffness, commuting transfers), wrong boundary edges (kernel
dimension), and a broken hybrid smoother (level-independent rates, gain over
plain edge smoothing)."""
import numpy as np
import pytest
import scipy.sparse.linalg as spla

import synthgen as sg
from oracle import fem, gmg
from oracle import nedelec as ne
from oracle import quadrature as quad


def _rand_tet(seed):
    g = np.random.Generator(np.random.PCG64(seed))
    X = g.uniform(-1, 1, size=(4, 3))
    J = np.stack([X[1] - X[0], X[2] - X[0], X[3] - X[0]], axis=1)
    if np.linalg.det(J) < 0:
        X[[1, 2]] = X[[2, 1]]
    return X


def _local_dofs(X, u):
    """Tangential line integrals over the 6 local edges (local orientation)."""
    out = np.zeros(6)
    for e, (a, b) in enumerate(ne.LOCAL_EDGES):
        t = X[b] - X[a]
        for s, w in zip(ne._GL_X, ne._GL_W):
            out[e] += w * u((X[a] + s * t)[None])[0] @ t
    return out


@pytest.mark.parametrize("seed", [1, 2, 3])
def test_basis_reproduces_constant_and_rotational_fields(seed):
    X = _rand_tet(seed)
    G, _ = fem.bary_gradients(X[None])
    g = np.random.Generator(np.random.PCG64(seed + 100))
    a, c = g.normal(size=3), g.normal(size=3)

    def u(x):
        return a[None] + np.cross(c[None], x)

    coef = _local_dofs(X, u)
    lam = g.dirichlet(np.ones(4), size=20)
    W = ne.whitney(lam, G[0])                                  # (20, 6, 3)
    got = np.einsum("e,qed->qd", coef, W)
    assert np.allclose(got, u(lam @ X), rtol=0, atol=1e-12)


def test_basis_curls_by_finite_differences():
    X = _rand_tet(7)
    G, _ = fem.bary_gradients(X[None])
    J = np.stack([X[1] - X[0], X[2] - X[0], X[3] - X[0]], axis=1)
    Jinv = np.linalg.inv(J)

    def lam_of(x):
        l123 = Jinv @ (x - X[0])
        return np.concatenate([[1 - l123.sum()], l123])

    x0 = X.mean(axis=0)
    h = 1e-3
    dW = np.zeros((3, 6, 3))                                   # d w_e / d x_k
    for k in range(3):
        ek = np.eye(3)[k] * h
        dW[k] = (ne.whitney(lam_of(x0 + ek)[None], G[0])[0]
                 - ne.whitney(lam_of(x0 - ek)[None], G[0])[0]) / (2 * h)
    curl = np.stack([dW[1, :, 2] - dW[2, :, 1], dW[2, :, 0] - dW[0, :, 2],
                     dW[0, :, 1] - dW[1, :, 0]], axis=1)
    assert np.allclose(curl, ne.whitney_curls(G)[0], rtol=0, atol=1e-9)


def test_mass_matrix_by_quadrature():
    X = np.stack([_rand_tet(s) for s in (11, 12)])
    G, vol = fem.bary_gradients(X)
    bary, w = quad.sym14()                                     # degree 5 >= 2
    M = np.zeros((2, 6, 6))
    for t in range(2):
        W = ne.whitney(bary, G[t])
        M[t] = vol[t] * np.einsum("q,qed,qfd->ef", w, W, W)
    assert np.allclose(ne.mass_local(X), M, rtol=1e-13, atol=1e-15)
    K = ne.curlcurl_local(X)
    assert np.allclose(K, np.swapaxes(K, 1, 2)) and np.linalg.eigvalsh(M).min() > 0


# the permuted mesh has local orientations that disagree with the global ones;
# the skewed tetrahedron has no edge along a coordinate axis
PERM = sg.permuted_cells(sg.kuhn_cube(1), 3)
SKEW = sg.MacroMesh(np.array([[0, 0, 0], [2, 1, 0], [1, 3, 1], [0, 1, 2]], dtype=np.int64),
                    np.array([[0, 1, 2, 3]], dtype=np.int64), 1, "skew_tet")


@pytest.mark.parametrize("macro,level", [(sg.kuhn_cube(1), 2), (sg.reference_tet(), 3), (PERM, 2),
                                         (SKEW, 2)])
def test_curl_grad_zero_and_gradient_mass_is_p1_stiffness(macro, level):
    lev = ne.NedelecLevel(macro, level)
    KG = lev.K_full @ lev.G_full
    assert abs(KG).max() <= 1e-12 * abs(lev.K_full).max()
    K1 = fem.assemble(lev.rm.cells, fem.p1_stiffness(lev.rm.cell_xyz), lev.rm.n_vertices)
    assert abs(lev.G_full.T @ lev.M_full @ lev.G_full - K1).max() <= 1e-12 * abs(K1).max()


@pytest.mark.parametrize("macro", [sg.kuhn_cube(2), sg.permuted_cells(sg.kuhn_cube(2), 5)])
def test_interpolant_energies_on_the_unit_cube(macro):
    lev = ne.NedelecLevel(macro, 1)
    a = np.array([0.3, -1.2, 0.7])
    c = np.array([1.1, 0.4, -0.8])
    ua = lev.interpolate(lambda x: np.broadcast_to(a, x.shape))
    assert abs(ua @ lev.M_full @ ua - a @ a) <= 1e-12
    uc = lev.interpolate(lambda x: np.cross(c[None], x))
    assert abs(uc @ lev.K_full @ uc - 4 * c @ c) <= 1e-12     # curl (c x x) = 2c, |Omega| = 1
    mom = np.full((3, 3), 0.25) + np.eye(3) * (1 / 3 - 0.25)  # int x_i x_j over [0,1]^3
    exact = (c @ c) * np.trace(mom) - c @ mom @ c             # int |c x x|^2
    assert abs(uc @ lev.M_full @ uc - exact) <= 1e-12


@pytest.mark.parametrize("macro,level", [(sg.kuhn_cube(1), 2), (sg.reference_tet(), 2), (PERM, 2),
                                         (SKEW, 2)])
def test_prolongation_commutes_with_gradient_and_reproduces_rotations(macro, level):
    f, c = ne.NedelecLevel(macro, level), ne.NedelecLevel(macro, level - 1)
    P = ne.nedelec_prolongation(f, c)
    P1 = gmg.p1_prolongation(gmg.Level(macro, level), gmg.Level(macro, level - 1))
    assert abs(P @ c.G_full - f.G_full @ P1).max() <= 1e-14
    a, r = np.array([0.2, 0.5, -0.4]), np.array([-0.7, 0.3, 1.3])

    def u(x):
        return a[None] + np.cross(r[None], x)

    assert np.allclose(P @ c.interpolate(u), f.interpolate(u), rtol=0, atol=1e-13)


@pytest.mark.parametrize("macro,level", [(sg.kuhn_cube(1), 1), (sg.reference_tet(), 2), (PERM, 1)])
def test_curlcurl_kernel_is_the_interior_gradients(macro, level):
    lev = ne.NedelecLevel(macro, level)
    ii = lev.interior
    K = lev.K_full[ii][:, ii].toarray()
    ev = np.linalg.eigvalsh(K)
    null = int(np.sum(ev < 1e-10 * ev.max()))
    assert null == len(lev.rm.interior)


def test_interpolation_error_is_first_order():
    bary, w = quad.sym14()
    errs = []
    for L in (2, 3, 4):
        lev = ne.NedelecLevel(sg.kuhn_cube(1), L)
        x = lev.interpolate(ne.manufactured)
        X = lev.rm.cell_xyz
        _, vol = fem.bary_gradients(X)
        uh = lev.evaluate(x, bary)
        pts = np.einsum("qi,tid->tqd", bary, X)
        d = uh - ne.manufactured(pts.reshape(-1, 3)).reshape(uh.shape)
        errs.append(np.sqrt(np.einsum("t,q,tqd,tqd->", vol, w, d, d)))
    rates = np.log2(np.array(errs[:-1]) / np.array(errs[1:]))
    assert np.all(rates > 0.9) and np.all(rates < 1.3), rates


def _rate(H, L, cycles=6, **kw):
    lev = H.levels[L]
    b = sg.uniform_vector(5, len(lev.interior))
    x = np.zeros_like(b)
    r = [np.linalg.norm(b)]
    for _ in range(cycles):
        x = ne.vcycle(H, L, x, b, **kw)
        r.append(np.linalg.norm(b - lev.A @ x))
    return (r[-1] / r[2]) ** (1 / (cycles - 2))


@pytest.mark.parametrize("macro", [sg.kuhn_cube(1), sg.reference_tet(), PERM, SKEW])
def test_galerkin_identity(macro):
    """Coarse N1 functions are fine N1 functions (nested spaces), so
    P^T A_f P equals the rediscretised coarse matrix."""
    H = ne.NedelecHierarchy(macro, 1, 3, alpha=1.0, beta=0.3)
    for l in (2, 3):
        P, Af, Ac = H.P[l], H.levels[l].A, H.levels[l - 1].A
        assert abs(P.T @ Af @ P - Ac).max() <= 1e-13 * abs(Ac).max()


def test_hiptmair_vcycle_is_level_independent_and_needs_the_potential_step():
    macro = sg.kuhn_cube(1)
    H3 = ne.NedelecHierarchy(macro, 1, 3, alpha=1.0, beta=1e-2)
    H4 = ne.NedelecHierarchy(macro, 1, 4, alpha=1.0, beta=1e-2)
    r3, r4 = _rate(H3, 3), _rate(H4, 4)                        # damped Jacobi, omega = 1/2
    assert r3 < 0.8 and r4 < 0.8 and abs(r3 - r4) < 0.05, (r3, r4)
    # without the potential-space step the near-kernel (gradient) errors stall
    no_pot = _rate(H4, 4, potential_smoother=lambda A, D, x, b: x)
    assert no_pot > 0.95, no_pot
    # order-2 Chebyshev smoothing in both spaces (the paper's choice)
    lam = {}
    for l in range(2, 5):
        lev = H4.levels[l]
        lam["e", len(lev.D)] = gmg.power_lambda_max(lev.A, lev.D, sg.uniform_vector(3, len(lev.D)))
        lam["p", len(lev.Dp)] = gmg.power_lambda_max(lev.Ap, lev.Dp, sg.uniform_vector(4, len(lev.Dp)))
    rc = _rate(H4, 4, edge_smoother=lambda A, D, x, b: gmg.chebyshev(A, D, x, b, lam["e", len(x)]),
               potential_smoother=lambda A, D, x, b: gmg.chebyshev(A, D, x, b, lam["p", len(x)]))
    assert rc < 0.55, rc


def test_manufactured_solution_and_fmg():
    """alpha = beta = 1: f = (2 pi^2 + 1) u.  The discrete solution converges
    in L2 at first order, and FMG with 5 V(1,1) per level and order-2
    Chebyshev smoothing in both spaces (Sec. 6) leaves an L2 algebraic error
    below 5 % of the L2 discretization error."""
    bary, w = quad.sym14()
    H = ne.NedelecHierarchy(sg.kuhn_cube(1), 1, 4)
    errs = []
    for L in (2, 3, 4):
        lev = H.levels[L]
        b = lev.load_vector(lambda x: (2 * np.pi ** 2 + 1) * ne.manufactured(x), (bary, w))
        bi = b[lev.interior]
        xi = spla.spsolve(lev.A.tocsc(), bi)
        x = np.zeros(lev.n)
        x[lev.interior] = xi
        X = lev.rm.cell_xyz
        _, vol = fem.bary_gradients(X)
        uh = lev.evaluate(x, bary)
        pts = np.einsum("qi,tid->tqd", bary, X)
        d = uh - ne.manufactured(pts.reshape(-1, 3)).reshape(uh.shape)
        errs.append(np.sqrt(np.einsum("t,q,tqd,tqd->", vol, w, d, d)))
    rates = np.log2(np.array(errs[:-1]) / np.array(errs[1:]))
    assert np.all(rates > 0.8), rates
    lam = {}
    for l in range(2, 5):
        lv = H.levels[l]
        lam["e", len(lv.D)] = gmg.power_lambda_max(lv.A, lv.D, sg.uniform_vector(3, len(lv.D)))
        lam["p", len(lv.Dp)] = gmg.power_lambda_max(lv.Ap, lv.Dp, sg.uniform_vector(4, len(lv.Dp)))
    xf = ne.fmg(H, bi, cycles=5,
                edge_smoother=lambda A, D, x, b: gmg.chebyshev(A, D, x, b, lam["e", len(x)]),
                potential_smoother=lambda A, D, x, b: gmg.chebyshev(A, D, x, b, lam["p", len(x)]))
    e = xf - xi
    Mi = lev.M_full[lev.interior][:, lev.interior]
    assert np.sqrt(e @ Mi @ e) < 0.05 * errs[-1]
