"""Pins of the oracle's textbook geometric multigrid."""
import numpy as np
import pytest
import scipy.sparse.linalg as spla

import synthgen as sg
from oracle import gmg


def _manufactured_rhs(lev):
    x, y, z = lev.xyz.T
    f = 3 * np.pi ** 2 * np.sin(np.pi * x) * np.sin(np.pi * y) * np.sin(np.pi * z)
    return (lev.M_full @ f)[lev.interior]


@pytest.mark.parametrize("macro,lmin,lmax", [(sg.reference_tet(), 2, 4), (sg.kuhn_cube(1), 1, 3),
                                            (sg.permuted_cells(sg.kuhn_cube(1), 3), 1, 3)])
def test_galerkin_identity_p1(macro, lmin, lmax):
    H = gmg.Hierarchy(macro, lmin, lmax)
    for l in range(lmin + 1, lmax + 1):
        P = H.P[l]
        Ac = (P.T @ H.levels[l].A @ P).toarray()
        assert np.allclose(Ac, H.levels[l - 1].A.toarray(), atol=1e-13)


@pytest.mark.parametrize("macro", [sg.kuhn_cube(1), sg.permuted_cells(sg.kuhn_cube(1), 3)],
                         ids=["cube1", "cube1perm"])
def test_prolongation_reproduces_linear_and_quadratic_functions(macro):
    H = gmg.Hierarchy(macro, 1, 3)
    f = lambda X: 0.3 + X @ np.array([1.0, -2.0, 0.5])
    for l in (2, 3):
        fi, co = H.levels[l], H.levels[l - 1]
        from oracle.gmg import p1_prolongation
        P = p1_prolongation(fi, co)
        assert np.allclose(P @ f(co.xyz), f(fi.xyz), atol=1e-14)
    H2 = gmg.Hierarchy(macro, 1, 2, space="P2")
    fi, co = H2.levels[2], H2.levels[1]
    q = lambda X: X[:, 0] ** 2 - 0.5 * X[:, 1] * X[:, 2] + X[:, 2]
    P = gmg.p2_prolongation(fi, co)
    assert np.allclose(P @ q(co.xyz), q(fi.xyz), atol=1e-14)


def test_coarse_level_is_solved_exactly():
    H = gmg.Hierarchy(sg.kuhn_cube(2), 1, 2)
    lev = H.levels[1]
    b = np.random.default_rng(0).uniform(-1, 1, len(lev.interior))
    x = gmg.vcycle(H, 1, np.zeros_like(b), b)
    assert np.allclose(lev.A @ x, b, atol=1e-13)


def test_vcycle_contraction_level_independent():
    rates = []
    for L in (3, 4, 5):
        H = gmg.Hierarchy(sg.kuhn_cube(1), 1, L)
        b = _manufactured_rhs(H.levels[L])
        x, it, hist = gmg.solve(H, b, tol=1e-10)
        rates.append((hist[-1] / hist[1]) ** (1.0 / max(it - 1, 1)))
    # weighted Jacobi (w = 2/3) V(3,3) on the 3D P1 Laplacian: the rate saturates
    # (0.27, 0.35, 0.38, 0.39 for L = 3..6): level independence shows as shrinking steps
    assert max(rates) < 0.42
    assert rates[2] - rates[1] < rates[1] - rates[0]


def test_solution_matches_direct_solve():
    H = gmg.Hierarchy(sg.reference_tet(), 2, 4)
    lev = H.levels[4]
    assert lev.n == 969 and len(lev.interior) == 455
    b = _manufactured_rhs(lev)
    x, it, hist = gmg.solve(H, b, tol=1e-10)
    xd = spla.spsolve(lev.A.tocsc(), b)
    assert hist[-1] <= 1e-10
    assert np.linalg.norm(x - xd) <= 1e-8 * np.linalg.norm(xd)


def test_p1_l2_error_is_second_order():
    errs = []
    for L in (2, 3, 4, 5):
        H = gmg.Hierarchy(sg.kuhn_cube(1), 1, L)
        lev = H.levels[L]
        b = _manufactured_rhs(lev)
        xh, _, _ = gmg.solve(H, b, tol=1e-11)
        u = np.prod(np.sin(np.pi * lev.xyz), axis=1)
        e = u.copy()
        e[lev.interior] -= xh
        errs.append(np.sqrt(e @ (lev.M_full @ e)))
    ratios = [errs[i] / errs[i + 1] for i in range(len(errs) - 1)]
    assert 3.5 < ratios[-1] < 4.5, ratios


def test_gauss_seidel_colouring_is_conflict_free_and_converges():
    H = gmg.Hierarchy(sg.kuhn_cube(1), 1, 3)
    lev = H.levels[3]
    c = lev.rm.coords[lev.interior]
    colour = c.sum(axis=1) % 4
    A = lev.A.tocoo()
    off = A.row != A.col
    assert np.all(colour[A.row[off]] != colour[A.col[off]])
    b = _manufactured_rhs(lev)
    cols = {l: H.levels[l].rm.coords[H.levels[l].interior].sum(axis=1) % 4 for l in H.levels}
    # smoother per level needs that level's colouring; run a two-level check on the finest
    x = np.zeros_like(b)
    r0 = np.linalg.norm(b)
    for _ in range(20):
        x = gmg.gauss_seidel_colours(lev.A, lev.D, x, b, colour)
    assert np.linalg.norm(b - lev.A @ x) < r0


def test_chebyshev_error_polynomial_on_diagonal_matrix():
    """For A = diag(lam) and D = I the Chebyshev step with b = 0 multiplies each
    error component by the scaled Chebyshev polynomial T_k((theta - lam)/delta) /
    T_k(theta/delta) (closed form), k = order."""
    import scipy.sparse as sp
    lam = np.linspace(0.05, 2.0, 37)
    A = sp.diags(lam).tocsr()
    D = np.ones_like(lam)
    e0 = np.ones_like(lam)
    lmax = 2.0
    for order in (1, 2, 3):
        e = gmg.chebyshev(A, D, e0.copy(), np.zeros_like(lam), lmax, order=order)
        a, c = 0.1 * lmax, 1.1 * lmax
        theta, delta = (a + c) / 2, (c - a) / 2
        Tk = np.polynomial.chebyshev.Chebyshev.basis(order)
        assert np.allclose(e, Tk((theta - lam) / delta) / Tk(theta / delta), rtol=1e-12, atol=1e-14)


def test_chebyshev_order_one_is_weighted_jacobi():
    H = gmg.Hierarchy(sg.kuhn_cube(1), 1, 3)
    lev = H.levels[3]
    x = sg.uniform_vector(3, len(lev.interior))
    b = sg.uniform_vector(4, len(lev.interior))
    lmax = 1.7
    theta = 0.6 * lmax
    assert np.allclose(gmg.chebyshev(lev.A, lev.D, x, b, lmax, order=1),
                       gmg.jacobi(lev.A, lev.D, x, b, 1.0 / theta), rtol=1e-14, atol=1e-14)


def test_power_iteration_finds_the_largest_eigenvalue():
    import scipy.sparse as sp
    lam = np.array([0.3, 1.0, 2.5, 0.7])
    A = sp.diags(lam).tocsr()
    got = gmg.power_lambda_max(A, np.ones(4), np.ones(4), iters=200)
    assert abs(got - 2.5) < 1e-12
    H = gmg.Hierarchy(sg.kuhn_cube(1), 2, 3)
    lev = H.levels[3]
    dense = np.linalg.eigvals(np.diag(1 / lev.D) @ lev.A.toarray()).real.max()
    est = gmg.power_lambda_max(lev.A, lev.D, sg.uniform_vector(9, len(lev.interior)), iters=400)
    assert abs(est - dense) < 1e-3 * dense and est <= dense * (1 + 1e-12)


def test_fmg_reaches_discretization_accuracy():
    """FMG with 5 V(1,1) Chebyshev-smoothed cycles per level on the manufactured
    Poisson problem (u = sin pi x sin pi y sin pi z on the unit cube): the
    algebraic error ||x - x_h|| is far below the discretization error ||x_h - u||."""
    import scipy.sparse.linalg as spla
    H = gmg.Hierarchy(sg.kuhn_cube(1), 1, 4)
    lev = H.levels[4]
    f = 3 * np.pi ** 2 * np.prod(np.sin(np.pi * lev.xyz), axis=1)
    b = (lev.M_full @ f)[lev.interior]
    lam = {len(H.levels[l].interior): gmg.power_lambda_max(
        H.levels[l].A, H.levels[l].D, sg.uniform_vector(11, len(H.levels[l].interior)))
        for l in range(2, 5)}

    def cheb(A, D, x, bb):
        return gmg.chebyshev(A, D, x, bb, lam[len(x)])

    x = gmg.fmg(H, b, cycles=5, nu1=1, nu2=1, smoother=cheb)
    xh = spla.spsolve(lev.A.tocsc(), b)
    u = np.prod(np.sin(np.pi * lev.xyz), axis=1)[lev.interior]
    assert np.linalg.norm(x - xh) < 0.05 * np.linalg.norm(xh - u)


def test_colour_gauss_seidel_is_the_sequential_sweep():
    """With no coupling inside a colour, the colour-ordered sweep equals the
    textbook point Gauss-Seidel sweep taken one DoF at a time in colour order;
    on a diagonal matrix one sweep solves exactly."""
    import scipy.sparse as sp
    g = np.random.Generator(np.random.PCG64(12))
    n = 40
    colour = np.arange(n) % 4
    # couple only DoFs of different colours (a symmetric, diagonally dominant matrix)
    R = g.uniform(-1, 1, size=(n, n))
    R = np.triu(R, 1) * (colour[:, None] != colour[None, :])
    A = R + R.T
    A += np.diag(np.abs(A).sum(axis=1) + 1.0)
    As = sp.csr_matrix(A)
    D = A.diagonal()
    x0, b = g.uniform(-1, 1, n), g.uniform(-1, 1, n)
    x = x0.copy()
    for c in range(4):
        for i in np.flatnonzero(colour == c):
            x[i] += (b[i] - A[i] @ x) / A[i, i]
    assert np.allclose(gmg.gauss_seidel_colours(As, D, x0, b, colour), x, rtol=1e-13, atol=1e-14)
    Dm = sp.diags(np.linspace(1, 3, n)).tocsr()
    xs = gmg.gauss_seidel_colours(Dm, Dm.diagonal(), x0, b, colour)
    assert np.allclose(xs, b / Dm.diagonal(), rtol=1e-15)


def test_fmg_coarse_start_is_the_galerkin_projection():
    """With no V-cycles FMG returns P A_c^-1 P^T b on two levels.  For the P1
    Laplacian A_c = P^T A P (Galerkin), so the residual is orthogonal to the
    coarse space: P^T (b - A x) = 0."""
    H = gmg.Hierarchy(sg.kuhn_cube(1), 2, 3)
    lev = H.levels[3]
    b = sg.uniform_vector(13, len(lev.interior))
    x = gmg.fmg(H, b, cycles=0)
    r = b - lev.A @ x
    assert np.linalg.norm(H.P[3].T @ r) <= 1e-12 * np.linalg.norm(b)
