"""Pins of the polynomial surrogate-stencil oracle (oracle.surrogate).

A coefficient that is constant (degree 0) or linear in x (degree 1) makes the
stencil weights polynomials of that degree in the position, so the
surrogate must reproduce the exact operator; for the smooth sinprod
coefficient the error must fall with the degree.  The extracted exact
weights are checked against two properties of the assembled matrix: zero
row sums and symmetry w(p, d) = w(p + d, -d)."""
import numpy as np
import pytest

import synthgen as sg
from oracle import surrogate as su

MESHES = [sg.kuhn_cube(1), sg.permuted_cells(sg.kuhn_cube(1), 3)]


def _err(S, A, seed=5):
    x = sg.uniform_vector(seed, S.rm.n_vertices)
    ref = S.A @ x
    return np.linalg.norm(A @ x - ref) / np.linalg.norm(ref)


@pytest.mark.parametrize("macro", MESHES, ids=["cube1", "cube1perm"])
def test_surrogate_is_exact_for_polynomial_coefficients(macro):
    S0 = su.SurrogateLevel(macro, 3, lambda X: np.full(len(X), 2.0))
    assert _err(S0, S0.surrogate(0)) < 1e-13
    S1 = su.SurrogateLevel(macro, 3, lambda X: 1.0 + X @ np.array([1.0, 2.0, 3.0]))
    assert _err(S1, S1.surrogate(0)) > 1e-2          # degree 0 cannot follow a linear k
    assert _err(S1, S1.surrogate(1)) < 1e-13


@pytest.mark.parametrize("macro", MESHES, ids=["cube1", "cube1perm"])
def test_surrogate_error_falls_with_the_degree(macro):
    S = su.SurrogateLevel(macro, 3, sg.sinprod_coefficient(*sg.SINPROD_AB))
    errs = [_err(S, S.surrogate(q)) for q in range(4)]
    assert all(b < a for a, b in zip(errs, errs[1:])), errs
    assert errs[-1] < 0.02


def test_exact_weights_have_zero_row_sums_and_are_symmetric():
    S = su.SurrogateLevel(sg.kuhn_cube(1), 3, sg.sinprod_coefficient(*sg.SINPROD_AB))
    scale = np.abs(S.A).max()
    for ids, nb, w in S.cells:
        assert np.abs(w.sum(axis=1)).max() < 1e-13 * scale
        for d in range(1, len(su.DIRS)):
            back = d + 1 if d % 2 else d - 1                    # the opposite direction
            wt = np.asarray(S.A[nb[:, d], ids]).ravel()
            assert np.allclose(w[:, d], wt, rtol=1e-13, atol=1e-15)
            assert np.all(su.DIRS[back] == -su.DIRS[d])


def test_exact_operator_is_the_multigrid_oracles_operator():
    """The surrogate's exact A is the same div-k-grad matrix the multigrid
    oracle assembles for the same coefficient (the pinned element matrix)."""
    from oracle import gmg
    kf = sg.sinprod_coefficient(*sg.SINPROD_AB)
    S = su.SurrogateLevel(sg.kuhn_cube(1), 3, kf)
    lev = gmg.Level(sg.kuhn_cube(1), 3, kind="divkgrad", coeff=kf)
    assert abs(S.A - lev.A_full).max() <= 1e-14 * abs(lev.A_full).max()


def test_fitted_weights_are_the_least_squares_projection():
    """The fitted interior weights w_s = B c satisfy the normal equations
    B^T (w - w_s) = 0 for the monomial basis B of the interior points (a
    wrong basis, a wrong point set or a dropped term fails it)."""
    S = su.SurrogateLevel(sg.kuhn_cube(1), 4, sg.sinprod_coefficient(*sg.SINPROD_AB))
    for q in (1, 2, 3):
        A = S.surrogate(q)
        ex = su.exponents(q)
        u = S.ijk / S.n
        B = np.stack([u[:, 0] ** a * u[:, 1] ** b * u[:, 2] ** c for a, b, c in ex], axis=1)
        for ids, nb, w in S.cells:
            ws = np.stack([np.asarray(A[ids, nb[:, d]]).ravel() for d in range(len(su.DIRS))],
                          axis=1)
            r = B.T @ (w - ws)
            assert np.abs(r).max() <= 1e-10 * np.abs(B.T @ w).max(), q


def test_seven_point_cube_weights_vanish_outside_the_seven_directions():
    """On a Kuhn-ordered cube the exact div-k-grad weights (any k) are exact
    zeros outside centre, +-(1,0,0), +-(1,-1,0), +-(0,-1,1), so every fitted
    coefficient there is zero: what the library's seven-point surrogate path
    relies on."""
    S = su.SurrogateLevel(sg.kuhn_cube(1), 3, sg.sinprod_coefficient(*sg.SINPROD_AB))
    seven = {(0, 0, 0), (1, 0, 0), (-1, 0, 0), (1, -1, 0), (-1, 1, 0), (0, -1, 1), (0, 1, -1)}
    off = [d for d, v in enumerate(su.DIRS) if tuple(v) not in seven]
    assert len(off) == 8
    for ids, nb, w in S.cells:
        assert np.all(w[:, off] == 0.0)
    A = S.surrogate(3)
    for ids, nb, w in S.cells:
        for d in off:
            assert np.all(np.asarray(A[ids, nb[:, d]]).ravel() == 0.0)
