"""Pins of the oracle's element matrices, quadrature and assembly (Sec. 5.2)."""
import itertools

import numpy as np
import pytest
import scipy.sparse as sp

import synthgen as sg
from oracle import fem, quadrature
from oracle.mesh import RefinedMesh, coord_key


def _assembled(macro, level, kind="laplace"):
    rm = RefinedMesh(macro, level)
    X = rm.cell_xyz
    K = {"laplace": fem.p1_stiffness, "mass": fem.p1_mass}[kind](X)
    return rm, fem.assemble(rm.cells, K, rm.n_vertices)


def test_p1_element_matrices_closed_forms():
    X = np.array([[[0, 0, 0], [1, 0, 0], [0, 1, 0], [0, 0, 1]]], dtype=float)
    K = fem.p1_stiffness(X)[0]
    # reference tet: grad l0 = (-1,-1,-1), grad l1..3 = unit vectors, |T| = 1/6
    G = np.array([[-1, -1, -1], [1, 0, 0], [0, 1, 0], [0, 0, 1]], dtype=float)
    assert np.allclose(K, G @ G.T / 6)
    M = fem.p1_mass(X)[0]
    assert np.allclose(M, (np.ones((4, 4)) + np.eye(4)) / 120)


@pytest.mark.parametrize("macro,level", [(sg.reference_tet(), 3), (sg.kuhn_cube(1), 2),
                                         (sg.kuhn_cube(2), 1), (sg.permuted_cells(sg.kuhn_cube(1), 3), 2)])
def test_p1_laplace_symmetric_zero_rowsum_patch(macro, level):
    rm, A = _assembled(macro, level)
    assert abs(A - A.T).max() < 1e-14
    assert np.abs(A @ np.ones(rm.n_vertices)).max() < 1e-13
    lin = rm.xyz @ np.array([0.3, -1.7, 2.2]) + 0.5
    r = A @ lin
    assert np.abs(r[rm.interior]).max() < 1e-12            # linear patch test


@pytest.mark.parametrize("macro,vol", [(sg.reference_tet(), 1 / 6), (sg.kuhn_cube(2), 1.0),
                                       (sg.permuted_cells(sg.kuhn_cube(2), 7), 1.0)])
def test_p1_mass_total(macro, vol):
    rm, M = _assembled(macro, 2, "mass")
    one = np.ones(rm.n_vertices)
    assert np.isclose(one @ (M @ one), vol, rtol=1e-14)


def test_reference_tet_interior_stencil_closed_form():
    # interior row of the reference-tet Laplacian, times 3n (hand-derived closed form)
    level = 3
    n = 2 ** level
    rm, A = _assembled(sg.reference_tet(), level)
    expect = {(0, 0, 0): 20, (1, 0, 0): -4, (0, 1, 0): -2, (0, 0, 1): -4,
              (-1, 1, 0): -1, (0, -1, 1): -1, (-1, 0, 1): 1, (1, -1, 1): 1}
    full = dict(expect)
    for d, v in expect.items():
        full[tuple(-x for x in d)] = v
    keys = coord_key(rm.coords, rm.side)
    p = np.array([2, 2, 2])
    row = np.searchsorted(keys, coord_key(p, rm.side))
    got = {}
    A = A.tocsr()
    for idx, val in zip(A.indices[A.indptr[row]:A.indptr[row + 1]],
                        A.data[A.indptr[row]:A.indptr[row + 1]]):
        d = tuple(rm.coords[idx] - p)
        if abs(val) > 1e-14:
            got[d] = val * 3 * n
    assert set(got) == {d for d, v in full.items() if v != 0}
    for d, v in full.items():
        if v:
            assert np.isclose(got[d], v, rtol=1e-13, atol=1e-13)


@pytest.mark.parametrize("m,level", [(1, 3), (2, 2)])
def test_kuhn_cube_laplacian_is_h_times_7_point(m, level):
    rm, A = _assembled(sg.kuhn_cube(m), level)
    N = m * 2 ** level
    h = 1.0 / N
    # textbook 7-point Laplacian on the (N+1)^3 grid with Neumann-free full rows
    T1 = sp.diags([-np.ones(N), 2 * np.ones(N + 1), -np.ones(N)], [-1, 0, 1]).tolil()
    T1[0, 0] = T1[N, N] = 1.0
    I = sp.identity(N + 1)
    L = sp.kron(sp.kron(I, I), T1) + sp.kron(sp.kron(I, T1), I) + sp.kron(sp.kron(T1, I), I)
    # canonical order: x fastest, z slowest == kron(Iz, Iy, Tx) ordering
    diff = (A - h * L.tocsr())
    ii = rm.interior
    assert abs(diff[ii][:, ii]).max() < 1e-13
    assert abs(diff[ii]).max() < 1e-13


def test_quadrature_exactness():
    bary, w = quadrature.sym14()
    assert len(w) == 14 and np.all(w > 0) and np.isclose(w.sum(), 1.0, atol=1e-15)
    for deg in range(6):
        for al in itertools.product(range(deg + 1), repeat=4):
            if sum(al) != deg:
                continue
            q = (w * np.prod(bary ** np.array(al), axis=1)).sum()
            assert abs(q - quadrature.exact_monomial(al)) < 1e-15
    # degree 6 is not integrated exactly (the rule is exactly of degree 5)
    al = (6, 0, 0, 0)
    assert abs((w * bary[:, 0] ** 6).sum() - quadrature.exact_monomial(al)) > 1e-6
    for qn in (2, 3, 4):
        b2, w2 = quadrature.stroud_conical(qn)
        assert np.all(w2 > 0)
        for al in itertools.product(range(2 * qn), repeat=4):
            if sum(al) <= 2 * qn - 1:
                q = (w2 * np.prod(b2 ** np.array(al), axis=1)).sum()
                assert abs(q - quadrature.exact_monomial(al)) < 1e-14


@pytest.mark.parametrize("macro", [sg.kuhn_cube(1), sg.permuted_cells(sg.kuhn_cube(1), 3)],
                         ids=["cube1", "cube1perm"])
def test_p2_stiffness_and_mass_invariants(macro):
    level = 2
    rm = RefinedMesh(macro, level)
    num = fem.P2Numbering(rm)
    assert num.n == (2 * 2 ** level + 1) ** 3
    X = rm.cell_xyz
    kfun = lambda x: 1 + 0.5 * np.sin(2 * np.pi * x[:, 0]) * np.sin(2 * np.pi * x[:, 1]) * \
        np.sin(2 * np.pi * x[:, 2])
    for kf in (None, kfun):
        A = fem.assemble(num.dofs, fem.p2_stiffness(X, kf), num.n)
        assert abs(A - A.T).max() < 1e-13
        assert np.abs(A @ np.ones(num.n)).max() < 1e-12
    A = fem.assemble(num.dofs, fem.p2_stiffness(X), num.n)
    M = fem.assemble(num.dofs, fem.p2_mass(X), num.n)
    one = np.ones(num.n)
    assert np.isclose(one @ M @ one, 1.0, rtol=1e-14)
    # quadratic patch test: (A q)_i = (-Lap q) (M 1)_i at interior DoFs
    x, y, z = num.xyz.T
    q = 0.7 * x * x - 0.2 * y * z + 1.3 * x * z + y
    lap = 1.4
    res = A @ q + lap * (M @ one)
    assert np.abs(res[num.interior]).max() < 1e-12
    # the P2 mass against exact quadratic integrals: int x^2 over the cube = 1/3
    assert np.isclose(one @ (M @ (x * x)), 1 / 3, rtol=1e-13)


def test_p1_divkgrad_reduces_to_laplace_for_constant_k():
    rm = RefinedMesh(sg.kuhn_cube(1), 2)
    X = rm.cell_xyz
    K1 = fem.p1_divkgrad(X, np.full((len(X), 4), 2.5))
    assert np.allclose(K1, 2.5 * fem.p1_stiffness(X), rtol=1e-15)
    kv = np.exp(np.sin(rm.xyz.sum(axis=1)))[rm.cells]
    A = fem.assemble(rm.cells, fem.p1_divkgrad(X, kv), rm.n_vertices)
    assert np.abs(A @ np.ones(rm.n_vertices)).max() < 1e-13
    assert abs(A - A.T).max() < 1e-14


def _rand_tets(seed, count):
    g = np.random.Generator(np.random.PCG64(seed))
    X = g.uniform(-1, 1, size=(count, 4, 3))
    return X


def test_p1_divkgrad_is_the_exact_integral_for_linear_k():
    """k linear: int_T k grad l_i . grad l_j = k(centroid) |T| grad l_i . grad l_j,
    and k(centroid) is the mean of the vertex values.  Checked against a
    degree-7 conical-product quadrature of k at the points (independent of the
    vertex-mean formula)."""
    X = _rand_tets(5, 6)
    a, c = 0.7, np.array([0.3, -0.5, 0.9])

    def k(x):
        return a + x @ c

    G, vol = fem.bary_gradients(X)
    bary, w = quadrature.stroud_conical(4)
    pts = np.einsum("qi,tid->tqd", bary, X)
    kint = vol * np.einsum("q,tq->t", w, k(pts.reshape(-1, 3)).reshape(pts.shape[:2]))
    ref = kint[:, None, None] * np.einsum("tid,tjd->tij", G, G)
    kv = k(X.reshape(-1, 3)).reshape(6, 4)
    assert np.allclose(fem.p1_divkgrad(X, kv), ref, rtol=1e-12, atol=1e-14)


def test_p2_stiffness_with_linear_k_matches_an_independent_rule():
    """k linear makes k grad phi_a . grad phi_b a cubic: the 14-point rule
    (degree 5) and a conical-product rule (degree 7) integrate it exactly."""
    X = _rand_tets(6, 4)
    c = np.array([0.4, 1.1, -0.6])

    def k(x):
        return 1.5 + x @ c

    K14 = fem.p2_stiffness(X, k)
    K7 = fem.p2_stiffness(X, k, rule=quadrature.stroud_conical(4))
    assert np.allclose(K14, K7, rtol=1e-12, atol=1e-13)
    # exact integral by monomials: k = sum_m k_m lam_m, grad phi as lam-polynomial terms
    G, vol = fem.bary_gradients(X)

    def e(*idx):
        a = [0, 0, 0, 0]
        for i in idx:
            a[i] += 1
        return tuple(a)

    for t in range(len(X)):
        kv = k(X[t])
        terms = [[(4.0, e(i), G[t, i]), (-1.0, e(), G[t, i])] for i in range(4)]
        terms += [[(4.0, e(i), G[t, j]), (4.0, e(j), G[t, i])] for i, j in fem.P2_EDGES]
        Kex = np.zeros((10, 10))
        for a_ in range(10):
            for b_ in range(10):
                acc = 0.0
                for ca, ea, ga in terms[a_]:
                    for cb, eb, gb in terms[b_]:
                        for m in range(4):
                            al = tuple(x + y + (1 if i == m else 0) for i, (x, y) in enumerate(zip(ea, eb)))
                            acc += kv[m] * ca * cb * (ga @ gb) * quadrature.exact_monomial(al)
                Kex[a_, b_] = vol[t] * acc
        assert np.allclose(K14[t], Kex, rtol=1e-12, atol=1e-13)
    # and a coefficient-free check: k = 1 + 0 x gives the plain stiffness
    assert np.allclose(fem.p2_stiffness(X, lambda x: np.ones(len(x))), fem.p2_stiffness(X),
                       rtol=1e-14, atol=1e-14)
