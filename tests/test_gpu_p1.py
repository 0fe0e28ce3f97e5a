"""GPU parity of the P1 path against the oracle (through the C ABI).

Index functions and ghost-layer maps: bit-exact.  Operator applications:
max-norm relative error <= 1e-12 (FP64) / 1e-5 (FP32), the tolerances of the
hot-path contract.  Sizes span several warps per x-line (ragged tails) and
several macro cells; the full cube at level 7 is covered by closed-form
properties (7-point identity, zero row sums, symmetry)."""
import numpy as np
import pytest

import synthgen as sg
from oracle import fem
from oracle import indexing as ix
from oracle import gmg as og
from oracle.mesh import RefinedMesh

from helpers import oracle_stored_to_canonical, rel_err

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

import paper_2308_01792_gb300 as hg

TOL = {torch.float64: 1e-12, torch.float32: 1e-5}

# the permuted meshes list each cell's vertices in a seeded order, so local and
# global orientations disagree and the refinement's inner diagonals change
CASES = [(sg.reference_tet(), 2, 4), (sg.reference_tet(), 0, 6), (sg.kuhn_cube(1), 0, 5),
         (sg.kuhn_cube(2), 1, 4), (sg.permuted_cells(sg.kuhn_cube(1), 3), 0, 4),
         (sg.permuted_cells(sg.kuhn_cube(2), 7), 1, 3)]
IDS = ["tet_L2-4", "tet_L0-6", "cube1_L0-5", "cube2_L1-4", "cube1perm_L0-4", "cube2perm_L1-3"]


@pytest.fixture(scope="module", params=range(len(CASES)), ids=IDS)
def case(request):
    macro, lmin, lmax = CASES[request.param]
    mesh = hg.Mesh(macro.xyz, macro.cells)
    H = hg.Hierarchy(mesh, lmin, lmax)
    return macro, H


def test_index_enumeration_bit_exact():
    for w in (1, 2, 3, 4, 5, 17, 33, 64, 65, 129, 257):
        n = ix.n_tet(w)
        out = torch.full((n,), -1, dtype=torch.int64, device="cuda")
        hg.index_enumerate(w, out)
        got = out.cpu().numpy()
        exp = np.empty(n, dtype=np.int64)
        for (i, j, k) in ix.index_set_tet(w):
            exp[ix.tw(w, i, j, k)] = i + (j << 20) + (k << 40)
        assert np.array_equal(got, exp), w


def test_canonical_numbering_bit_exact(case):
    macro, H = case
    for L in range(H.lmin, H.lmax + 1):
        rm = RefinedMesh(macro, L)
        ns, nu, ni, stride = H.size(L)
        assert nu == rm.n_vertices and ni == len(rm.interior)
        s2c, xyz, dirich = H.canonical_info(L)
        assert np.array_equal(s2c, oracle_stored_to_canonical(macro, rm, stride))
        assert np.array_equal(xyz, rm.xyz)
        assert np.array_equal(dirich, rm.boundary)


def test_ghost_layer_map_bit_exact(case):
    macro, H = case
    for L in range(H.lmin, H.lmax + 1):
        rm = RefinedMesh(macro, L)
        ns, nu, ni, stride = H.size(L)
        o = oracle_stored_to_canonical(macro, rm, stride)
        n = 2 ** L
        # oracle: cell-boundary points grouped by global vertex
        groups = {}
        for c in range(len(macro.cells)):
            for (i, j, k) in ix.index_set_tet(n + 1):
                if i == 0 or j == 0 or k == 0 or i + j + k == n:
                    t = ix.tw(n + 1, i, j, k)
                    groups.setdefault(o[c * stride + t], []).append((c, t))
        exp = sorted(tuple(sorted(g)) for g in groups.values())
        rows = H.interface_dump(L).cpu().numpy()
        got = []
        for r in rows:
            nc = r[0]
            cp = [(int(r[1 + 2 * q]), int(r[2 + 2 * q])) for q in range(nc)]
            assert cp == sorted(cp)                 # summed in ascending cell order
            got.append(tuple(cp))
        assert sorted(got) == exp


def _oracle_level(macro, L, kind="laplace"):
    rm = RefinedMesh(macro, L)
    X = rm.cell_xyz
    K = fem.p1_stiffness(X) if kind == "laplace" else fem.p1_mass(X)
    return rm, fem.assemble(rm.cells, K, rm.n_vertices)


@pytest.mark.parametrize("dtype", [torch.float64, torch.float32])
@pytest.mark.parametrize("kind", ["laplace", "mass"])
def test_apply_matches_assembled_oracle(case, dtype, kind):
    macro, H = case
    op = hg.Operator(H, hg.HG_OP_P1_LAPLACE if kind == "laplace" else hg.HG_OP_P1_MASS)
    for L in range(H.lmin, H.lmax + 1):
        rm, A = _oracle_level(macro, L, kind)
        xc = sg.uniform_vector(L, rm.n_vertices)
        # INNER mask: homogeneous Dirichlet values, interior rows
        xi = xc.copy()
        xi[rm.boundary] = 0
        x = H.from_canonical(L, torch.tensor(xi, dtype=dtype, device="cuda"))
        y = H.zeros(L, dtype)
        op.apply(L, x, y)
        yc = H.to_canonical(L, y).cpu().double().numpy()
        ref = A @ xi
        ii = rm.interior
        if len(ii):
            assert rel_err(yc[ii], ref[ii]) <= TOL[dtype], (L, rel_err(yc[ii], ref[ii]))
        assert np.all(yc[rm.boundary] == 0)
        # every stored copy holds the canonical value exactly
        s2c, _, _ = H.canonical_info(L)
        ys = y.cpu().double().numpy()
        valid = s2c >= 0
        assert np.array_equal(ys[valid], yc[s2c[valid]])
        # ALL mask: full Neumann rows with nonzero boundary values
        x = H.from_canonical(L, torch.tensor(xc, dtype=dtype, device="cuda"))
        y = H.zeros(L, dtype)
        op.apply(L, x, y, mask=hg.HG_MASK_ALL)
        yc = H.to_canonical(L, y).cpu().double().numpy()
        assert rel_err(yc, A @ xc) <= TOL[dtype]
        # ADD mode: y += A x
        y0 = sg.uniform_vector(100 + L, rm.n_vertices)
        y = H.from_canonical(L, torch.tensor(y0, dtype=dtype, device="cuda"))
        op.apply(L, x, y, mode=hg.HG_ADD, mask=hg.HG_MASK_ALL)
        yc = H.to_canonical(L, y).cpu().double().numpy()
        assert rel_err(yc, y0 + A @ xc) <= TOL[dtype] * 2


@pytest.mark.parametrize("dtype", [torch.float64, torch.float32])
@pytest.mark.parametrize("mode", ["replace", "add"])
@pytest.mark.parametrize("kind", ["laplace", "mass"])
def test_inner_mask_zeroes_dirichlet_entries(case, dtype, mode, kind):
    """HG_MASK_INNER on a destination that starts NONZERO everywhere: A x
    (REPLACE) or y + A x (ADD) on the other DoFs, exactly 0 at the Dirichlet
    DoFs (homogeneous Dirichlet values), for both modes."""
    macro, H = case
    op = hg.Operator(H, hg.HG_OP_P1_LAPLACE if kind == "laplace" else hg.HG_OP_P1_MASS)
    L = H.lmax
    rm, A = _oracle_level(macro, L, kind)
    xi = sg.uniform_vector(200 + L, rm.n_vertices)
    xi[rm.boundary] = 0
    y0 = sg.uniform_vector(300 + L, rm.n_vertices)
    x = H.from_canonical(L, torch.tensor(xi, dtype=dtype, device="cuda"))
    y = H.from_canonical(L, torch.tensor(y0, dtype=dtype, device="cuda"))
    add = mode == "add"
    op.apply(L, x, y, mode=hg.HG_ADD if add else hg.HG_REPLACE)
    yc = H.to_canonical(L, y).cpu().double().numpy()
    y0r = torch.tensor(y0, dtype=dtype).double().numpy()
    ref = (y0r if add else 0.0) + A @ xi
    ii = rm.interior
    if len(ii):
        assert rel_err(yc[ii], ref[ii]) <= TOL[dtype] * 2
    assert np.all(yc[rm.boundary] == 0)
    s2c, _, _ = H.canonical_info(L)
    ys = y.cpu().double().numpy()
    valid = s2c >= 0
    assert np.array_equal(ys[valid], yc[s2c[valid]])


@pytest.mark.parametrize("dtype", [torch.float64, torch.float32])
def test_residual_and_jacobi_match_oracle(case, dtype):
    macro, H = case
    op = hg.Operator(H)
    L = H.lmax
    rm, A = _oracle_level(macro, L)
    ii = rm.interior
    AII = A[ii][:, ii]
    D = AII.diagonal()
    xc = sg.uniform_vector(1, rm.n_vertices)
    bc = sg.uniform_vector(2, rm.n_vertices)
    xc[rm.boundary] = 0
    bc[rm.boundary] = 0
    x = H.from_canonical(L, torch.tensor(xc, dtype=dtype, device="cuda"))
    b = H.from_canonical(L, torch.tensor(bc, dtype=dtype, device="cuda"))
    r = H.zeros(L, dtype)
    op.residual(L, x, b, r)
    rc = H.to_canonical(L, r).cpu().double().numpy()
    ref = bc[ii] - AII @ xc[ii]
    assert rel_err(rc[ii], ref) <= TOL[dtype] * 4
    assert np.all(rc[rm.boundary] == 0)
    xo = H.zeros(L, dtype)
    op.jacobi(L, x, b, xo, omega=2.0 / 3.0)
    xoc = H.to_canonical(L, xo).cpu().double().numpy()
    ref = og.jacobi(AII, D, xc[ii], bc[ii], 2.0 / 3.0)
    assert rel_err(xoc[ii], ref) <= TOL[dtype] * 4
    assert np.all(xoc[rm.boundary] == 0)


@pytest.mark.parametrize("dtype", [torch.float64, torch.float32])
def test_transfers_match_oracle_prolongation(case, dtype):
    macro, H = case
    if H.lmax == H.lmin:
        pytest.skip("single level")
    Hm = og.Hierarchy(macro, max(H.lmin, H.lmax - 2), H.lmax)
    for L in range(Hm.lmin + 1, Hm.lmax + 1):
        fi, co = Hm.levels[L], Hm.levels[L - 1]
        P = Hm.P[L]
        # prolongation: x_f += P e_c
        ec = sg.uniform_vector(3, co.n)
        ec[co.boundary] = 0
        xf0 = sg.uniform_vector(4, fi.n)
        xf0[fi.boundary] = 0
        e = H.from_canonical(L - 1, torch.tensor(ec, dtype=dtype, device="cuda"))
        x = H.from_canonical(L, torch.tensor(xf0, dtype=dtype, device="cuda"))
        H.prolong_add(L, e, x)
        got = H.to_canonical(L, x).cpu().double().numpy()
        ref = xf0.copy()
        ref[fi.interior] += P @ ec[co.interior]
        assert rel_err(got, ref) <= TOL[dtype]
        # restriction: r_c = P^T r_f
        rf = sg.uniform_vector(5, fi.n)
        rf[fi.boundary] = 0
        r = H.from_canonical(L, torch.tensor(rf, dtype=dtype, device="cuda"))
        rcv = H.zeros(L - 1, dtype)
        H.restrict(L, r, rcv)
        got = H.to_canonical(L - 1, rcv).cpu().double().numpy()
        ref = np.zeros(co.n)
        ref[co.interior] = P.T @ rf[fi.interior]
        assert rel_err(got, ref) <= TOL[dtype] * 2


@pytest.mark.parametrize("dtype", [torch.float64, torch.float32])
def test_dot_counts_each_dof_once(case, dtype):
    macro, H = case
    L = H.lmax
    rm = RefinedMesh(macro, L)
    a = sg.uniform_vector(6, rm.n_vertices)
    c = sg.uniform_vector(7, rm.n_vertices)
    x = H.from_canonical(L, torch.tensor(a, dtype=dtype, device="cuda"))
    y = H.from_canonical(L, torch.tensor(c, dtype=dtype, device="cuda"))
    av = torch.tensor(a, dtype=dtype).double().numpy()
    cv = torch.tensor(c, dtype=dtype).double().numpy()
    full = H.dot(L, x, y, mask=hg.HG_MASK_ALL)
    inner = H.dot(L, x, y)
    assert abs(full - av @ cv) <= 1e-12 * np.abs(av * cv).sum()
    ii = rm.interior
    assert abs(inner - av[ii] @ cv[ii]) <= 1e-12 * np.abs(av * cv).sum()
    assert H.dot(L, x, y) == inner                   # deterministic


def test_full_size_cube_level7_properties():
    """Unit cube, 6 Kuhn cells, level 7 (2 146 689 DoFs): the P1 Laplacian is
    h times the textbook 7-point stencil (closed form), rows sum to zero."""
    macro = sg.kuhn_cube(1)
    H = hg.Hierarchy(hg.Mesh(macro.xyz, macro.cells), 7, 7)
    op = hg.Operator(H)
    N = 128
    h = 1.0 / N
    for dtype in (torch.float64, torch.float32):
        xc = sg.uniform_vector(0, (N + 1) ** 3)
        x3 = xc.reshape(N + 1, N + 1, N + 1).copy()     # [z, y, x]
        x3[0], x3[-1], x3[:, 0], x3[:, -1], x3[:, :, 0], x3[:, :, -1] = 0, 0, 0, 0, 0, 0
        x = H.from_canonical(7, torch.tensor(x3.ravel(), dtype=dtype, device="cuda"))
        y = H.zeros(7, dtype)
        op.apply(7, x, y)
        yc = H.to_canonical(7, y).cpu().double().numpy().reshape(N + 1, N + 1, N + 1)
        ref = np.zeros_like(x3)
        c = x3[1:-1, 1:-1, 1:-1]
        ref[1:-1, 1:-1, 1:-1] = h * (6 * c - x3[:-2, 1:-1, 1:-1] - x3[2:, 1:-1, 1:-1]
                                     - x3[1:-1, :-2, 1:-1] - x3[1:-1, 2:, 1:-1]
                                     - x3[1:-1, 1:-1, :-2] - x3[1:-1, 1:-1, 2:])
        assert rel_err(yc, ref) <= TOL[dtype]
        one = H.from_canonical(7, torch.ones((N + 1) ** 3, dtype=dtype, device="cuda"))
        op.apply(7, one, y, mask=hg.HG_MASK_ALL)
        assert torch.abs(y).max().item() <= 64 * TOL[dtype] * h
