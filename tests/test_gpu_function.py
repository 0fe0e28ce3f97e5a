"""GPU tests of the function layer (Sec. 5.1: a function holds one vector per
level of the hierarchy) through the C ABI: host <-> device copies in
canonical order, the function-handle apply and solve against the oracle.

Copies are value moves (and a round to nearest for a change of element
type), so they are checked bit-exactly; applies to the contract's
tolerances (1e-12 FP64, 1e-5 FP32)."""
import numpy as np
import pytest

import synthgen as sg
from oracle import fem
from oracle.mesh import RefinedMesh

from helpers import oracle_stored_to_canonical, rel_err

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

import paper_2308_01792_gb300 as hg

CASES = [(sg.reference_tet(), 2, 4), (sg.kuhn_cube(2), 1, 4),
         (sg.permuted_cells(sg.kuhn_cube(1), 3), 0, 4)]
IDS = ["tet_L2-4", "cube2_L1-4", "cube1perm_L0-4"]


@pytest.fixture(scope="module", params=range(len(CASES)), ids=IDS)
def case(request):
    macro, lmin, lmax = CASES[request.param]
    H = hg.Hierarchy(hg.Mesh(macro.xyz, macro.cells), lmin, lmax)
    return macro, H


@pytest.mark.parametrize("dtype", [torch.float32, torch.float64])
@pytest.mark.parametrize("host", ["numpy", "pinned"])
def test_copy_from_host_sets_every_stored_copy(case, dtype, host):
    macro, H = case
    f = hg.Function(H, dtype)
    for L in range(H.lmin, H.lmax + 1):
        rm = RefinedMesh(macro, L)
        ns, nu, _, stride = H.size(L)
        c = sg.uniform_vector(3 + L, nu).astype(np.float64 if dtype == torch.float64 else np.float32)
        hb = c if host == "numpy" else torch.from_numpy(c).pin_memory()
        f[L].fill_(7.0)
        f.copy_from_host(L, hb)
        torch.cuda.synchronize()
        got = f[L].cpu().numpy()
        s2c = oracle_stored_to_canonical(macro, rm, stride)
        live = s2c >= 0
        assert np.array_equal(got[live], c[s2c[live]]), L
        assert np.all(got[~live] == 7.0), L                  # padding untouched
        back = np.empty_like(c) if host == "numpy" else torch.empty(nu, dtype=dtype).pin_memory()
        f.copy_to_host(L, back)
        torch.cuda.synchronize()
        back = back if host == "numpy" else back.numpy()
        assert np.array_equal(back, c), L


def test_copy_converts_element_types(case):
    macro, H = case
    L = H.lmax
    nu = H.size(L)[1]
    c = sg.uniform_vector(11, nu) * 1e-3 + 1.0 / 3.0          # values that FP32 must round
    f32 = hg.Function(H, torch.float32, levels=[L])
    f32.copy_from_host(L, c)                                   # FP64 host -> FP32 function
    out32 = np.empty(nu, dtype=np.float32)
    f32.copy_to_host(L, out32)
    torch.cuda.synchronize()
    assert np.array_equal(out32, c.astype(np.float32))
    out64 = np.empty(nu)
    f32.copy_to_host(L, out64)                                 # FP32 function -> FP64 host
    torch.cuda.synchronize()
    assert np.array_equal(out64, c.astype(np.float32).astype(np.float64))


@pytest.mark.parametrize("dtype", [torch.float32, torch.float64])
def test_apply_function_matches_oracle(case, dtype):
    macro, H = case
    op = hg.Operator(H)
    x = hg.Function(H, dtype)
    y = hg.Function(H, dtype)
    s = torch.cuda.Stream()
    for L in range(H.lmin, H.lmax + 1):
        rm = RefinedMesh(macro, L)
        A = fem.assemble(rm.cells, fem.p1_stiffness(rm.cell_xyz), rm.n_vertices)
        nu = rm.n_vertices
        xc = sg.uniform_vector(20 + L, nu)
        xc[rm.boundary] = 0
        x.copy_from_host(L, xc, stream=s)
        op.apply_function(L, x, y, stream=s)
        out = np.empty(nu)
        y.copy_to_host(L, out, stream=s)
        s.synchronize()
        ref = A @ xc.astype(np.float32 if dtype == torch.float32 else np.float64).astype(np.float64)
        ii = rm.interior
        if len(ii):
            assert rel_err(out[ii], ref[ii]) <= (1e-12 if dtype == torch.float64 else 1e-5), L
        assert np.all(out[rm.boundary] == 0.0), L
        # the same as the raw-pointer call on the bound tensors
        y2 = torch.zeros_like(y[L])
        op.apply(L, x[L], y2, stream=s)
        s.synchronize()
        assert torch.equal(y2, y[L])


def test_solve_function_matches_solve():
    macro = sg.kuhn_cube(1)
    H = hg.Hierarchy(hg.Mesh(macro.xyz, macro.cells), 1, 5)
    op = hg.Operator(H)
    G = hg.GMG(op)
    nu = H.size(5)[1]
    _, _, dirich = H.canonical_info(5)
    bc = sg.uniform_vector(9, nu)
    bc[dirich] = 0.0
    b = hg.Function(H, torch.float64, levels=[5])
    x = hg.Function(H, torch.float64, levels=[5])
    b.copy_from_host(5, bc)
    it, rel = G.solve_function(x, b, tol=1e-10, max_iter=50)
    assert rel <= 1e-10
    xr = H.zeros(5, torch.float64)
    it2, rel2 = G.solve(xr, b[5], tol=1e-10, max_iter=50)
    assert (it, rel) == (it2, rel2)
    assert torch.equal(xr, x[5])


def test_function_errors(case):
    macro, H = case
    L = H.lmax
    nu = H.size(L)[1]
    f = hg.Function(H, torch.float64, levels=[L])
    g32 = hg.Function(H, torch.float32, levels=[L])
    op = hg.Operator(H)
    with pytest.raises(ValueError):
        f.copy_from_host(L, np.zeros(nu + 1))                  # wrong length (binding)
    with pytest.raises(hg.HGError):                            # no vector bound on lmin
        f.copy_from_host(H.lmin, np.zeros(H.size(H.lmin)[1]))
    with pytest.raises(hg.HGError):
        op.apply_function(L, f, g32)                           # element types differ
    with pytest.raises(hg.HGError):
        op.apply_function(L, f, f)                             # x and y identical
    p = hg.ctypes.c_void_p()
    hg._call("hg_function_data", f._h, L, hg.ctypes.byref(p))
    assert p.value == f[L].data_ptr()
    with pytest.raises(hg.HGError):                            # level outside the hierarchy
        hg._call("hg_function_copy_canonical", f._h, L + 1, hg.ctypes.c_void_p(1), hg.HG_F64, 1,
                 hg.HG_COPY_TO_HOST, None)
    with pytest.raises(hg.HGError):                            # short buffer
        hg._call("hg_function_bind", f._h, L, hg.ctypes.c_void_p(f[L].data_ptr()), 8)
