"""The tests of test_gpu_p1.py again with the column-march constant-stencil
kernel forced for every P1 constant-stencil operation (hg_set_p1_kernel), so
that it meets the same oracle parity bars as the plane-window kernel."""
import pytest

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

import paper_2308_01792_gb300 as hg

from test_gpu_p1 import *  # noqa: F401,F403  (the same tests, collected here again)


@pytest.fixture(scope="module", autouse=True)
def _march_kernel():
    hg.set_p1_kernel(hg.HG_P1_KERNEL_MARCH)
    yield
    hg.set_p1_kernel(hg.HG_P1_KERNEL_AUTO)


@pytest.mark.parametrize("pattern_mesh", ["cube", "perm"])
@pytest.mark.parametrize("dtype", [torch.float32, torch.float64])
def test_march_equals_plane_windows_bit_for_bit(pattern_mesh, dtype):
    """Both kernels form the interior sums in the same order and share the
    interface items, so their results have the same bits (seven-point cube
    stencils and general 15-point stencils of a permuted mesh)."""
    import synthgen as sg
    macro = sg.kuhn_cube(2) if pattern_mesh == "cube" else sg.permuted_cells(sg.kuhn_cube(2), 7)
    H = hg.Hierarchy(hg.Mesh(macro.xyz, macro.cells), 3, 5)
    op = hg.Operator(H)
    for L in (3, 4, 5):
        nu = H.size(L)[1]
        x = H.from_canonical(L, torch.tensor(sg.uniform_vector(90 + L, nu), dtype=dtype,
                                             device="cuda"))
        b = H.from_canonical(L, torch.tensor(sg.uniform_vector(95 + L, nu), dtype=dtype,
                                             device="cuda"))
        outs = {}
        for mode in (hg.HG_P1_KERNEL_WINDOWS, hg.HG_P1_KERNEL_MARCH):
            hg.set_p1_kernel(mode)
            y, r, xj = H.zeros(L, dtype), H.zeros(L, dtype), H.zeros(L, dtype)
            op.apply(L, x, y, mask=hg.HG_MASK_ALL)
            op.residual(L, x, b, r)
            op.jacobi(L, x, b, xj)
            outs[mode] = (y, r, xj)
        hg.set_p1_kernel(hg.HG_P1_KERNEL_MARCH)
        for a, c in zip(outs[hg.HG_P1_KERNEL_WINDOWS], outs[hg.HG_P1_KERNEL_MARCH]):
            assert torch.equal(a, c), L
