"""hg_dot_noalloc: the dot product for callers that cannot allocate device memory.

Callers such as code running inside a device memory pool or arena, or code
that must avoid the implicit synchronisation of cudaMalloc/cudaFree, get the
same deterministic FP64 dot as hg_dot without any allocation: the partial sums
live in one fixed device array of the library.  This file runs last so that a
failure here does not hide failures elsewhere; it passes alone or after the
rest of the suite."""
import numpy as np
import pytest

import synthgen as sg

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

import paper_2308_01792_gb300 as hg

TOL = 1e-12   # relative, as for the other FP64 reductions


@pytest.mark.parametrize("dtype", [torch.float64, torch.float32])
@pytest.mark.parametrize("macro,level", [(sg.kuhn_cube(2), 6), (sg.reference_tet(), 5),
                                         (sg.kuhn_cube(1), 1)])
def test_noalloc_dot_matches_hg_dot_twice(macro, level, dtype):
    H = hg.Hierarchy(hg.Mesh(macro.xyz, macro.cells), level, level)
    _, nu, _, _ = H.size(level)
    x = H.from_canonical(level, torch.tensor(sg.uniform_vector(21, nu), dtype=dtype,
                                             device="cuda"))
    y = H.from_canonical(level, torch.tensor(sg.uniform_vector(22, nu), dtype=dtype,
                                             device="cuda"))
    # the canonical vectors as the GPU holds them (rounded to dtype), in FP64
    a = torch.tensor(sg.uniform_vector(21, nu), dtype=dtype).double().numpy()
    c = torch.tensor(sg.uniform_vector(22, nu), dtype=dtype).double().numpy()
    _, _, dirich = H.canonical_info(level)
    inner = ~np.asarray(dirich, dtype=bool)
    out = torch.full((1,), float("nan"), dtype=torch.float64, device="cuda")
    for mask in (hg.HG_MASK_INNER, hg.HG_MASK_ALL):
        ref = H.dot(level, x, y, mask=mask)
        keep = inner if mask == hg.HG_MASK_INNER else np.ones(nu, dtype=bool)
        exact = a[keep] @ c[keep]               # each unique DoF once (NumPy)
        bound = TOL * np.abs(a * c).sum()
        for _ in range(2):                      # two calls in a row share the array
            out.fill_(float("nan"))
            H.dot_noalloc(level, x, y, out, mask=mask)
            got = out.item()
            assert abs(got - ref) <= TOL * max(abs(ref), 1.0), (mask, got, ref)
            assert abs(got - exact) <= bound, (mask, got, exact)


def test_noalloc_dot_rejects_levels_beyond_its_scratch():
    macro = sg.kuhn_cube(3)                    # 162 cells x 2145 rows at level 6 > 131072
    H = hg.Hierarchy(hg.Mesh(macro.xyz, macro.cells), 6, 6)
    x = H.zeros(6, torch.float64)
    out = torch.zeros(1, dtype=torch.float64, device="cuda")
    with pytest.raises(hg.HGError) as e:
        H.dot_noalloc(6, x, x, out)
    assert e.value.code == -1                   # HG_ERR_INVALID_ARG
    assert "at most 131072 rows" in str(e.value)
