"""The tests of test_gpu_cheb_fmg.py again with the column-march constant-stencil
kernel forced for every P1 constant-stencil operation (hg_set_p1_kernel), so
that it meets the same oracle parity bars as the plane-window kernel."""
import pytest

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

import paper_2308_01792_gb300 as hg

from test_gpu_cheb_fmg import *  # noqa: F401,F403  (the same tests, collected here again)


@pytest.fixture(scope="module", autouse=True)
def _march_kernel():
    hg.set_p1_kernel(hg.HG_P1_KERNEL_MARCH)
    yield
    hg.set_p1_kernel(hg.HG_P1_KERNEL_AUTO)
