"""Argument checks of the Python binding that need no GPU.  The kernels
index the full stored length of every vector they are given and read every
vector in the dtype of the first, so the binding refuses a vector that is
shorter than the level's stored length or has another dtype before the call
reaches the library; the network calls check their [n, 16] samples and n
targets the same way.  Stand-in tensors (dtype, device flag, length) and a
hierarchy whose sizes are set by hand stand in for CUDA objects here."""
import pytest

torch = pytest.importorskip("torch")

import paper_2308_01792_gb300 as hg


class FakeTensor:
    def __init__(self, n, dtype=torch.float64, cuda=True, contiguous=True):
        self.n, self.dtype, self.is_cuda, self._c = n, dtype, cuda, contiguous

    def is_contiguous(self):
        return self._c

    def numel(self):
        return self.n

    def data_ptr(self):
        return 256


def _hier(sizes):
    H = hg.Hierarchy.__new__(hg.Hierarchy)
    H._h, H.lmin, H.lmax, H._n_stored = None, 1, 3, {}
    H.size = lambda level, space=hg.HG_SPACE_P1: (sizes[(level, space)], 0, 0, 0)
    return H


def test_vectors_shorter_than_the_level_or_of_another_dtype_are_refused():
    H = _hier({(3, hg.HG_SPACE_P1): 1000, (2, hg.HG_SPACE_P1): 200})
    H._vec(3, hg.HG_SPACE_P1, torch.float64, FakeTensor(1000), FakeTensor(1024))
    with pytest.raises(ValueError, match="need 1000"):
        H._vec(3, hg.HG_SPACE_P1, torch.float64, FakeTensor(1000), FakeTensor(999))
    with pytest.raises(TypeError):
        H._vec(3, hg.HG_SPACE_P1, torch.float64, FakeTensor(1000, torch.float32))
    with pytest.raises(ValueError, match="contiguous CUDA"):
        H._vec(3, hg.HG_SPACE_P1, torch.float64, FakeTensor(1000, cuda=False))
    with pytest.raises(ValueError, match="contiguous CUDA"):
        H._vec(3, hg.HG_SPACE_P1, torch.float64, FakeTensor(1000, contiguous=False))
    # restriction: the coarse vector is checked against the coarser level
    with pytest.raises(ValueError, match="need 200"):
        H.restrict(3, FakeTensor(1000), FakeTensor(199))
    with pytest.raises(TypeError):
        H.prolong_add(3, FakeTensor(200, torch.float32), FakeTensor(1000))


def test_operator_and_multigrid_calls_check_their_vectors_first():
    P1, P2 = hg.HG_SPACE_P1, hg.HG_SPACE_P2
    H = _hier({(3, P1): 1000, (2, P2): 900, (1, P2): 150, (2, P1): 200})
    op = hg.Operator.__new__(hg.Operator)
    op._h, op.hier, op.kind, op.space, op.lmax = None, H, hg.HG_OP_P1_LAPLACE, P1, 3
    with pytest.raises(ValueError):
        op.apply(3, FakeTensor(1000), FakeTensor(10))
    with pytest.raises(TypeError):
        op.residual(3, FakeTensor(1000), FakeTensor(1000, torch.float32), FakeTensor(1000))
    with pytest.raises(ValueError):
        op.jacobi(3, FakeTensor(1000), FakeTensor(1000), FakeTensor(5))
    n1 = hg.Operator.__new__(hg.Operator)
    n1._h, n1.hier, n1.kind, n1.space, n1.lmax = None, H, hg.HG_OP_N1_CURLCURL, P2, 2
    with pytest.raises(ValueError, match="need 150"):
        n1.n1_prolong_add(2, FakeTensor(149), FakeTensor(900))
    with pytest.raises(ValueError, match="need 900"):
        n1.n1_gradient(2, FakeTensor(200), FakeTensor(899))
    with pytest.raises(ValueError, match="need 200"):
        n1.n1_gradient_t(2, FakeTensor(900), FakeTensor(10))
    G = hg.GMG.__new__(hg.GMG)
    G._h, G.op = None, op
    with pytest.raises(TypeError):                      # solves take FP64 vectors
        G.solve(FakeTensor(1000, torch.float32), FakeTensor(1000, torch.float32))
    with pytest.raises(ValueError):                     # on the operator's finest level
        G.solve(FakeTensor(200), FakeTensor(200))
    with pytest.raises(ValueError):
        G.vcycle(3, FakeTensor(1000), FakeTensor(999))


class FakeRows(FakeTensor):
    def __init__(self, shape, dtype, **kw):
        super().__init__(shape[0] * (shape[1] if len(shape) > 1 else 1), dtype, **kw)
        self.shape = shape

    def dim(self):
        return len(self.shape)


def test_network_calls_check_samples_and_targets():
    net = hg.MLP.__new__(hg.MLP)
    net._h = None
    with pytest.raises(ValueError, match=r"\[n, 16\]"):
        net.forward(FakeRows((100, 15), torch.float32))
    with pytest.raises(ValueError, match=r"\[n, 16\]"):
        net.forward(FakeRows((100, 16), torch.bfloat16))
    with pytest.raises(ValueError, match="need 100"):
        net.forward(FakeRows((100, 16), torch.float32), out=FakeTensor(99, torch.float32))
    with pytest.raises(ValueError, match=r"\[n, 16\]"):
        net.grad(FakeRows((100, 16), torch.float32), FakeTensor(100, torch.float32))
    with pytest.raises(TypeError):
        net.grad(FakeRows((100, 16), torch.bfloat16), FakeTensor(100, torch.float64))
    with pytest.raises(ValueError, match="need 100"):
        net.train(FakeRows((100, 16), torch.bfloat16), FakeTensor(50, torch.float32), 1, 10, 1e-3)


def test_function_calls_check_their_buffers_first():
    """Functions: element type at creation, the bound tensor's dtype, and the
    host buffer of a canonical copy (contiguous host float32/float64 memory of
    exactly the level's unique DoF count) are checked before the library is
    called."""
    import numpy as np
    H = hg.Hierarchy.__new__(hg.Hierarchy)
    H._h, H.lmin, H.lmax, H._n_stored = None, 1, 3, {}
    H.size = lambda level, space=hg.HG_SPACE_P1: (1024, 729, 0, 0)
    with pytest.raises(TypeError, match="float32 or float64"):
        hg.Function(H, torch.bfloat16)
    f = hg.Function.__new__(hg.Function)
    f._h, f.hier, f.space, f.dtype, f._t = None, H, hg.HG_SPACE_P1, torch.float64, {}
    with pytest.raises(TypeError):
        f.bind(3, FakeTensor(1024, torch.float32))
    with pytest.raises(ValueError, match="729"):
        f.copy_from_host(3, np.zeros(728))
    with pytest.raises(ValueError):
        f.copy_to_host(3, np.zeros(729, dtype=np.int64))
    with pytest.raises(ValueError):
        f.copy_to_host(3, np.zeros(1458)[::2])                  # not contiguous
    with pytest.raises(ValueError, match="host tensor"):
        f.copy_from_host(3, FakeTensor(729))                    # device memory
    with pytest.raises(ValueError, match="host tensor"):
        f.copy_from_host(3, FakeTensor(729, cuda=False, contiguous=False))
