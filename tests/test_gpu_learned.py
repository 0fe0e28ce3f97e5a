"""GPU checks of the learned smoother: BF16 tensor-core forward and gradient
against the FP64 oracle, training, the smoothing step, and what the trained
network gains in multigrid over the plain smoother."""
import time

import numpy as np
import pytest

import synthgen as sg
from oracle import mlp as om

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

import paper_2308_01792_gb300 as hg
from paper_2308_01792_gb300 import learned


def _flat(W1, W2, w3):
    return np.concatenate([W1.ravel(), W2.ravel(), w3]).astype(np.float32)


def _oracle_bf16_forward(W1, W2, w3, X):
    """Oracle forward with the kernels' roundings: bf16 inputs, weights and h1."""
    Xb = om.bf16(X)
    z1 = Xb @ om.bf16(W1.astype(np.float32)).T
    h1 = om.bf16(np.maximum(z1, 0))
    z2 = h1 @ om.bf16(W2.astype(np.float32)).T
    return np.maximum(z2, 0) @ w3.astype(np.float32).astype(np.float64)


def test_forward_matches_oracle():
    W1, W2, w3 = om.init_weights(3)
    X = np.random.default_rng(0).normal(size=(1000, 16))
    X[:, 15] = 0
    net = hg.MLP(_flat(W1, W2, w3))
    got = net.forward(torch.tensor(X, dtype=torch.float32, device="cuda")).cpu().double().numpy()
    ref = _oracle_bf16_forward(W1, W2, w3, X.astype(np.float32))
    assert np.abs(got - ref).max() <= 1e-4 * np.abs(ref).max()
    # against the exact FP64 network: within bf16 precision
    exact, _ = om.forward(W1, W2, w3, X)
    assert np.abs(got - exact).max() <= 3e-2 * np.abs(exact).max()


def test_gradient_matches_oracle():
    W1, W2, w3 = om.init_weights(4)
    rng = np.random.default_rng(1)
    X = rng.normal(size=(4096, 16))
    X[:, 15] = 0
    t = rng.normal(size=4096)
    Xb = torch.tensor(X, dtype=torch.bfloat16, device="cuda")
    net = hg.MLP(_flat(W1, W2, w3))
    loss, g = net.grad(Xb, torch.tensor(t, dtype=torch.float32, device="cuda"))
    Xr = Xb.float().cpu().double().numpy()       # the bf16 samples the kernel sees
    L, dW1, dW2, dw3 = om.loss_and_grad(om.bf16(W1.astype(np.float32)),
                                        om.bf16(W2.astype(np.float32)),
                                        w3.astype(np.float32).astype(np.float64), Xr, t)
    ref = np.concatenate([dW1.ravel(), dW2.ravel(), dw3])
    assert abs(loss - L) <= 1e-3 * L
    assert np.linalg.norm(g - ref) <= 3e-2 * np.linalg.norm(ref)
    for a, b in ((g[:512], dW1), (g[512:1536], dW2), (g[1536:], dw3)):
        assert np.linalg.norm(a - b.ravel()) <= 5e-2 * np.linalg.norm(b)


def test_training_fits_a_teacher_network():
    rng = np.random.default_rng(2)
    X = rng.normal(size=(65536, 16))
    X[:, 15] = 0
    Xb = torch.tensor(X, dtype=torch.bfloat16, device="cuda")
    T1, T2, t3 = om.init_weights(20)
    t, _ = om.forward(T1, T2, t3, Xb.float().cpu().double().numpy())
    tt = torch.tensor(t, dtype=torch.float32, device="cuda")
    net, loss = learned.train(Xb, tt, steps=0, seed=5)
    l0, _ = net.grad(Xb, tt)
    loss = net.train(Xb, tt, steps=600, batch=8192, lr=3e-3)
    assert loss < 0.2 * l0, (l0, loss)


def _cube_problem(m=2, lmin=1, level=4, seed=1000):
    macro = sg.kuhn_cube(m)
    H = hg.Hierarchy(hg.Mesh(macro.xyz, macro.cells), lmin, level)
    _, xyz, dirich = H.canonical_info(level)
    op = hg.Operator(H, hg.HG_OP_P1_DIVKGRAD, coeff=learned.lognormal_coefficient(xyz, seed))
    return macro, H, op, xyz, dirich


def test_zero_network_step_is_jacobi():
    macro, H, op, xyz, dirich = _cube_problem()
    L = H.lmax
    G = hg.GMG(op)
    G.set_learned(hg.MLP())                      # zero weights: N = 0
    bc = sg.uniform_vector(3, len(xyz))
    bc[dirich] = 0
    b = H.from_canonical(L, torch.tensor(bc, dtype=torch.float32, device="cuda"))
    x1 = H.zeros(L, torch.float32)
    G.vcycle(L, x1, b)
    G.set_learned(None)
    x2 = H.zeros(L, torch.float32)
    G.vcycle(L, x2, b)
    a = H.to_canonical(L, x1).cpu().double().numpy()
    c = H.to_canonical(L, x2).cpu().double().numpy()
    assert np.abs(a - c).max() <= 1e-5 * np.abs(c).max()


def test_learned_smoother_gain_over_plain():
    """Train on white-noise error pairs of fields of seeds 1..24 (level 4 of the
    4x4x4 Kuhn cube), then solve a held-out field (seed 1000) at level 5 to
    1e-8 with FP32 V-cycles in FP64 refinement, with and without the network."""
    macro = sg.kuhn_cube(4)
    X, t, npairs = learned.make_noise_pairs(macro, 0, 4, range(1, 25), draws=4, stride=2)
    net, loss = learned.train(X, t, steps=3000, batch=65536, lr=1e-3)
    zero_loss = hg.MLP().grad(X, t)[0]
    assert loss < 0.5 * zero_loss
    H = hg.Hierarchy(hg.Mesh(macro.xyz, macro.cells), 0, 5)
    _, xyz, dirich = H.canonical_info(5)
    op = hg.Operator(H, hg.HG_OP_P1_DIVKGRAD, coeff=learned.lognormal_coefficient(xyz, 1000))
    bc = sg.uniform_vector(5, len(xyz))
    bc[dirich] = 0
    b = H.from_canonical(5, torch.tensor(bc, device="cuda"))
    res = {}
    for name, use in (("plain", False), ("learned", True)):
        G = hg.GMG(op)
        G.set_learned(net if use else None)
        x = H.zeros(5, torch.float64)
        G.solve(x, b, tol=1e-8, max_iter=100, precision=hg.HG_PREC_MIXED)   # warm-up
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        it, rel = G.solve(x, b, tol=1e-8, max_iter=100, precision=hg.HG_PREC_MIXED)
        torch.cuda.synchronize()
        res[name] = (it, rel, time.perf_counter() - t0, G.learned_fallbacks() if use else 0)
    print("learned-smoother gain:", npairs, "pairs,", len(t), "samples, loss", loss, res)
    assert res["learned"][1] <= 1e-8 and res["plain"][1] <= 1e-8
    # what the network gains: strictly fewer refinement steps than the plain smoother
    assert res["learned"][0] < res["plain"][0], res


# ---------------------------------------------------------------------------
# the smoothing step and the training samples against the oracle's restatement
# (oracle/learned.py), on a mesh whose cells list their vertices in permuted
# order, so that every cell gathers its features in a different lattice frame

def _perm_problem(L=4):
    from oracle import fem
    from oracle.mesh import RefinedMesh
    macro = sg.permuted_cells(sg.kuhn_cube(1), 3)
    H = hg.Hierarchy(hg.Mesh(macro.xyz, macro.cells), L - 1, L)
    _, xyz, dirich = H.canonical_info(L)
    kfun = lambda p: learned.lognormal_coefficient(p, 1000)
    op = hg.Operator(H, hg.HG_OP_P1_DIVKGRAD, coeff=kfun(xyz))
    rm = RefinedMesh(macro, L)
    kv = kfun(rm.xyz)[rm.cells]
    A = fem.assemble(rm.cells, fem.p1_divkgrad(rm.cell_xyz, kv), rm.n_vertices)
    return macro, H, op, rm, A.diagonal().copy(), dirich


def _gpu_residual(H, op, L, xc, bc):
    x = H.from_canonical(L, torch.tensor(xc, dtype=torch.float32, device="cuda"))
    b = H.from_canonical(L, torch.tensor(bc, dtype=torch.float32, device="cuda"))
    r = H.zeros(L, torch.float32)
    op.residual(L, x, b, r)
    return x, r, H.to_canonical(L, r).cpu().double().numpy()


def test_learned_step_matches_oracle():
    from oracle import learned as ol
    L = 4
    macro, H, op, rm, D, dirich = _perm_problem(L)
    xc = sg.uniform_vector(11, rm.n_vertices)
    bc = sg.uniform_vector(12, rm.n_vertices)
    xc[dirich] = 0
    bc[dirich] = 0
    x, r, rc = _gpu_residual(H, op, L, xc, bc)
    W1, W2, w3 = om.init_weights(9, scale=2.0)
    net = hg.MLP(_flat(W1, W2, w3))
    out = H.zeros(L, torch.float32)
    hg.learned_step(op, net, L, x, r, out, 0.6)
    got = H.to_canonical(L, out).cpu().double().numpy()
    x32 = xc.astype(np.float32).astype(np.float64)
    ref = ol.learned_step(macro, rm, x32, rc, D, W1, W2, w3, 0.6, forward=om.forward_bf16)
    corr = ref - ol.learned_step(macro, rm, x32, rc, D, np.zeros_like(W1), np.zeros_like(W2),
                                 np.zeros_like(w3), 0.6)
    assert np.abs(corr).max() > 0.05 * np.abs(ref).max()        # the network matters here
    # FP32 step, bf16 features (a feature may round to the other neighbour of
    # its bf16 interval when s differs in the last FP32 bits)
    assert np.abs(got - ref).max() <= 1e-5 * np.abs(ref).max() + 2e-2 * np.abs(corr).max()
    assert np.array_equal(got[dirich], x32[dirich])


@pytest.mark.parametrize("d", [0, 1, 4, 7, 10, 11, 13, 14])
def test_learned_step_gathers_in_each_cells_frame(d):
    """A network returning max(F_d, 0), with x = 0 and omega = 0: the step is
    bf16(max(s, 0)) at the neighbour in local direction d of every
    cell-interior vertex, 0 elsewhere."""
    from oracle import learned as ol
    L = 4
    macro, H, op, rm, D, dirich = _perm_problem(L)
    bc = sg.uniform_vector(13, rm.n_vertices)
    bc[dirich] = 0
    x, r, rc = _gpu_residual(H, op, L, np.zeros(rm.n_vertices), bc)
    W1 = np.zeros((32, 16))
    W1[0, d] = 1.0
    W2 = np.zeros((32, 32))
    W2[0, 0] = 1.0
    w3 = np.zeros(32)
    w3[0] = 1.0
    net = hg.MLP(_flat(W1, W2, w3))
    out = H.zeros(L, torch.float32)
    hg.learned_step(op, net, L, x, r, out, 0.0)
    got = H.to_canonical(L, out).cpu().double().numpy()
    ref = ol.learned_step(macro, rm, np.zeros(rm.n_vertices), rc, D, W1, W2, w3, 0.0,
                          forward=om.forward_bf16)
    assert np.count_nonzero(ref) > 0.2 * rm.n_vertices / 8
    assert np.allclose(got, ref, rtol=2 ** -7, atol=0)


def test_learned_samples_match_oracle():
    from oracle import learned as ol
    L = 4
    macro, H, op, rm, D, dirich = _perm_problem(L)
    xc = sg.uniform_vector(14, rm.n_vertices)
    bc = sg.uniform_vector(15, rm.n_vertices)
    xs = sg.uniform_vector(16, rm.n_vertices)
    for v in (xc, bc, xs):
        v[dirich] = 0
    x, r, rc = _gpu_residual(H, op, L, xc, bc)
    xstar = H.from_canonical(L, torch.tensor(xs, dtype=torch.float32, device="cuda"))
    for stride, offset in ((1, 0), (3, 1)):
        X, t = hg.learn_samples(op, L, r, xstar, x, 0.5, stride, offset)
        Xr, tr = ol.learned_samples(macro, rm, rc, D, xs.astype(np.float32).astype(np.float64),
                                    xc.astype(np.float32).astype(np.float64), 0.5, stride, offset)
        Xg = X.float().cpu().double().numpy()
        tg = t.cpu().double().numpy()
        assert Xg.shape == Xr.shape
        assert np.abs(Xg - Xr).max() <= 2 ** -8 * 1.01         # bf16 features of unit vectors
        assert np.abs(tg - tr).max() <= 1e-4 * np.abs(tr).max()
