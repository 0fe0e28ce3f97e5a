"""Batched persistent solves of many independent P1 Poisson problems of uneven
size (unit cubes of 6 m^3 macro-tetrahedra, level drawn per problem, seeded
uniform right-hand sides), through the C ABI.

Checked: every problem reaches the tolerance; each batched solution equals
the one-at-a-time mixed-precision solve of the same problem (same step count,
same iterate up to the rounding of the per-problem norms); graph replay is
bit-identical to plain launches; the autotuned kernel variant changes
nothing beyond rounding; the batched solutions satisfy the oracle's assembled
systems; and bad batches are rejected on the host."""
import numpy as np
import pytest

import synthgen as sg
from oracle import gmg as og

from helpers import rel_err

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

import paper_2308_01792_gb300 as hg

TOL = 1e-8


def _problems(draw, seed0):
    """Shared hierarchy/operator per (m, level); one GMG per problem."""
    shared = {}
    Gs, xs, bs, keys = [], [], [], []
    for p, (m, L) in enumerate(draw):
        if (m, L) not in shared:
            macro = sg.kuhn_cube(m)
            H = hg.Hierarchy(hg.Mesh(macro.xyz, macro.cells), 0, L)
            op = hg.Operator(H)
            shared[(m, L)] = [H, op, hg.GMG(op), False]
        H, op, G0, used = shared[(m, L)]
        G = G0.clone() if used else G0
        shared[(m, L)][3] = True
        _, xyz, dirich = H.canonical_info(L)
        bc = sg.uniform_vector(seed0 + p, len(xyz))
        bc[dirich] = 0.0
        Gs.append(G)
        bs.append(H.from_canonical(L, torch.tensor(bc, device="cuda")))
        xs.append(H.zeros(L, torch.float64))
        keys.append((m, L))
    return shared, Gs, xs, bs, keys


@pytest.fixture(scope="module")
def batch():
    # the first 16 problems of the 512-problem draw, levels capped at 5
    draw = [(m, min(L, 5)) for m, L in sg.batched_problem_draw(42, 512)[:16]]
    return (draw,) + _problems(draw, 100)


def test_batch_converges_and_equals_single_solves(batch):
    draw, shared, Gs, xs, bs, keys = batch
    B = hg.Batch(Gs, xs, bs, graph=True, autotune=True)
    it, rel = B.solve(tol=TOL, max_iter=60)
    rows, gf, us = B.tuning()
    print("batch:", draw, "iters", it.tolist(), "tuned rows", rows, "grid factor", gf, us, "us")
    assert rows in (0, 1, 2) and gf in (1, 2, 4) and us > 0
    assert np.all(rel <= TOL) and np.all(it > 0)
    for p, G in enumerate(Gs):
        H = shared[keys[p]][0]
        L = keys[p][1]
        x1 = H.zeros(L, torch.float64)
        it1, rel1 = G.solve(x1, bs[p], tol=TOL, max_iter=60, precision=hg.HG_PREC_MIXED)
        assert it[p] == it1, p
        assert rel[p] == pytest.approx(rel1, rel=1e-9), p
        assert rel_err(xs[p].cpu().numpy(), x1.cpu().numpy()) <= 1e-11, p


def test_graph_replay_bit_identical_and_variant_invariant(batch):
    draw, shared, Gs, xs, bs, keys = batch
    xg = [torch.zeros_like(v) for v in xs]
    xp = [torch.zeros_like(v) for v in xs]
    xt = [torch.zeros_like(v) for v in xs]
    itg, _ = hg.Batch(Gs, xg, bs, graph=True, autotune=False).solve(tol=TOL, max_iter=60)
    itp, _ = hg.Batch(Gs, xp, bs, graph=False, autotune=False).solve(tol=TOL, max_iter=60)
    itt, _ = hg.Batch(Gs, xt, bs, graph=True, autotune=True).solve(tol=TOL, max_iter=60)
    assert np.array_equal(itg, itp) and np.array_equal(itg, itt)
    for p in range(len(xs)):
        assert torch.equal(xg[p], xp[p]), p
        assert rel_err(xt[p].cpu().numpy(), xg[p].cpu().numpy()) <= 1e-12, p


def test_batch_solutions_satisfy_oracle_systems():
    """Small uneven batch; residuals measured with the oracle's assembled
    matrices (FP64, canonical order)."""
    draw = [(1, 3), (2, 3), (1, 4), (2, 2), (3, 3), (1, 2)]
    shared, Gs, xs, bs, keys = _problems(draw, 500)
    it, rel = hg.Batch(Gs, xs, bs).solve(tol=TOL, max_iter=60)
    oracle_levels = {}
    for p, (m, L) in enumerate(draw):
        if (m, L) not in oracle_levels:
            oracle_levels[(m, L)] = og.Level(sg.kuhn_cube(m), L)
        lev = oracle_levels[(m, L)]
        H = shared[(m, L)][0]
        xg = H.to_canonical(L, xs[p]).cpu().numpy()
        bg = H.to_canonical(L, bs[p]).cpu().numpy()
        assert np.all(xg[lev.boundary] == 0)
        bi = bg[lev.interior]
        ro = np.linalg.norm(bi - lev.A @ xg[lev.interior]) / np.linalg.norm(bi)
        assert ro <= TOL * 1.01, (p, ro, rel[p])


def test_converged_problem_keeps_its_iterate():
    """A zero right-hand side converges at step 0 and stays exactly zero while
    its batch mates iterate."""
    draw = [(1, 4), (2, 4)]
    shared, Gs, xs, bs, keys = _problems(draw, 700)
    bs[0].zero_()
    it, rel = hg.Batch(Gs, xs, bs).solve(tol=TOL, max_iter=60)
    assert it[0] == 0 and rel[0] == 0.0 and it[1] > 0
    assert torch.count_nonzero(xs[0]) == 0


def test_not_converged_and_bad_batches():
    draw = [(1, 3), (1, 4)]
    shared, Gs, xs, bs, keys = _problems(draw, 800)
    B = hg.Batch(Gs, xs, bs)
    with pytest.raises(hg.HGError) as e:
        B.solve(tol=1e-14, max_iter=2)
    assert e.value.code == -5
    it, rel = B.solve(tol=1e-14, max_iter=2, check=False)
    assert np.all(it == 2) and np.all(rel > 1e-14)
    with pytest.raises(hg.HGError):          # the same problem twice
        hg.Batch([Gs[0], Gs[0]], [xs[0], xs[1]], [bs[0], bs[1]])
    with pytest.raises(ValueError):          # FP32 vectors
        hg.Batch(Gs, [x.float() for x in xs], bs)
    H, op, G0, _ = shared[(1, 3)]
    kop = hg.Operator(H, hg.HG_OP_P1_DIVKGRAD, coeff=np.ones(H.canonical_info(3)[1].shape[0]))
    with pytest.raises(hg.HGError):          # variable coefficients are not batched
        hg.Batch([hg.GMG(kop)], [xs[0]], [bs[0]])
