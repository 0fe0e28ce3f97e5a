"""Distribution of the macro cells over ranks (Sec. 2: primitives distributed
over processes, one ghost-layer exchange per application) on the CPU, with
gloo ranks (world sizes 2 and 3) and no GPU.

The library's partition (hg_partition_cells) and exchange plan
(hg_exchange_plan) are host code.  Each rank stores only its own cells;
the per-copy partial sums are taken from the oracle (the assembled matrix of
each macro cell's own micro-cells), exchanged by gloo point-to-point
messages along the plan, and summed by the plan's recipe.  Checked: every
cross-rank point gets the global row of the assembled operator, and the
plan's order reproduces the single-device order (all copies in ascending
cell id) bit for bit; conjugate gradients run over the ranks (owned-copy dots
and an FP64 all-reduce) reproduce the single-domain iterates."""
import os

import numpy as np
import pytest

import synthgen as sg
from oracle import fem
from oracle.mesh import RefinedMesh

from helpers import oracle_stored_to_canonical

torch = pytest.importorskip("torch")
import torch.distributed as dist
import torch.multiprocessing as mp

import paper_2308_01792_gb300 as hg

MESHES = {"cube2": sg.kuhn_cube(2), "cube2perm": sg.permuted_cells(sg.kuhn_cube(2), 7)}


def _cell_partials(macro, rm, x):
    """partial[c] = A_c x: the P1 Laplacian of macro cell c's micro-cells only."""
    per = 8 ** rm.level
    Ke = fem.p1_stiffness(rm.cell_xyz)
    out = []
    for c in range(len(macro.cells)):
        sl = slice(c * per, (c + 1) * per)
        out.append(fem.assemble(rm.cells[sl], Ke[sl], rm.n_vertices) @ x)
    return out


def _local_partials(macro, rm, part, rank, stride, x):
    """The rank's local stored vector of partials: slot (local cell, t) holds
    the partial of its own cell at that lattice point."""
    s2c = oracle_stored_to_canonical(macro, rm, stride)
    parts = _cell_partials(macro, rm, x)
    mine = np.flatnonzero(part == rank)
    y = np.zeros(len(mine) * stride)
    gids = np.full(len(mine) * stride, -1, dtype=np.int64)
    for lc, c in enumerate(mine):
        g = s2c[c * stride:(c + 1) * stride]
        ok = g >= 0
        y[lc * stride:(lc + 1) * stride][ok] = parts[c][g[ok]]
        gids[lc * stride:(lc + 1) * stride] = g
    return y, gids, parts


@pytest.mark.parametrize("nparts", [1, 2, 3, 5, 8, 48])
def test_partition_is_balanced_and_deterministic(nparts):
    m = MESHES["cube2"]
    M = hg.Mesh(m.xyz, m.cells)
    p = hg.partition_cells(M, nparts)
    assert np.array_equal(p, hg.partition_cells(M, nparts))
    cnt = np.bincount(p, minlength=nparts)
    assert cnt.min() >= 1 and cnt.max() - cnt.min() <= 1, cnt
    with pytest.raises(hg.HGError):
        hg.partition_cells(M, 49)


def test_exchange_plan_refuses_bad_arguments():
    m = MESHES["cube2"]
    M = hg.Mesh(m.xyz, m.cells)
    part = hg.partition_cells(M, 2)
    with pytest.raises(hg.HGError):
        hg.exchange_plan(M, 2, part, 2)                   # rank outside 0..nparts-1
    bad = part.copy()
    bad[5] = -1
    with pytest.raises(hg.HGError, match="outside"):
        hg.exchange_plan(M, 2, bad, 0)                    # a cell without a valid part
    with pytest.raises(hg.HGError, match="level"):
        hg.exchange_plan(M, 10, part, 0)
    one = np.zeros_like(part)
    P = hg.exchange_plan(M, 2, one, 0)                    # one rank: nothing to exchange
    assert len(P["point_start"]) == 1 and len(P["send_idx"]) == 0 and len(P["target_idx"]) == 0


def test_bisection_cuts_across_the_longest_extent():
    """Two parts of the 2x2x2 cube: the cut is a coordinate plane through the
    middle, so each part is the cells of one half (centroids on one side)."""
    m = MESHES["cube2"]
    p = hg.partition_cells(hg.Mesh(m.xyz, m.cells), 2)
    cen = m.xyz[m.cells].mean(axis=1)
    assert np.all(cen[p == 0, 0] < 0.5) and np.all(cen[p == 1, 0] > 0.5)


@pytest.mark.parametrize("name", list(MESHES))
@pytest.mark.parametrize("level,nparts", [(1, 2), (2, 2), (2, 3), (3, 4)])
def test_plan_pairs_and_covers_every_cross_rank_point(name, level, nparts):
    """Send counts of r to s equal receive counts of s from r; the planned
    points are exactly the lattice points whose copies lie on two or more
    ranks (found from the oracle's canonical numbering); every term of a
    point is one copy, in ascending cell id."""
    macro = MESHES[name]
    M = hg.Mesh(macro.xyz, macro.cells)
    part = hg.partition_cells(M, nparts)
    rm = RefinedMesh(macro, level)
    plans = [hg.exchange_plan(M, level, part, r) for r in range(nparts)]
    stride = plans[0]["stride"]
    s2c = oracle_stored_to_canonical(macro, rm, stride)
    for r in range(nparts):
        for s in range(nparts):
            assert plans[r]["send_count"][s] == plans[s]["recv_count"][r]
    # cells holding every canonical point
    holders = [set() for _ in range(rm.n_vertices)]
    for c in range(len(macro.cells)):
        for g in s2c[c * stride:(c + 1) * stride]:
            if g >= 0:
                holders[g].add(c)
    for r in range(nparts):
        P = plans[r]
        mine = np.flatnonzero(part == r)
        gl = lambda li: s2c[mine[li // stride] * stride + li % stride]  # noqa: E731
        want = sorted(g for g in range(rm.n_vertices)
                      if len({part[c] for c in holders[g]}) > 1 and
                      any(part[c] == r for c in holders[g]))
        got = []
        for p in range(len(P["point_start"]) - 1):
            tg = P["target_idx"][P["target_start"][p]:P["target_start"][p + 1]]
            g = {int(gl(t)) for t in tg}
            assert len(g) == 1                              # one lattice point
            g = g.pop()
            got.append(g)
            assert len(tg) == sum(part[c] == r for c in holders[g])
            assert P["point_start"][p + 1] - P["point_start"][p] == len(holders[g])
        assert sorted(got) == want


def _rank_main(rank, port, name, level, out, world=2):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        macro = MESHES[name]
        M = hg.Mesh(macro.xyz, macro.cells)
        part = hg.partition_cells(M, world)
        P = hg.exchange_plan(M, level, part, rank)
        rm = RefinedMesh(macro, level)
        x = sg.uniform_vector(77, rm.n_vertices)
        y, gids, parts = _local_partials(macro, rm, part, rank, P["stride"], x)
        # the exchange: this rank's partials to every rank it shares points
        # with, in the plan's order; receive buffers concatenated by rank
        sends = np.concatenate([[0], np.cumsum(P["send_count"])])
        recvs = np.concatenate([[0], np.cumsum(P["recv_count"])])
        recvbuf = torch.zeros(int(recvs[-1]), dtype=torch.float64)
        reqs = []
        for r in range(world):
            if r == rank:
                continue
            if P["send_count"][r]:
                sb = torch.tensor(y[P["send_idx"][sends[r]:sends[r + 1]]], dtype=torch.float64)
                reqs.append(dist.isend(sb, r))
            if P["recv_count"][r]:
                reqs.append(dist.irecv(recvbuf[recvs[r]:recvs[r + 1]], r))
        for q in reqs:
            q.wait()
        recv = recvbuf.numpy()
        yo = y.copy()
        for p in range(len(P["point_start"]) - 1):
            acc = 0.0
            for src in P["term_src"][P["point_start"][p]:P["point_start"][p + 1]]:
                acc += y[src] if src >= 0 else recv[-1 - src]
            yo[P["target_idx"][P["target_start"][p]:P["target_start"][p + 1]]] = acc
        # single-device order: all copies' partials in ascending cell id
        ref_order = {}
        stride = P["stride"]
        s2c = oracle_stored_to_canonical(macro, rm, stride)
        for c in range(len(macro.cells)):
            for g in s2c[c * stride:(c + 1) * stride]:
                if g >= 0:
                    ref_order.setdefault(int(g), []).append(c)
        A = fem.assemble(rm.cells, fem.p1_stiffness(rm.cell_xyz), rm.n_vertices)
        full = A @ x
        tg = P["target_idx"]
        res = {"n_points": len(P["point_start"]) - 1, "exact_order": True, "max_rel": 0.0}
        for t in tg:
            g = int(gids[t])
            acc = 0.0
            for c in ref_order[g]:
                acc += parts[c][g]
            res["exact_order"] &= bool(yo[t] == acc)
            res["max_rel"] = max(res["max_rel"], abs(yo[t] - full[g]) / np.abs(full).max())
        out[rank] = res
    finally:
        dist.barrier()
        dist.destroy_process_group()


@pytest.mark.parametrize("name,level,world", [("cube2", 2, 2), ("cube2perm", 3, 2),
                                              ("cube2", 2, 3)])
def test_rank_exchange_reproduces_the_global_apply(name, level, world):
    """World size 2, and 3 (edges and vertices then hold copies on three ranks,
    each sending to both others)."""
    port = 29500 + (os.getpid() + 7 * level + world) % 1000
    with mp.Manager() as m:
        out = m.dict()
        mp.spawn(_rank_main, args=(port, name, level, out, world), nprocs=world, join=True)
        res = dict(out)
    for rank in range(world):
        r = res[rank]
        assert r["n_points"] > 0
        assert r["exact_order"], r
        assert r["max_rel"] <= 1e-13, r


def _owned_copies(P, gids, n_local):
    """Local stored indices of the copies this rank owns: per lattice point the
    copy of the lowest global cell id.  A point of the plan is owned here iff
    its first term (ascending cell id) is local; every other point has all its
    copies here, and the first of them (local cells are in ascending id) owns
    it."""
    planned = np.zeros(n_local, dtype=bool)
    planned[P["target_idx"]] = True
    own = []
    seen = set()
    for li in range(n_local):
        g = int(gids[li])
        if g < 0 or planned[li] or g in seen:
            continue
        seen.add(g)
        own.append(li)
    for p in range(len(P["point_start"]) - 1):
        first = int(P["term_src"][P["point_start"][p]])
        if first >= 0:
            own.append(first)
    return np.array(sorted(own), dtype=np.int64)


def _cg_rank_main(rank, port, name, level, iters, out, world):
    """Conjugate gradients on the Dirichlet P1 Laplacian with every rank
    holding only its own cells: applies through per-copy partials, the plan's
    exchange and sum recipe; dots over owned copies and an FP64 all-reduce."""
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        macro = MESHES[name]
        M = hg.Mesh(macro.xyz, macro.cells)
        part = hg.partition_cells(M, world)
        P = hg.exchange_plan(M, level, part, rank)
        rm = RefinedMesh(macro, level)
        stride = P["stride"]
        s2c = oracle_stored_to_canonical(macro, rm, stride)
        mine = np.flatnonzero(part == rank)
        per = 8 ** rm.level
        Ke = fem.p1_stiffness(rm.cell_xyz)
        Ac = [fem.assemble(rm.cells[c * per:(c + 1) * per], Ke[c * per:(c + 1) * per],
                           rm.n_vertices) for c in mine]
        gids = np.concatenate([s2c[c * stride:(c + 1) * stride] for c in mine])
        n_local = len(gids)
        valid = gids >= 0
        dirichlet = np.zeros(n_local, dtype=bool)
        dirichlet[valid] = rm.boundary[gids[valid]]
        planned = np.zeros(n_local, dtype=bool)
        planned[P["target_idx"]] = True
        # copies of the points with all copies on this rank, grouped by point
        local_groups = {}
        for li in np.flatnonzero(valid & ~planned):
            local_groups.setdefault(int(gids[li]), []).append(li)
        owned = _owned_copies(P, gids, n_local)
        sends = np.concatenate([[0], np.cumsum(P["send_count"])])
        recvs = np.concatenate([[0], np.cumsum(P["recv_count"])])

        def apply(xs):
            partial = np.zeros(n_local)
            for lc in range(len(mine)):
                sl = slice(lc * stride, (lc + 1) * stride)
                g = gids[sl]
                ok = g >= 0
                xg = np.zeros(rm.n_vertices)
                xg[g[ok]] = xs[sl][ok]
                partial[sl][ok] = (Ac[lc] @ xg)[g[ok]]
            ys = np.zeros(n_local)
            for copies in local_groups.values():
                acc = 0.0
                for li in copies:
                    acc += partial[li]
                ys[copies] = acc
            recvbuf = torch.zeros(int(recvs[-1]), dtype=torch.float64)
            reqs = []
            for r in range(world):
                if r == rank:
                    continue
                if P["send_count"][r]:
                    sb = torch.tensor(partial[P["send_idx"][sends[r]:sends[r + 1]]],
                                      dtype=torch.float64)
                    reqs.append(dist.isend(sb, r))
                if P["recv_count"][r]:
                    reqs.append(dist.irecv(recvbuf[recvs[r]:recvs[r + 1]], r))
            for q in reqs:
                q.wait()
            recv = recvbuf.numpy()
            for p in range(len(P["point_start"]) - 1):
                acc = 0.0
                for src in P["term_src"][P["point_start"][p]:P["point_start"][p + 1]]:
                    acc += partial[src] if src >= 0 else recv[-1 - src]
                ys[P["target_idx"][P["target_start"][p]:P["target_start"][p + 1]]] = acc
            ys[dirichlet] = 0.0
            return ys

        def dot(a, b):
            t = torch.tensor([float(np.dot(a[owned], b[owned]))], dtype=torch.float64)
            dist.all_reduce(t)
            return float(t[0])

        bg = sg.uniform_vector(91, rm.n_vertices)
        bg[rm.boundary] = 0.0
        b = np.where(valid, bg[np.maximum(gids, 0)], 0.0)
        # the owned copies cover every lattice point once over all ranks
        t = torch.tensor([float(len(owned))], dtype=torch.float64)
        dist.all_reduce(t)
        n_owned = int(t[0])
        dot_err = abs(dot(b, b) - float(bg @ bg)) / float(bg @ bg)
        x = np.zeros(n_local)
        r = b.copy()
        p = r.copy()
        rr = dot(r, r)
        for _ in range(iters):
            q = apply(p)
            alpha = rr / dot(p, q)
            x += alpha * p
            r -= alpha * q
            rr_new = dot(r, r)
            p = r + (rr_new / rr) * p
            rr = rr_new
        copies_agree = all(np.all(x[c] == x[c[0]]) for c in local_groups.values())
        for pt in range(len(P["point_start"]) - 1):
            tg = P["target_idx"][P["target_start"][pt]:P["target_start"][pt + 1]]
            copies_agree &= bool(np.all(x[tg] == x[tg[0]]))
        out[rank] = {"x": x[valid], "g": gids[valid], "n_owned": n_owned,
                     "dot_err": dot_err, "copies_agree": copies_agree, "rr": rr}
    finally:
        dist.barrier()
        dist.destroy_process_group()


@pytest.mark.parametrize("name,level,world", [("cube2", 2, 2), ("cube2perm", 2, 3)])
def test_rank_cg_reproduces_the_single_domain_cg(name, level, world):
    """CG over ranks that hold only their own cells equals CG on the assembled
    Dirichlet matrix: iterates within 1e-11 of the global run after 12 steps
    (only the dots' summation order differs), copies of every shared point
    identical, owned copies counting every lattice point once."""
    iters = 12
    macro = MESHES[name]
    rm = RefinedMesh(macro, level)
    port = 29500 + (os.getpid() + 11 * level + 5 * world + 500) % 1000
    with mp.Manager() as m:
        out = m.dict()
        mp.spawn(_cg_rank_main, args=(port, name, level, iters, out, world), nprocs=world,
                 join=True)
        res = dict(out)
    A = fem.assemble(rm.cells, fem.p1_stiffness(rm.cell_xyz), rm.n_vertices).tocsr()
    I = rm.interior
    AII = A[I][:, I]
    b = sg.uniform_vector(91, rm.n_vertices)[I]
    x = np.zeros(len(I))
    r = b.copy()
    p = r.copy()
    rr = r @ r
    for _ in range(iters):
        q = AII @ p
        alpha = rr / (p @ q)
        x += alpha * p
        r -= alpha * q
        rr_new = r @ r
        p = r + (rr_new / rr) * p
        rr = rr_new
    xg = np.zeros(rm.n_vertices)
    xg[I] = x
    assert rr > 1e-20 * (b @ b)                  # still iterating: rounding has not decided it
    for rank in range(world):
        o = res[rank]
        assert o["n_owned"] == rm.n_vertices
        assert o["dot_err"] <= 1e-14
        assert o["copies_agree"]
        assert np.abs(o["x"] - xg[o["g"]]).max() <= 1e-11 * np.abs(xg).max()
