"""Multigrid over ranks (Sec. 2: macro primitives distributed over processes,
one ghost-layer exchange per operator application; Sec. 5.1: functions and
operators on a range of levels) on the CPU, with gloo ranks and no GPU.

Every rank holds only its own macro cells on every level, with the
library's partition (hg_partition_cells) and one exchange plan per level
(hg_exchange_plan).  Per-copy partials come from the oracle (each macro
cell's own assembled matrix, the cell's block of the nodal interpolation);
the emulated ranks:
  * apply: partials per copy, summed over the local copies of rank-local
    points and by the plan's recipe at cross-rank points;
  * the Jacobi diagonal: the same sum of the cells' diagonals;
  * restriction: each fine point contributes once, from the copy of its
    lowest-id cell (the owner, read from the plan: a planned point is owned
    here iff its first term is local), then the coarse level's sum;
  * prolongation: per cell from the cell's own coarse copies (every coarse
    DoF a fine point interpolates from lies in each cell holding the point),
    so the copies agree without an exchange;
  * coarse solve agglomerated: the owned coarse values gathered on rank 0,
    solved there, the solution broadcast.
Checked against the oracle's V-cycle on the assembled matrices: the
iterates after three V(2,2) cycles agree to 1e-11, and every copy of every
point holds the same value."""
import os

import numpy as np
import pytest
import scipy.linalg as sla

import synthgen as sg
from oracle import fem, gmg
from oracle.mesh import RefinedMesh

from helpers import oracle_stored_to_canonical
from test_partition_dist import MESHES, _owned_copies

torch = pytest.importorskip("torch")
import torch.distributed as dist
import torch.multiprocessing as mp

import paper_2308_01792_gb300 as hg

LMIN, LMAX, NU, OMEGA, CYCLES = 1, 3, 2, 2.0 / 3.0, 3


class _RankLevel:
    """One level as one rank stores it: its own cells' copies of the points."""

    def __init__(self, macro, M, part, rank, world, level):
        self.rank, self.world = rank, world
        self.P = P = hg.exchange_plan(M, level, part, rank)
        self.rm = rm = RefinedMesh(macro, level)
        self.stride = stride = P["stride"]
        s2c = oracle_stored_to_canonical(macro, rm, stride)
        self.mine = mine = np.flatnonzero(part == rank)
        self.gids = gids = np.concatenate([s2c[c * stride:(c + 1) * stride] for c in mine])
        self.n_local = n_local = len(gids)
        self.valid = valid = gids >= 0
        boundary = np.zeros(n_local, dtype=bool)
        boundary[valid] = rm.boundary[gids[valid]]
        self.free = valid & ~boundary
        planned = np.zeros(n_local, dtype=bool)
        planned[P["target_idx"]] = True
        self.local_groups = {}
        for li in np.flatnonzero(valid & ~planned):
            self.local_groups.setdefault(int(gids[li]), []).append(li)
        self.owned = _owned_copies(P, gids, n_local)
        self.owned_flag = np.zeros(n_local, dtype=bool)
        self.owned_flag[self.owned] = True
        per = 8 ** level
        Ke = fem.p1_stiffness(rm.cell_xyz)
        self.Ac = [fem.assemble(rm.cells[c * per:(c + 1) * per], Ke[c * per:(c + 1) * per],
                                rm.n_vertices).tocsr() for c in mine]
        self.sends = np.concatenate([[0], np.cumsum(P["send_count"])])
        self.recvs = np.concatenate([[0], np.cumsum(P["recv_count"])])
        dpart = np.zeros(n_local)
        for lc in range(len(mine)):
            sl, g, ok = self.cell(lc)
            dpart[sl][ok] = self.Ac[lc].diagonal()[g[ok]]
        self.diag = self.sum_copies(dpart)

    def cell(self, lc):
        sl = slice(lc * self.stride, (lc + 1) * self.stride)
        g = self.gids[sl]
        return sl, g, g >= 0

    def sum_copies(self, partial):
        """Full value of every point at every copy: local copies summed in
        ascending cell id, cross-rank points by the plan (one exchange)."""
        P, world, rank = self.P, self.world, self.rank
        ys = np.zeros(self.n_local)
        for copies in self.local_groups.values():
            acc = 0.0
            for li in copies:
                acc += partial[li]
            ys[copies] = acc
        recvbuf = torch.zeros(int(self.recvs[-1]), dtype=torch.float64)
        reqs = []
        for r in range(world):
            if r == rank:
                continue
            if P["send_count"][r]:
                sb = torch.tensor(partial[P["send_idx"][self.sends[r]:self.sends[r + 1]]],
                                  dtype=torch.float64)
                reqs.append(dist.isend(sb, r))
            if P["recv_count"][r]:
                reqs.append(dist.irecv(recvbuf[self.recvs[r]:self.recvs[r + 1]], r))
        for q in reqs:
            q.wait()
        recv = recvbuf.numpy()
        for p in range(len(P["point_start"]) - 1):
            acc = 0.0
            for src in P["term_src"][P["point_start"][p]:P["point_start"][p + 1]]:
                acc += partial[src] if src >= 0 else recv[-1 - src]
            ys[P["target_idx"][P["target_start"][p]:P["target_start"][p + 1]]] = acc
        return ys

    def apply(self, xs):
        partial = np.zeros(self.n_local)
        for lc in range(len(self.mine)):
            sl, g, ok = self.cell(lc)
            xg = np.zeros(self.rm.n_vertices)
            xg[g[ok]] = xs[sl][ok]
            partial[sl][ok] = (self.Ac[lc] @ xg)[g[ok]]
        ys = self.sum_copies(partial)
        ys[~self.free] = 0.0
        return ys


class _RankTransfer:
    """The cells' blocks of the nodal interpolation between two levels."""

    def __init__(self, fine, coarse, Pfull):
        self.fine, self.coarse = fine, coarse
        self.blocks = []
        for lc in range(len(fine.mine)):
            _, gf, okf = fine.cell(lc)
            _, gc, okc = coarse.cell(lc)
            Pc = Pfull[gf[okf]][:, gc[okc]].tocsr()
            # every coarse DoF a fine point of the cell interpolates from is in the cell
            assert np.allclose(Pc.sum(axis=1).A1, Pfull[gf[okf]].sum(axis=1).A1, rtol=0, atol=0)
            self.blocks.append((np.flatnonzero(okf), np.flatnonzero(okc), Pc))

    def restrict(self, r):
        f, c = self.fine, self.coarse
        partial = np.zeros(c.n_local)
        for lc, (fo, co, Pc) in enumerate(self.blocks):
            rf = r[lc * f.stride + fo] * f.owned_flag[lc * f.stride + fo]
            partial[lc * c.stride + co] += Pc.T @ rf
        out = c.sum_copies(partial)
        out[~c.free] = 0.0
        return out

    def prolong(self, e):
        f, c = self.fine, self.coarse
        out = np.zeros(f.n_local)
        for lc, (fo, co, Pc) in enumerate(self.blocks):
            out[lc * f.stride + fo] = Pc @ e[lc * c.stride + co]
        out[~f.free] = 0.0
        return out


def _gmg_rank_main(rank, port, name, out, world):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        macro = MESHES[name]
        M = hg.Mesh(macro.xyz, macro.cells)
        part = hg.partition_cells(M, world)
        lev = {l: _RankLevel(macro, M, part, rank, world, l) for l in range(LMIN, LMAX + 1)}
        olev = {l: gmg.Level(macro, l) for l in range(LMIN, LMAX + 1)}
        xfer = {l: _RankTransfer(lev[l], lev[l - 1], gmg.p1_prolongation(olev[l], olev[l - 1]))
                for l in range(LMIN + 1, LMAX + 1)}
        coarse = olev[LMIN]
        chol = sla.cho_factor(coarse.A.toarray()) if rank == 0 else None

        def coarse_solve(b):
            L = lev[LMIN]
            mine = (L.gids[L.owned], b[L.owned])
            gathered = [None] * world
            dist.all_gather_object(gathered, mine)
            box = [None]
            if rank == 0:                               # agglomerated on one rank
                bg = np.zeros(coarse.n)
                for ids, vals in gathered:
                    bg[ids] = vals
                xg = np.zeros(coarse.n)
                xg[coarse.interior] = sla.cho_solve(chol, bg[coarse.interior])
                box = [xg]
            dist.broadcast_object_list(box, src=0)
            return np.where(L.valid, box[0][np.maximum(L.gids, 0)], 0.0)

        def smooth(L, x, b):
            for _ in range(NU):
                r = b - L.apply(x)
                x = x.copy()
                x[L.free] += OMEGA * r[L.free] / L.diag[L.free]
            return x

        def vcycle(l, x, b):
            if l == LMIN:
                return coarse_solve(b)
            L = lev[l]
            x = smooth(L, x, b)
            r = b - L.apply(x)
            bc = xfer[l].restrict(r)
            ec = vcycle(l - 1, np.zeros(lev[l - 1].n_local), bc)
            x = x + xfer[l].prolong(ec)
            return smooth(L, x, b)

        L = lev[LMAX]
        bg = sg.uniform_vector(93, L.rm.n_vertices)
        bg[L.rm.boundary] = 0.0
        b = np.where(L.valid, bg[np.maximum(L.gids, 0)], 0.0)
        x = np.zeros(L.n_local)
        for _ in range(CYCLES):
            x = vcycle(LMAX, x, b)
        agree = all(np.all(x[c] == x[c[0]]) for c in L.local_groups.values())
        P = L.P
        for p in range(len(P["point_start"]) - 1):
            tg = P["target_idx"][P["target_start"][p]:P["target_start"][p + 1]]
            agree &= bool(np.all(x[tg] == x[tg[0]]))
        r = b - L.apply(x)
        t = torch.tensor([float(r[L.owned] @ r[L.owned])], dtype=torch.float64)
        dist.all_reduce(t)
        out[rank] = {"x": x[L.valid], "g": L.gids[L.valid], "agree": agree,
                     "rr": float(t[0]), "n_planned": [len(lev[l].P["point_start"]) - 1
                                                      for l in lev]}
    finally:
        dist.barrier()
        dist.destroy_process_group()


@pytest.mark.parametrize("name,world", [("cube2", 2), ("cube2perm", 3)])
def test_rank_vcycles_reproduce_the_single_domain_vcycles(name, world):
    macro = MESHES[name]
    port = 29500 + (os.getpid() + 13 * world + 250) % 1000
    with mp.Manager() as m:
        out = m.dict()
        mp.spawn(_gmg_rank_main, args=(port, name, out, world), nprocs=world, join=True)
        res = dict(out)
    H = gmg.Hierarchy(macro, LMIN, LMAX)
    fine = H.levels[LMAX]
    I = fine.interior
    bg = sg.uniform_vector(93, fine.n)
    b = bg[I]
    x = np.zeros(len(I))
    for _ in range(CYCLES):
        x = gmg.vcycle(H, LMAX, x, b, NU, NU, OMEGA)
    xg = np.zeros(fine.n)
    xg[I] = x
    r = b - fine.A @ x
    assert np.linalg.norm(r) < 0.2 * np.linalg.norm(b)     # the cycles do reduce the residual
    for rank in range(world):
        o = res[rank]
        assert all(n > 0 for n in o["n_planned"])           # every level exchanges across ranks
        assert o["agree"]
        assert np.abs(o["x"] - xg[o["g"]]).max() <= 1e-11 * np.abs(xg).max()
        assert abs(np.sqrt(o["rr"]) - np.linalg.norm(r)) <= 1e-10 * np.linalg.norm(r)
