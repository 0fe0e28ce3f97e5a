// Distribution of the macro cells over ranks (Sec. 2: the macro primitives
// are distributed over processes, and one ghost-layer exchange per operator
// application makes the copies of the shared points agree).  Host only.
//
// Partition: recursive coordinate bisection of the cell centroids; each cut
// is along the longest extent of the current set's centroid bounding box,
// with the cells sorted by that coordinate (then the other two, then the
// cell id), and splits the set in proportion to the part counts on either
// side.  Deterministic for a given mesh and part count.
//
// Exchange plan of one rank and level: every interface point whose copies
// (cells containing it) lie on two or more ranks is enumerated in a fixed
// global order (faces, edges, vertices in mesh order; points in primitive
// order); a rank sends, for every such point it shares with rank r, the
// partial sums of its own copies (ascending cell id) and receives r's in
// the same order.  The full value of a point is the sum of all copies'
// partials in ascending global cell id, the order the single-device kernels
// use, so a distributed apply reproduces the single-device result exactly.
#include <algorithm>
#include <array>
#include <cstring>
#include <numeric>
#include <vector>

#include "hg_host.h"
#include "hytet.h"

using namespace hg;

struct hg_mesh : Mesh {};

namespace {

void rcb(const Mesh& m, std::vector<int>& cells, int p0, int np, int32_t* part) {
  if (np <= 1 || cells.size() <= 1) {
    for (int c : cells) part[c] = p0;
    return;
  }
  std::vector<std::array<double, 3>> cen(cells.size());
  double lo[3] = {1e300, 1e300, 1e300}, hi[3] = {-1e300, -1e300, -1e300};
  for (size_t q = 0; q < cells.size(); ++q) {
    for (int a = 0; a < 3; ++a) {
      double s = 0.0;
      for (int v = 0; v < 4; ++v) s += m.xyz[3 * m.cells[cells[q]][v] + a];
      cen[q][a] = 0.25 * s;
      lo[a] = std::min(lo[a], cen[q][a]);
      hi[a] = std::max(hi[a], cen[q][a]);
    }
  }
  int ax = 0;
  for (int a = 1; a < 3; ++a)
    if (hi[a] - lo[a] > hi[ax] - lo[ax]) ax = a;
  std::vector<size_t> ord(cells.size());
  std::iota(ord.begin(), ord.end(), 0);
  std::sort(ord.begin(), ord.end(), [&](size_t x, size_t y) {
    for (int s = 0; s < 3; ++s) {
      const int a = (ax + s) % 3;
      if (cen[x][a] != cen[y][a]) return cen[x][a] < cen[y][a];
    }
    return cells[x] < cells[y];
  });
  const int nl = np / 2;
  const size_t cut = (cells.size() * nl + np / 2) / np;
  std::vector<int> left, right;
  for (size_t q = 0; q < ord.size(); ++q) (q < cut ? left : right).push_back(cells[ord[q]]);
  rcb(m, left, p0, nl, part);
  rcb(m, right, p0 + nl, np - nl, part);
}

IfaceCopy make_copy(const Mesh& m, const Prim& p, int dim, int c) {
  IfaceCopy cp;
  cp.cell = c;
  for (int q = 0; q < 4; ++q) cp.loc[q] = -1;
  for (int a = 0; a <= dim; ++a)
    for (int q = 0; q < 4; ++q)
      if (m.cells[c][q] == p.vid[a]) cp.loc[a] = (int8_t)q;
  return cp;
}

}  // namespace

extern "C" {

int hg_partition_cells(const hg_mesh* m, int nparts, int32_t* part) {
  if (!m || !part || nparts < 1 || nparts > m->nc) {
    set_error("hg_partition_cells: need a mesh, an output array and 1 <= nparts <= %lld",
              m ? (long long)m->nc : 0LL);
    return HG_ERR_INVALID_ARG;
  }
  std::vector<int> cells(m->nc);
  std::iota(cells.begin(), cells.end(), 0);
  rcb(*m, cells, 0, nparts, part);
  return HG_OK;
}

int hg_exchange_plan(const hg_mesh* m, int level, const int32_t* part, int nparts, int rank,
                     int64_t sizes[6], int64_t* send_count, int64_t* send_idx,
                     int64_t* recv_count, int64_t* point_start, int64_t* term_src,
                     int64_t* target_start, int64_t* target_idx) {
  if (!m || !part || !sizes || nparts < 1 || rank < 0 || rank >= nparts) {
    set_error("hg_exchange_plan: bad argument");
    return HG_ERR_INVALID_ARG;
  }
  if (level < 0 || level > 9) {
    set_error("hg_exchange_plan: level %d outside 0..9", level);
    return HG_ERR_LEVEL_RANGE;
  }
  for (int64_t c = 0; c < m->nc; ++c)
    if (part[c] < 0 || part[c] >= nparts) {
      set_error("hg_exchange_plan: cell %lld has part %d outside 0..%d", (long long)c, part[c],
                nparts - 1);
      return HG_ERR_INVALID_ARG;
    }
  const int n = 1 << level, w = n + 1;
  const int64_t stride = (ntet(w) + 32 + 31) / 32 * 32;
  // points shared across ranks, in the global order, with their copies
  std::vector<std::vector<int64_t>> send(nparts);
  std::vector<int64_t> rcount(nparts, 0);
  std::vector<int64_t> pstart{0}, tstart{0}, tidx;
  std::vector<std::pair<int, int64_t>> terms;  // (source rank, local index there or recv slot)
  // receive slots are laid out per source rank in the same global order: a
  // first pass counts them, a second assigns offsets
  std::vector<std::vector<std::pair<int, int64_t>>> pending;  // per point: (rank, idx)
  // rank-local cell numbers: each rank's cells in ascending global id
  std::vector<std::vector<int64_t>> lcells(nparts);
  for (int64_t c = 0; c < m->nc; ++c) lcells[part[c]].push_back(c);
  auto local_of = [&](int r, int64_t c) {
    return (int64_t)(std::lower_bound(lcells[r].begin(), lcells[r].end(), c) - lcells[r].begin());
  };
  auto visit = [&](const Prim& p, int dim) {
    const int np = prim_points(dim, n);
    if (np <= 0 || p.cells.size() < 2) return;
    bool mine = false, other = false;
    for (int c : p.cells) {
      if (part[c] == rank) mine = true;
      else other = true;
    }
    bool multi = false;
    for (int c : p.cells) multi |= part[c] != part[p.cells[0]];
    if (!multi || !mine || !other) return;
    std::vector<IfaceCopy> cps;
    for (int c : p.cells) cps.push_back(make_copy(*m, p, dim, c));
    for (int pt = 0; pt < np; ++pt) {
      int wts[3];
      prim_point_weights(dim, n, pt, wts);
      std::vector<std::pair<int, int64_t>> cp;
      for (const IfaceCopy& c : cps) {
        int i, j, k;
        copy_local_ijk(c, dim, wts, i, j, k);
        const int r = part[c.cell];
        cp.push_back({r, local_of(r, c.cell) * stride + tw(w, i, j, k)});
      }
      // my copies go to every other rank holding a copy of this point
      std::vector<char> holds(nparts, 0);
      for (auto& e : cp) holds[e.first] = 1;
      for (int r = 0; r < nparts; ++r) {
        if (r == rank || !holds[r]) continue;
        for (auto& e : cp)
          if (e.first == rank) send[r].push_back(e.second);
      }
      pending.push_back(cp);
    }
  };
  for (auto& p : m->faces) visit(p, 2);
  for (auto& p : m->edges) visit(p, 1);
  for (auto& p : m->verts) visit(p, 0);
  for (auto& cp : pending)
    for (auto& e : cp)
      if (e.first != rank) rcount[e.first]++;
  std::vector<int64_t> roff(nparts, 0), rnext(nparts, 0);
  for (int r = 1; r < nparts; ++r) roff[r] = roff[r - 1] + rcount[r - 1];
  for (auto& cp : pending) {
    for (auto& e : cp) {
      if (e.first == rank) {
        terms.push_back({rank, e.second});
        tidx.push_back(e.second);
      } else {
        terms.push_back({e.first, roff[e.first] + rnext[e.first]++});
      }
    }
    pstart.push_back((int64_t)terms.size());
    tstart.push_back((int64_t)tidx.size());
  }
  int64_t nsend = 0, nrecv = 0;
  for (int r = 0; r < nparts; ++r) {
    nsend += (int64_t)send[r].size();
    nrecv += rcount[r];
  }
  sizes[0] = nsend;
  sizes[1] = nrecv;
  sizes[2] = (int64_t)pending.size();
  sizes[3] = (int64_t)terms.size();
  sizes[4] = (int64_t)tidx.size();
  sizes[5] = stride;
  if (send_count)
    for (int r = 0; r < nparts; ++r) send_count[r] = (int64_t)send[r].size();
  if (recv_count)
    for (int r = 0; r < nparts; ++r) recv_count[r] = rcount[r];
  if (send_idx) {
    int64_t o = 0;
    for (int r = 0; r < nparts; ++r)
      for (int64_t v : send[r]) send_idx[o++] = v;
  }
  if (point_start) std::copy(pstart.begin(), pstart.end(), point_start);
  if (term_src)
    for (size_t q = 0; q < terms.size(); ++q)
      term_src[q] = terms[q].first == rank ? terms[q].second : -(1 + terms[q].second);
  if (target_start) std::copy(tstart.begin(), tstart.end(), target_start);
  if (target_idx) std::copy(tidx.begin(), tidx.end(), target_idx);
  return HG_OK;
}

}  // extern "C"
