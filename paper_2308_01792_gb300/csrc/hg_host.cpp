// Host side of the library: macro mesh and primitive graph (Sec. 2), the
// per-level device maps of the refinement hierarchy (Sec. 3-4), per-cell
// stencil tables of constant-coefficient operators (Sec. 5.2), and the C ABI
// glue for everything except multigrid (hg_gmg.cpp).
#include <cuda_runtime.h>

#include <algorithm>
#include <array>
#include <climits>
#include <cmath>
#include <cstdarg>
#include <cstdio>
#include <cstring>
#include <map>
#include <memory>
#include <numeric>
#include <set>
#include <vector>

#include "hg_host.h"

namespace hg {

static thread_local std::string g_err;

void set_error(const char* fmt, ...) {
  char buf[1024];
  va_list ap;
  va_start(ap, fmt);
  vsnprintf(buf, sizeof buf, fmt, ap);
  va_end(ap);
  g_err = buf;
}

int cuda_fail(cudaError_t e, const char* what) {
  set_error("CUDA error %d (%s) in %s", (int)e, cudaGetErrorString(e), what);
  return HG_ERR_CUDA;
}

// ------------------------------------------------------------------ mesh
int Mesh::build(const double* xyz_, int64_t nv_, const int64_t* cells_, int64_t nc_) {
  nv = nv_;
  nc = nc_;
  xyz.assign(xyz_, xyz_ + 3 * nv);
  cells.resize(nc);
  for (int64_t c = 0; c < nc; ++c) {
    std::array<int64_t, 4> v;
    for (int m = 0; m < 4; ++m) {
      v[m] = cells_[4 * c + m];
      if (v[m] < 0 || v[m] >= nv) {
        set_error("cell %lld references vertex %lld outside [0,%lld)", (long long)c,
                  (long long)v[m], (long long)nv);
        return HG_ERR_BAD_MESH;
      }
    }
    for (int a = 0; a < 4; ++a)
      for (int b = a + 1; b < 4; ++b)
        if (v[a] == v[b]) {
          set_error("cell %lld repeats vertex %lld", (long long)c, (long long)v[a]);
          return HG_ERR_BAD_MESH;
        }
    cells[c] = v;
    double J[9];
    cell_jacobian(c, J);
    double det = J[0] * (J[4] * J[8] - J[5] * J[7]) - J[1] * (J[3] * J[8] - J[5] * J[6]) +
                 J[2] * (J[3] * J[7] - J[4] * J[6]);
    double scale = 0;
    for (int q = 0; q < 9; ++q) scale = std::max(scale, std::fabs(J[q]));
    if (!(std::fabs(det) > 1e-14 * scale * scale * scale)) {
      set_error("cell %lld has zero volume", (long long)c);
      return HG_ERR_BAD_MESH;
    }
  }
  // primitives: faces (opposite local vertex f), edges, vertices
  std::map<std::array<int64_t, 3>, int> fmap;
  std::map<std::array<int64_t, 2>, int> emap;
  cell_face.assign(nc, {});
  cell_edge.assign(nc, {});
  for (int64_t c = 0; c < nc; ++c) {
    for (int f = 0; f < 4; ++f) {
      std::array<int64_t, 3> key;
      int q = 0;
      for (int m = 0; m < 4; ++m)
        if (m != f) key[q++] = cells[c][m];
      std::sort(key.begin(), key.end());
      auto it = fmap.find(key);
      int id;
      if (it == fmap.end()) {
        id = (int)faces.size();
        fmap.emplace(key, id);
        faces.push_back({{key[0], key[1], key[2]}, {}});
      } else {
        id = it->second;
      }
      faces[id].cells.push_back((int)c);
      cell_face[c][f] = id;
    }
    for (int e = 0; e < 6; ++e) {
      std::array<int64_t, 2> key = {cells[c][kEdgeVerts[e][0]], cells[c][kEdgeVerts[e][1]]};
      std::sort(key.begin(), key.end());
      auto it = emap.find(key);
      int id;
      if (it == emap.end()) {
        id = (int)edges.size();
        emap.emplace(key, id);
        edges.push_back({{key[0], key[1], -1}, {}});
      } else {
        id = it->second;
      }
      edges[id].cells.push_back((int)c);
      cell_edge[c][e] = id;
    }
  }
  verts.assign(nv, {});
  for (int64_t v = 0; v < nv; ++v) verts[v].vid = {v, -1, -1};
  for (int64_t c = 0; c < nc; ++c)
    for (int m = 0; m < 4; ++m) verts[cells[c][m]].cells.push_back((int)c);
  // every macro vertex is a primitive with one copy per containing cell; a
  // vertex of no cell would have none
  for (int64_t v = 0; v < nv; ++v)
    if (verts[v].cells.empty()) {
      set_error("vertex %lld belongs to no cell", (long long)v);
      return HG_ERR_BAD_MESH;
    }
  n_boundary_faces = 0;
  for (auto& f : faces) {
    if (f.cells.size() > 2) {
      set_error("face (%lld,%lld,%lld) shared by %zu cells: not conforming",
                (long long)f.vid[0], (long long)f.vid[1], (long long)f.vid[2], f.cells.size());
      return HG_ERR_BAD_MESH;
    }
    f.dirichlet = f.cells.size() == 1;
    n_boundary_faces += f.dirichlet;
  }
  // Sec. 2: cells meet only in common faces, edges or vertices, so the two
  // cells of an interior face lie on opposite sides of it (a repeated or
  // folded-over cell puts both opposite vertices on the same side)
  for (const auto& f : faces) {
    if (f.cells.size() != 2) continue;
    const int fid = (int)(&f - faces.data());
    const double* a = &xyz[3 * f.vid[0]];
    const double* b = &xyz[3 * f.vid[1]];
    const double* d = &xyz[3 * f.vid[2]];
    const double u[3] = {b[0] - a[0], b[1] - a[1], b[2] - a[2]};
    const double w[3] = {d[0] - a[0], d[1] - a[1], d[2] - a[2]};
    const double nrm[3] = {u[1] * w[2] - u[2] * w[1], u[2] * w[0] - u[0] * w[2],
                           u[0] * w[1] - u[1] * w[0]};
    double side[2];
    for (int q = 0; q < 2; ++q) {
      const int64_t c = f.cells[q];
      int opp = 0;
      while (cell_face[c][opp] != fid) ++opp;
      const double* p = &xyz[3 * cells[c][opp]];
      side[q] = nrm[0] * (p[0] - a[0]) + nrm[1] * (p[1] - a[1]) + nrm[2] * (p[2] - a[2]);
    }
    if (!(side[0] * side[1] < 0)) {
      set_error("cells %d and %d lie on the same side of their common face (%lld,%lld,%lld): "
                "they overlap", f.cells[0], f.cells[1], (long long)f.vid[0],
                (long long)f.vid[1], (long long)f.vid[2]);
      return HG_ERR_BAD_MESH;
    }
  }
  std::vector<char> vb(nv, 0);
  std::set<std::array<int64_t, 2>> be;
  for (auto& f : faces)
    if (f.dirichlet) {
      for (int m = 0; m < 3; ++m) vb[f.vid[m]] = 1;
      for (int a = 0; a < 3; ++a)
        for (int b = a + 1; b < 3; ++b) be.insert({f.vid[a], f.vid[b]});
    }
  for (auto& e : edges) e.dirichlet = be.count({e.vid[0], e.vid[1]}) > 0;
  for (int64_t v = 0; v < nv; ++v) verts[v].dirichlet = vb[v] != 0;
  for (auto* prims : {&faces, &edges, &verts})
    for (auto& p : *prims) std::sort(p.cells.begin(), p.cells.end());
  // integer lattice: smallest D <= 64 making every coordinate an integer
  grid_denom = 0;
  for (int D = 1; D <= 64 && !grid_denom; ++D) {
    bool ok = true;
    for (double x : xyz) {
      double s = x * D;
      if (std::fabs(s - std::nearbyint(s)) > 1e-9 || std::fabs(s) > 1e6) {
        ok = false;
        break;
      }
    }
    if (ok) grid_denom = D;
  }
  if (grid_denom) {
    ixyz.resize(3 * nv);
    for (int64_t q = 0; q < 3 * nv; ++q) ixyz[q] = (int64_t)std::nearbyint(xyz[q] * grid_denom);
  }
  return HG_OK;
}

void Mesh::cell_jacobian(int64_t c, double J[9]) const {
  // columns x1-x0, x2-x0, x3-x0 ; J[r*3+col]
  const double* p0 = &xyz[3 * cells[c][0]];
  for (int col = 0; col < 3; ++col) {
    const double* p = &xyz[3 * cells[c][col + 1]];
    for (int r = 0; r < 3; ++r) J[r * 3 + col] = p[r] - p0[r];
  }
}

// Primitive of a class (bit f = on the face opposite local vertex f) of cell c.
const Prim* Mesh::class_prim(int64_t c, int cls) const {
  int nb = __builtin_popcount(cls);
  if (nb == 0 || nb == 4) return nullptr;
  if (nb == 1) {
    int f = __builtin_ctz(cls);
    return &faces[cell_face[c][f]];
  }
  int rest[4], q = 0;
  for (int m = 0; m < 4; ++m)
    if (!(cls >> m & 1)) rest[q++] = m;
  if (nb == 3) return &verts[cells[c][rest[0]]];
  for (int e = 0; e < 6; ++e)
    if (kEdgeVerts[e][0] == rest[0] && kEdgeVerts[e][1] == rest[1]) return &edges[cell_edge[c][e]];
  return nullptr;
}

uint8_t Mesh::class_flags(int64_t c, int cls) const {
  if (cls == 0) return CF_OWNER;
  const Prim* p = class_prim(c, cls);
  if (!p) return 0;
  uint8_t f = 0;
  if (p->dirichlet) f |= CF_DIRICHLET;
  if (p->cells.front() == (int)c) f |= CF_OWNER;
  if (p->cells.size() >= 2) f |= CF_MULTI;
  return f;
}

// ------------------------------------------------------------ streaming plan
int stream_ctas(int n, int ncells, int n_items, int sms) {
  const int64_t pts = (int64_t)ncells * ntet(n + 1);
  const int64_t want = std::max<int64_t>((pts + 2047) / 2048, ((int64_t)n_items + 15) / 16);
  return (int)std::max<int64_t>(1, std::min<int64_t>(std::max(sms, 1), want));
}

int stream_band_rows(int n, int esize) {
  const int w = n + 1;
  // whole planes when plane 0 (the largest) fits a slot with its 16-byte rounding
  if (ntri(w) * esize + 32 <= kStreamSlotBytes) return w;
  // else bands of rows whose staged range (rows j0-1 .. j0+rows) fits a slot
  return std::max(1, kStreamSlotBytes / (w * esize) - 2);
}

int stream_plan(int n, int ncells, int nctas, int esize, StreamPlanHost& P) {
  const int w = n + 1;
  const int V = 16 / esize;
  const int JB = stream_band_rows(n, esize);
  if (JB < w && (int64_t)(JB + 2) * w * esize + 32 > kStreamSlotBytes) {
    set_error("streaming plan: no band of rows fits a slot at w = %d", w);
    return HG_ERR_UNSUPPORTED;
  }
  auto rs = [&](int j, int k) { return (int64_t)tw(w, 0, j, k); };
  // the sequence of pieces (cell, plane k, rows [ja, jb)): per cell, band and
  // plane, consecutive rows of at most kStreamPiece points (one row at least)
  struct Piece { int cell, k, ja, jb; double cost; };
  std::vector<Piece> seq;
  double total = 0;
  for (int c = 0; c < ncells; ++c)
    for (int j0 = 0; j0 < w; j0 += JB)
      for (int k = 0; k <= w - 1 - j0; ++k) {
        const int jend = std::min(j0 + JB, w - k);
        for (int ja = j0; ja < jend;) {
          int jb = ja;
          int64_t pts = 0;
          while (jb < jend && (jb == ja || pts + (w - k - jb) <= kStreamPiece)) pts += w - k - jb++;
          // cost: points, staged elements (three planes' rows) and a fixed part
          const double cost = (double)pts + 0.75 * (double)pts + 96.0;
          seq.push_back({c, k, ja, jb, cost});
          total += cost;
          ja = jb;
        }
      }
  P = StreamPlanHost{};
  P.nctas = nctas;
  P.band_rows = JB;
  P.cta_copies.assign(nctas + 1, 0);
  P.cta_items.assign(nctas + 1, 0);
  size_t q = 0;
  double acc = 0;
  for (int g = 0; g < nctas; ++g) {
    P.cta_copies[g] = (int32_t)P.copies.size();
    P.cta_items[g] = (int32_t)(P.items.size() / 3);
    const int copy0 = (int)P.copies.size();
    const size_t item0 = P.items.size();
    const double target = total * (g + 1) / nctas;
    const size_t q0 = q;
    while (q < seq.size() && (g == nctas - 1 || acc + 0.5 * seq[q].cost <= target)) acc += seq[q++].cost;
    // the rows each (cell, band, plane) must have staged: the union over the
    // CTA's pieces of rows max(ja-1,0) .. min(jb, w-1-kk) of planes kk = k-1..k+1
    struct Need { int cell, j0, kk, jlo, jhi; };
    std::vector<Need> need;   // in (cell, band, plane) order
    auto band_of = [&](int ja) { return ja / JB * JB; };
    for (size_t t = q0; t < q; ++t) {
      const Piece& p = seq[t];
      for (int kk = std::max(p.k - 1, 0); kk <= std::min(p.k + 1, w - 1); ++kk) {
        const int jlo = std::max(p.ja - 1, 0), jhi = std::min(p.jb, w - 1 - kk);
        if (jlo > jhi) continue;
        const int j0 = band_of(p.ja);
        bool found = false;
        for (auto& nd : need)
          if (nd.cell == p.cell && nd.j0 == j0 && nd.kk == kk) {
            nd.jlo = std::min(nd.jlo, jlo);
            nd.jhi = std::max(nd.jhi, jhi);
            found = true;
            break;
          }
        if (!found) need.push_back({p.cell, j0, kk, jlo, jhi});
      }
    }
    std::sort(need.begin(), need.end(), [](const Need& x, const Need& y) {
      return x.cell != y.cell ? x.cell < y.cell : x.j0 != y.j0 ? x.j0 < y.j0 : x.kk < y.kk;
    });
    // copies: consecutive staged ranges that are contiguous in the cell's
    // array (whole-plane tails and heads) share a copy while it fits a slot
    std::vector<int> cop(need.size());
    std::vector<int64_t> cga(need.size());
    for (size_t a0 = 0; a0 < need.size();) {
      const int64_t g0 = rs(need[a0].jlo, need[a0].kk);
      int64_t gend = rs(need[a0].jhi, need[a0].kk) + (w - need[a0].kk - need[a0].jhi);
      size_t a1 = a0 + 1;
      while (a1 < need.size() && a1 - a0 < 64 && need[a1].cell == need[a0].cell &&
             need[a1].j0 == need[a0].j0 && need[a1].kk == need[a1 - 1].kk + 1) {
        const int64_t h0 = rs(need[a1].jlo, need[a1].kk);
        const int64_t h1 = rs(need[a1].jhi, need[a1].kk) + (w - need[a1].kk - need[a1].jhi);
        if (h0 != gend) break;  // not contiguous with the previous range
        if (((h1 + V - 1) / V * V - g0 / V * V) * esize > kStreamSlotBytes) break;
        gend = h1;
        ++a1;
      }
      const int64_t ga = g0 / V * V, ge = (gend + V - 1) / V * V;
      if ((ge - ga) * esize > kStreamSlotBytes) {
        set_error("streaming plan: a staged range of %lld elements exceeds a slot", (long long)(ge - ga));
        return HG_ERR_UNSUPPORTED;
      }
      const int c = (int)P.copies.size() - copy0;
      P.copies.push_back({need[a0].cell, (int)ga, (int)(ge - ga), 0});
      for (size_t t = a0; t < a1; ++t) {
        cop[t] = c;
        cga[t] = ga;
      }
      a0 = a1;
    }
    auto copy_of = [&](int cell, int j0, int kk, int& c, int64_t& ga) {
      for (size_t t = 0; t < need.size(); ++t)
        if (need[t].cell == cell && need[t].j0 == j0 && need[t].kk == kk) {
          c = cop[t];
          ga = cga[t];
          return;
        }
      c = -1;
      ga = 0;
    };
    // items: the pieces, with the copies holding planes k, k-1, k+1
    for (size_t t = q0; t < q; ++t) {
      const Piece& p = seq[t];
      const int j0 = band_of(p.ja);
      int c0, cm = -1, cp = -1;
      int64_t g0 = 0, gm = 0, gp = 0;
      copy_of(p.cell, j0, p.k, c0, g0);
      if (p.k >= 1) copy_of(p.cell, j0, p.k - 1, cm, gm);
      if (p.k + 1 <= w - 1 && std::max(p.ja - 1, 0) <= std::min(p.jb, w - 1 - (p.k + 1)))
        copy_of(p.cell, j0, p.k + 1, cp, gp);
      P.items.push_back({p.cell, p.k, p.ja | (p.jb << 16), 0});
      P.items.push_back({c0, cm, cp, 0});
      P.items.push_back({(int)g0, (int)gm, (int)gp, 0});
    }
    // arrivals: every slot phase expects kStreamArrive; each item arrives once on
    // each distinct copy it reads, the first reader of a copy adds the rest
    const int ncop = (int)P.copies.size() - copy0;
    std::vector<int> readers(ncop, 0);
    for (size_t t = item0; t < P.items.size(); t += 3) {
      const int4 c = P.items[t + 1];
      readers[c.x]++;
      if (c.y >= 0 && c.y != c.x) readers[c.y]++;
      if (c.z >= 0 && c.z != c.x && c.z != c.y) readers[c.z]++;
    }
    for (int c = 0; c < ncop; ++c)
      if (readers[c] < 1 || readers[c] > kStreamArrive) {
        set_error("streaming plan: copy %d of CTA %d has %d readers", c, g, readers[c]);
        return HG_ERR_UNSUPPORTED;
      }
    std::vector<char> seen(ncop, 0);
    for (size_t t = item0; t < P.items.size(); t += 3) {
      const int4 c = P.items[t + 1];
      auto cnt = [&](int cc) {
        const int r = seen[cc] ? 1 : 1 + kStreamArrive - readers[cc];
        seen[cc] = 1;
        return r;
      };
      const int n0 = cnt(c.x);
      const int nm = (c.y >= 0 && c.y != c.x) ? cnt(c.y) : 0;
      const int np = (c.z >= 0 && c.z != c.x && c.z != c.y) ? cnt(c.z) : 0;
      P.items[t].w = n0 | (nm << 10) | (np << 20);
    }
  }
  P.cta_copies[nctas] = (int32_t)P.copies.size();
  P.cta_items[nctas] = (int32_t)(P.items.size() / 3);
  return HG_OK;
}

// ------------------------------------------------------------ hierarchy
template <class T>
static int upload(T** dst, const std::vector<T>& src) {
  *dst = nullptr;
  if (src.empty()) return HG_OK;
  HG_CUDA(cudaMalloc((void**)dst, src.size() * sizeof(T)));
  HG_CUDA(cudaMemcpy(*dst, src.data(), src.size() * sizeof(T), cudaMemcpyHostToDevice));
  return HG_OK;
}

int Hier::build_level(int l) {
  LevelHost& H = lv[l - lmin];
  LevelDev& L = H.dev;
  memset(&L, 0, sizeof L);
  L.level = l;
  L.n = 1 << l;
  L.w = L.n + 1;
  L.ncells = (int)mesh->nc;
  // padded to a multiple of 32 elements with at least 32 spare: the interior
  // tiles' window loads of lanes past a row's end reach up to 25 elements
  // beyond the cell's last lattice point
  L.cell_stride = (ntet(L.w) + 32 + 31) / 32 * 32;
  L.n_stored = L.cell_stride * mesh->nc;
  const int n = L.n, w = L.w;
  // class flags
  std::vector<uint8_t> fl(16 * mesh->nc);
  for (int64_t c = 0; c < mesh->nc; ++c)
    for (int cls = 0; cls < 16; ++cls) fl[16 * c + cls] = mesh->class_flags(c, cls);
  H.cls_flags = fl;
  if (int r = upload(&L.cls_flags, fl)) return r;
  // interface primitives: non-Dirichlet first, then Dirichlet
  std::vector<IfacePrim> prims;
  std::vector<IfaceCopy> copies;
  for (int pass = 0; pass < 2; ++pass) {
    auto add = [&](const Prim& p, int dim) {
      if ((int)p.dirichlet != pass || prim_points(dim, n) <= 0) return;
      IfacePrim ip;
      ip.dim = dim;
      ip.ncopies = (int)p.cells.size();
      ip.first_copy = (int)copies.size();
      ip.dirichlet = p.dirichlet;
      for (int c : p.cells) {
        IfaceCopy cp;
        cp.cell = c;
        for (int m = 0; m < 4; ++m) cp.loc[m] = -1;
        for (int m = 0; m <= dim; ++m)
          for (int q = 0; q < 4; ++q)
            if (mesh->cells[c][q] == p.vid[m]) cp.loc[m] = (int8_t)q;
        copies.push_back(cp);
      }
      prims.push_back(ip);
      if (pass == 0) L.n_prims_inner++;
      L.max_copies = std::max(L.max_copies, ip.ncopies);
    };
    for (auto& p : mesh->faces) add(p, 2);
    for (auto& p : mesh->edges) add(p, 1);
    for (auto& p : mesh->verts) add(p, 0);
  }
  L.n_prims = (int)prims.size();
  std::vector<int32_t> pbase(prims.size() + 1, 0);
  for (size_t q = 0; q < prims.size(); ++q) pbase[q + 1] = pbase[q] + prim_points(prims[q].dim, n);
  H.prims = prims;
  H.copies = copies;
  H.prim_point_base = pbase;
  if (int r = upload(&L.prims, prims)) return r;
  if (int r = upload(&L.copies, copies)) return r;
  if (int r = upload(&L.prim_point_base, pbase)) return r;
  // interface items: 32 consecutive points of one primitive (inner primitives first)
  std::vector<int4> items;
  std::vector<int32_t> item_prim;
  for (int q = 0; q < (int)prims.size(); ++q) {
    const IfacePrim& P = prims[q];
    const int meta = P.dim | (P.ncopies << 4) | (P.dirichlet << 12);
    for (int p0 = 0; p0 < prim_points(P.dim, n); p0 += 32) {
      items.push_back({P.first_copy, p0, meta, 0});
      item_prim.push_back(q);
    }
    if (q + 1 == L.n_prims_inner) L.n_items_inner = (int)items.size();
  }
  L.n_items = (int)items.size();
  if (int r = upload(&L.items, items)) return r;
  if (int r = upload(&L.item_prim, item_prim)) return r;
  // apply items: floor(32 / ncopies) points of one primitive, one lane per
  // (point, copy); primitives with more than 32 copies keep 32 points per item
  // (one lane per point)
  std::vector<int4> citems;
  for (int q = 0; q < (int)prims.size(); ++q) {
    const IfacePrim& P = prims[q];
    const int meta = P.dim | (P.ncopies << 4) | (P.dirichlet << 12);
    const int per = P.ncopies <= 32 ? 32 / P.ncopies : 32;
    const int np = prim_points(P.dim, n);
    for (int p0 = 0; p0 < np; p0 += per) citems.push_back({P.first_copy, p0, meta, std::min(per, np - p0)});
  }
  L.n_citems = (int)citems.size();
  if (int r = upload(&L.citems, citems)) return r;
  {
    // what each lane of an apply item works on (the kernels would otherwise
    // derive it from the item, the primitive's point index and the copy)
    std::vector<uint2> clane((size_t)L.n_citems * 32, uint2{0u, 63u << 24});
    for (int q = 0; q < L.n_citems; ++q) {
      const int4 it = citems[q];
      const int dim = it.z & 15, C = (it.z >> 4) & 255, dirichlet = (it.z >> 12) & 1;
      if (C > 32) continue;
      for (int lane = 0; lane < 32; ++lane) {
        // copy-major lanes: lane = c * P + pt (P = 32 / C points), so that the lanes of
        // one copy hold consecutive points of the primitive in one cell
        const int P = 32 / C, c = lane / P, pt = lane - c * P;
        const bool act = c < C && pt < it.w;
        int wts[3];
        prim_point_weights(dim, n, it.y + (act ? pt : 0), wts);
        const IfaceCopy& cp = copies[it.x + (act ? c : 0)];
        int i, j, k;
        copy_local_ijk(cp, dim, wts, i, j, k);
        clane[(size_t)q * 32 + lane] =
            uint2{(uint32_t)i | ((uint32_t)j << 10) | ((uint32_t)k << 20) | ((uint32_t)dirichlet << 30),
                  (uint32_t)cp.cell | ((uint32_t)C << 24) | ((uint32_t)act << 30)};
      }
    }
    if (int r = upload(&L.clane, clane)) return r;
  }
  // the same items restricted to primitives with two or more copies (the
  // streaming kernel forms every single-copy point inside its runs)
  std::vector<int4> mitems;
  for (int q = 0; q < (int)prims.size(); ++q) {
    const IfacePrim& P = prims[q];
    if (P.ncopies < 2) continue;
    const int meta = P.dim | (P.ncopies << 4) | (P.dirichlet << 12);
    const int per = P.ncopies <= 32 ? 32 / P.ncopies : 32;
    const int np = prim_points(P.dim, n);
    for (int p0 = 0; p0 < np; p0 += per) mitems.push_back({P.first_copy, p0, meta, std::min(per, np - p0)});
    if (!P.dirichlet) L.n_mitems_inner = (int)mitems.size();
  }
  L.n_mitems = (int)mitems.size();
  if (int r = upload(&L.mitems, mitems)) return r;
  // per item and lane (copy-major: lane = c * P + pt, copy c of point pt, P =
  // 32 / C points, so that one copy's lanes hold consecutive points of the
  // primitive in one cell): the copy's stored index and its class-stencil row
  // cell * 16 + class ({-1, 0}: no copy; items of primitives with more than 32
  // copies derive theirs in the kernel)
  {
    std::vector<int2> ml((size_t)L.n_mitems * 32, int2{-1, 0});
    for (int q = 0; q < L.n_mitems; ++q) {
      const int4 it = mitems[q];
      const int dim = it.z & 15, C = (it.z >> 4) & 255;
      if (C > 32) continue;
      const int P = 32 / C;
      for (int lane = 0; lane < 32; ++lane) {
        const int c = lane / P, pt = lane - c * P;
        if (c >= C || pt >= it.w) continue;
        int wts[3];
        prim_point_weights(dim, n, it.y + pt, wts);
        const IfaceCopy& cp = copies[it.x + c];
        int i, j, k;
        copy_local_ijk(cp, dim, wts, i, j, k);
        const int64_t g = (int64_t)cp.cell * L.cell_stride + tw(w, i, j, k);
        ml[(size_t)q * 32 + lane] = int2{(int)g, cp.cell * 16 + point_class(n, i, j, k)};
      }
    }
    if (int r = upload(&L.mlanes, ml)) return r;
  }
  {
    // the streaming kernel's plans, one per element size
    int dev = 0, sms = 0;
    HG_CUDA(cudaGetDevice(&dev));
    HG_CUDA(cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev));
    const int nctas = stream_ctas(n, (int)mesh->nc, L.n_mitems, sms);
    for (int dt = 0; dt < 2; ++dt) {
      StreamPlanHost P;
      if (int r = stream_plan(n, (int)mesh->nc, nctas, dt == HG_F64 ? 8 : 4, P)) return r;
      StreamPlanDev& D = L.splan[dt];
      D.nctas = nctas;
      D.band_rows = P.band_rows;
      if (int r = upload(&D.copies, P.copies)) return r;
      if (int r = upload(&D.items, P.items)) return r;
      if (int r = upload(&D.cta_copies, P.cta_copies)) return r;
      if (int r = upload(&D.cta_items, P.cta_items)) return r;
    }
  }
  const std::vector<int4> ptiles = plane_tiles(n);
  L.n_ptiles_cell = (int)ptiles.size();
  if (int r = upload(&L.ptiles, ptiles)) return r;
  const std::vector<int2> march = march_items(n);
  L.n_march_cell = (int)march.size();
  if (int r = upload(&L.march, march)) return r;
  // canonical numbering by exact lattice coordinates
  if (mesh->grid_denom) {
    std::vector<int64_t> keys(L.n_stored, -1);
    const int64_t off = 1 << 20;
    for (int64_t c = 0; c < mesh->nc; ++c) {
      const int64_t* X[4];
      for (int m = 0; m < 4; ++m) X[m] = &mesh->ixyz[3 * mesh->cells[c][m]];
      for (int k = 0; k <= n; ++k)
        for (int j = 0; j + k <= n; ++j)
          for (int i = 0; i + j + k <= n; ++i) {
            int64_t P[3];
            for (int r = 0; r < 3; ++r)
              P[r] = X[0][r] * n + i * (X[1][r] - X[0][r]) + j * (X[2][r] - X[0][r]) +
                     k * (X[3][r] - X[0][r]) + off;
            keys[c * L.cell_stride + tw(w, i, j, k)] = (P[2] << 42) | (P[1] << 21) | P[0];
          }
    }
    std::vector<int64_t> uniq;
    uniq.reserve(L.n_stored);
    for (int64_t kk : keys)
      if (kk >= 0) uniq.push_back(kk);
    std::sort(uniq.begin(), uniq.end());
    uniq.erase(std::unique(uniq.begin(), uniq.end()), uniq.end());
    L.n_unique = (int64_t)uniq.size();
    std::vector<int32_t> canon(L.n_stored, -1);
    std::vector<int64_t> rep(L.n_unique, -1);
    std::vector<uint8_t> dir(L.n_unique, 0);
    for (int64_t c = 0; c < mesh->nc; ++c)
      for (int k = 0; k <= n; ++k)
        for (int j = 0; j + k <= n; ++j)
          for (int i = 0; i + j + k <= n; ++i) {
            int64_t s = c * L.cell_stride + tw(w, i, j, k);
            int64_t u = std::lower_bound(uniq.begin(), uniq.end(), keys[s]) - uniq.begin();
            canon[s] = (int32_t)u;
            if (rep[u] < 0) rep[u] = s;
            dir[u] = (fl[16 * c + point_class(n, i, j, k)] & CF_DIRICHLET) ? 1 : 0;
          }
    H.canon = canon;
    H.canon_rep = rep;
    // Gauss-Seidel colours of the exact lattice points
    if (mesh->gs_abc[0] >= 0) {
      const int a = mesh->gs_abc[0], b = mesh->gs_abc[1], cc = mesh->gs_abc[2];
      std::vector<uint8_t> col(L.n_stored, 0);
      for (int64_t c = 0; c < mesh->nc; ++c) {
        const int64_t* X[4];
        for (int m = 0; m < 4; ++m) X[m] = &mesh->ixyz[3 * mesh->cells[c][m]];
        for (int k = 0; k <= n; ++k)
          for (int j = 0; j + k <= n; ++j)
            for (int i = 0; i + j + k <= n; ++i) {
              int64_t P[3];
              for (int r = 0; r < 3; ++r)
                P[r] = X[0][r] * n + i * (X[1][r] - X[0][r]) + j * (X[2][r] - X[0][r]) +
                       k * (X[3][r] - X[0][r]);
              const int64_t v = a * P[0] + b * P[1] + cc * P[2];
              col[c * L.cell_stride + tw(w, i, j, k)] = (uint8_t)(((v % 4) + 4) % 4);
            }
      }
      H.colour = col;
      if (int r = upload(&L.colour, col)) return r;
    }
    H.dirichlet = dir;
    H.canon_keys = uniq;
    H.canon_xyz.resize(3 * L.n_unique);
    const double den = (double)mesh->grid_denom * n;
    for (int64_t u = 0; u < L.n_unique; ++u) {
      int64_t kk = uniq[u];
      H.canon_xyz[3 * u + 0] = (double)((kk & ((1 << 21) - 1)) - off) / den;
      H.canon_xyz[3 * u + 1] = (double)(((kk >> 21) & ((1 << 21) - 1)) - off) / den;
      H.canon_xyz[3 * u + 2] = (double)((kk >> 42) - off) / den;
    }
    L.n_inner = 0;
    for (auto d : dir) L.n_inner += d == 0;
    if (int r = upload(&L.canon, canon)) return r;
    if (int r = upload(&L.canon_rep, rep)) return r;
  } else {
    // without an exact lattice the unique count follows from the primitive graph
    int64_t nu = (int64_t)mesh->nc * ntet(n - 3) + (int64_t)mesh->faces.size() * ntri(n - 2) +
                 (int64_t)mesh->edges.size() * std::max(n - 1, 0) + mesh->nv;
    L.n_unique = nu;
    int64_t nb = 0;
    for (auto& f : mesh->faces) nb += f.dirichlet ? ntri(n - 2) : 0;
    for (auto& e : mesh->edges) nb += e.dirichlet ? std::max(n - 1, 0) : 0;
    for (auto& v : mesh->verts) nb += v.dirichlet;
    L.n_inner = nu - nb;
  }
  // every table a kernel reads must be on the device
  if (!L.cls_flags || (L.n_prims && (!L.prims || !L.copies || !L.prim_point_base)) ||
      (L.n_items && (!L.items || !L.item_prim)) ||
      (L.n_citems && (!L.citems || !L.clane)) || (L.n_ptiles_cell && !L.ptiles) ||
      (L.n_march_cell && !L.march) ||
      (L.n_mitems && (!L.mitems || !L.mlanes)) || !L.splan[0].cta_items || !L.splan[1].cta_items ||
      (mesh->grid_denom && (!L.canon || !L.canon_rep))) {
    set_error("internal: level %d device tables incomplete", l);
    return HG_ERR_CUDA;
  }
  return HG_OK;
}

void Mesh::find_colouring() {
  gs_abc[0] = -1;
  if (!grid_denom) return;
  static const int dirs[7][3] = {{1, 0, 0}, {0, 1, 0}, {0, 0, 1}, {-1, 1, 0},
                                 {-1, 0, 1}, {0, -1, 1}, {1, -1, 1}};
  for (int a = 0; a < 4; ++a)
    for (int b = 0; b < 4; ++b)
      for (int c = 0; c < 4; ++c) {
        bool ok = true;
        for (int64_t e = 0; e < nc && ok; ++e) {
          const int64_t* X[4];
          for (int m = 0; m < 4; ++m) X[m] = &ixyz[3 * cells[e][m]];
          for (int d = 0; d < 7 && ok; ++d) {
            int64_t g[3];
            for (int r = 0; r < 3; ++r)
              g[r] = dirs[d][0] * (X[1][r] - X[0][r]) + dirs[d][1] * (X[2][r] - X[0][r]) +
                     dirs[d][2] * (X[3][r] - X[0][r]);
            const int64_t v = a * g[0] + b * g[1] + c * g[2];
            if (((v % 4) + 4) % 4 == 0) ok = false;
          }
        }
        if (ok) {
          gs_abc[0] = a;
          gs_abc[1] = b;
          gs_abc[2] = c;
          return;
        }
      }
}

// Limits of the per-level tables, checked on the finest lattice before
// anything is allocated: the stored->canonical map and the row items are
// int32; the canonical keys pack each exact lattice coordinate (vertex
// coordinate x D x 2^level) into 21 bits around an offset of 2^20; interface
// items keep a primitive's copy count in 8 bits.
int Hier::check_limits() const {
  const int64_t n = int64_t(1) << lmax;
  const int64_t n_stored = (ntet(n + 1) + 32 + 31) / 32 * 32 * mesh->nc;
  if (n_stored > INT32_MAX) {
    set_error("level %d of %lld cells has %lld stored points; at most 2^31 - 1 are supported",
              lmax, (long long)mesh->nc, (long long)n_stored);
    return HG_ERR_UNSUPPORTED;
  }
  if (mesh->grid_denom) {
    int64_t amax = 0;
    for (int64_t x : mesh->ixyz) amax = std::max(amax, x < 0 ? -x : x);
    if (amax * n >= (int64_t(1) << 20)) {
      set_error("lattice coordinates reach %lld at level %d (vertex coordinates x %d x 2^%d); the "
                "canonical numbering holds magnitudes below 2^20: scale the mesh down",
                (long long)(amax * n), lmax, mesh->grid_denom, lmax);
      return HG_ERR_UNSUPPORTED;
    }
  }
  if (mesh->nc >= (int64_t(1) << 24)) {
    set_error("%lld macro cells; at most 2^24 - 1 are supported (24-bit cell ids of the apply "
              "items)", (long long)mesh->nc);
    return HG_ERR_UNSUPPORTED;
  }
  for (const auto* prims : {&mesh->faces, &mesh->edges, &mesh->verts})
    for (const auto& p : *prims)
      if (p.cells.size() > 255) {
        set_error("a macro primitive is shared by %zu cells; at most 255 are supported",
                  p.cells.size());
        return HG_ERR_UNSUPPORTED;
      }
  return HG_OK;
}

int Hier::build(const Mesh* m, int lmin_, int lmax_) {
  mesh = m;
  const_cast<Mesh*>(m)->find_colouring();
  lmin = lmin_;
  lmax = lmax_;
  if (int r = check_limits()) return r;
  lv.resize(lmax - lmin + 1);
  HG_CUDA(cudaMalloc(&err_dev, sizeof(int)));
  HG_CUDA(cudaMemset(err_dev, 0, sizeof(int)));
  HG_CUDA(cudaMallocHost(&err_host, sizeof(int)));
  *err_host = 0;
  int64_t scratch = 0;
  for (int l = lmin; l <= lmax; ++l) {
    if (int r = build_level(l)) return r;
    lv[l - lmin].dev.err = err_dev;
    scratch = std::max(scratch, dot_scratch_len(lv[l - lmin].dev));
  }
  HG_CUDA(cudaMalloc(&dot_scratch, scratch * sizeof(double)));
  HG_CUDA(cudaMalloc(&dot_result, sizeof(double)));
  HG_CUDA(cudaMallocHost(&dot_host, sizeof(double)));
  return HG_OK;
}

int Hier::fetch_error(cudaStream_t s) const {
  HG_CUDA(cudaMemcpyAsync(err_host, err_dev, sizeof(int), cudaMemcpyDeviceToHost, s));
  return HG_OK;
}

int Hier::check_error() const {
  if (*err_host == 0) return HG_OK;
  const int code = *err_host;
  *err_host = 0;
  cudaMemset(err_dev, 0, sizeof(int));
  set_error("a kernel gave up a bounded wait (device error %d)", code);
  return HG_ERR_TIMEOUT;
}

Hier::~Hier() {
  for (auto& H : lv) {
    LevelDev& L = H.dev;
    cudaFree(L.cls_flags);
    cudaFree(L.canon);
    cudaFree(L.canon_rep);
    cudaFree(L.prims);
    cudaFree(L.copies);
    cudaFree(L.prim_point_base);
    cudaFree(L.citems);
    cudaFree(L.clane);
    cudaFree(L.mitems);
    cudaFree(L.mlanes);
    for (auto& D : L.splan) {
      cudaFree(D.copies);
      cudaFree(D.items);
      cudaFree(D.cta_copies);
      cudaFree(D.cta_items);
    }
    cudaFree(L.colour);
    cudaFree(L.ptiles);
    cudaFree(L.march);
    cudaFree(L.items);
    cudaFree(L.item_prim);
  }
  cudaFree(dot_scratch);
  cudaFree(dot_result);
  if (dot_host) cudaFreeHost(dot_host);
  cudaFree(err_dev);
  if (err_host) cudaFreeHost(err_host);
}

// --------------------------------------------------- element matrices
// The six micro-cell subgroups (Sec. 3.2): vertex offsets of the cell
// anchored at p, and the polytope side length w = n - delta.
const int kTypeOff[6][4][3] = {
    {{0, 0, 0}, {1, 0, 0}, {0, 1, 0}, {0, 0, 1}},  // I-up (w = n)
    {{1, 1, 0}, {1, 0, 1}, {0, 1, 1}, {1, 1, 1}},  // I-down (w = n-2)
    {{0, 1, 0}, {1, 0, 1}, {1, 0, 0}, {0, 0, 1}},  // octahedral, w = n-1 (4 cells around
    {{0, 1, 0}, {1, 0, 1}, {0, 0, 1}, {0, 1, 1}},  // the inner edge p+e2 -- p+e1+e3)
    {{0, 1, 0}, {1, 0, 1}, {0, 1, 1}, {1, 1, 0}},
    {{0, 1, 0}, {1, 0, 1}, {1, 1, 0}, {1, 0, 0}}};
const int kTypeDelta[6] = {0, 2, 1, 1, 1, 1};
const int kEdgeVerts[6][2] = {{0, 1}, {0, 2}, {0, 3}, {1, 2}, {1, 3}, {2, 3}};

void micro_cell_coords(const Mesh& m, int64_t c, int n, int type, double X[4][3]) {
  const double* V[4];
  for (int q = 0; q < 4; ++q) V[q] = &m.xyz[3 * m.cells[c][q]];
  for (int a = 0; a < 4; ++a)
    for (int r = 0; r < 3; ++r) {
      const int* o = kTypeOff[type][a];
      X[a][r] = V[0][r] + (o[0] * (V[1][r] - V[0][r]) + o[1] * (V[2][r] - V[0][r]) +
                           o[2] * (V[3][r] - V[0][r])) / (double)n;
    }
}

// Barycentric gradients G[4][3] and volume of a tetrahedron.
void bary_gradients(const double X[4][3], double G[4][3], double* vol) {
  double J[3][3];
  for (int r = 0; r < 3; ++r)
    for (int col = 0; col < 3; ++col) J[r][col] = X[col + 1][r] - X[0][r];
  double det = J[0][0] * (J[1][1] * J[2][2] - J[1][2] * J[2][1]) -
               J[0][1] * (J[1][0] * J[2][2] - J[1][2] * J[2][0]) +
               J[0][2] * (J[1][0] * J[2][1] - J[1][1] * J[2][0]);
  double inv[3][3];
  inv[0][0] = (J[1][1] * J[2][2] - J[1][2] * J[2][1]) / det;
  inv[0][1] = (J[0][2] * J[2][1] - J[0][1] * J[2][2]) / det;
  inv[0][2] = (J[0][1] * J[1][2] - J[0][2] * J[1][1]) / det;
  inv[1][0] = (J[1][2] * J[2][0] - J[1][0] * J[2][2]) / det;
  inv[1][1] = (J[0][0] * J[2][2] - J[0][2] * J[2][0]) / det;
  inv[1][2] = (J[0][2] * J[1][0] - J[0][0] * J[1][2]) / det;
  inv[2][0] = (J[1][0] * J[2][1] - J[1][1] * J[2][0]) / det;
  inv[2][1] = (J[0][1] * J[2][0] - J[0][0] * J[2][1]) / det;
  inv[2][2] = (J[0][0] * J[1][1] - J[0][1] * J[1][0]) / det;
  for (int d = 0; d < 3; ++d) {
    G[0][d] = 0;
    for (int q = 0; q < 3; ++q) {
      G[q + 1][d] = inv[q][d];
      G[0][d] -= inv[q][d];
    }
  }
  *vol = std::fabs(det) / 6.0;
}

void p1_element_matrix(int kind, const double X[4][3], double K[4][4]) {
  double G[4][3], vol;
  bary_gradients(X, G, &vol);
  for (int a = 0; a < 4; ++a)
    for (int b = 0; b < 4; ++b) {
      if (kind == HG_OP_P1_MASS) {
        K[a][b] = vol * (a == b ? 2.0 : 1.0) / 20.0;
      } else {
        K[a][b] = vol * (G[a][0] * G[b][0] + G[a][1] * G[b][1] + G[a][2] * G[b][2]);
      }
    }
}

int dir_index(int di, int dj, int dk) {
  for (int d = 0; d < kNDir; ++d) {
    int a, b, c;
    dir_offset(d, a, b, c);
    if (a == di && b == dj && c == dk) return d;
  }
  return -1;
}

// Is the micro-cell of `type` that has the point in class `cls` as its corner
// `a` inside the macro cell?  Exact for the six subgroups (see kTypeOff).
bool incident_inside(int cls, int type, int a) {
  const int* o = kTypeOff[type][a];
  for (int r = 0; r < 3; ++r)
    if (o[r] && (cls >> (r + 1) & 1)) return false;  // needs coordinate r >= 1
  int s = o[0] + o[1] + o[2];
  if (s == kTypeDelta[type] && (cls & 1)) return false;  // needs i+j+k <= n-1
  return true;
}

// Stencil tables S[cls][dir] of one macro cell at n intervals (FP64).
void p1_cell_stencils(const Mesh& m, int64_t c, int n, int kind, double S[16][16]) {
  double K[6][4][4];
  for (int t = 0; t < 6; ++t) {
    double X[4][3];
    micro_cell_coords(m, c, n, t, X);
    p1_element_matrix(kind, X, K[t]);
  }
  for (int cls = 0; cls < 16; ++cls) {
    for (int d = 0; d < 16; ++d) S[cls][d] = 0.0;
    for (int t = 0; t < 6; ++t)
      for (int a = 0; a < 4; ++a) {
        if (!incident_inside(cls, t, a)) continue;
        for (int b = 0; b < 4; ++b) {
          const int* oa = kTypeOff[t][a];
          const int* ob = kTypeOff[t][b];
          int d = dir_index(ob[0] - oa[0], ob[1] - oa[1], ob[2] - oa[2]);
          S[cls][d] += K[t][a][b];
        }
      }
  }
}

// Plane-window tiles of one cell lattice with n intervals: in plane k
// (1..n-3) the interior points lie in the cell-local offset range
// [rs(1,k)+1, rs(n-k-2,k)+1]; a window covers 30 consecutive offsets (lanes
// 1..30, halo lanes 0 and 31), a tile up to kPlaneSteps windows; a tile is
// (k | windows << 16, lane-0 offset, j0 << 16 | i0, 0) with (j0, i0) the
// lattice row and column of lane 0's offset.
// Column-march items: the cell-interior points (i, j, k >= 1, i + j + k <= n-1)
// of plane k in strips of 32 columns i0..i0+31 (i0 = 1, 33, ...), each strip
// cut into bands of kMarchRows rows j0..j1-1 that hold at least one interior
// point of column i0: (k | i0 << 16, j0 | j1 << 16).
std::vector<int2> march_items(int n) {
  std::vector<int2> v;
  for (int k = 1; k <= n - 3; ++k)
    for (int i0 = 1; i0 <= n - 2 - k; i0 += 32) {
      const int jmax = n - 1 - k - i0;
      for (int j0 = 1; j0 <= jmax; j0 += kMarchRows)
        v.push_back({k | (i0 << 16), j0 | (std::min(j0 + kMarchRows, jmax + 1) << 16)});
    }
  return v;
}

std::vector<int4> plane_tiles(int n) {
  const int w = n + 1;
  std::vector<int4> ptiles;
  for (int k = 1; k <= n - 3; ++k) {
    const int ga = (int)row_start(w, 1, k) + 1, gb = (int)row_start(w, n - k - 2, k) + 1;
    const int nwin = (gb - ga + 1 + 29) / 30;
    for (int t0 = 0; t0 < nwin; t0 += kPlaneSteps) {
      const int z = ga - 1 + 30 * t0;
      int j = 0, r = z - (int)row_start(w, 0, k), len = w - k;
      while (r >= len) { r -= len; --len; ++j; }
      ptiles.push_back({k | (std::min(kPlaneSteps, nwin - t0) << 16), z, (j << 16) | r, 0});
    }
  }
  return ptiles;
}

int lattice_index(const Hier* h, int space, int level) {
  const int lat = space == HG_SPACE_P2 ? level + 1 : level;
  if (space != HG_SPACE_P1 && space != HG_SPACE_P2) return -1;
  if (level < 0 || lat < h->lmin || lat > h->lmax) return -1;
  return lat - h->lmin;
}

int Op::build(const Hier* h, int kind_, const double* coeff) {
  hier = h;
  kind = kind_;
  lmin = h->lmin;
  lmax = h->lmax;
  if (kind == HG_OP_P2_LAPLACE || kind == HG_OP_P2_MASS || kind == HG_OP_P2_DIVKGRAD)
    return build_p2(coeff);
  if (kind == HG_OP_N1_CURLCURL) return build_n1(coeff);
  if (kind == HG_OP_P1_DIVKGRAD) return build_divkgrad(coeff);
  if (kind == HG_OP_P1_DIVKGRAD_STORED) {
    if (int r = build_divkgrad(coeff)) return r;
    return build_stored();
  }
  if (kind == HG_OP_P1_DIVKGRAD_SURROGATE) {
    set_error("HG_OP_P1_DIVKGRAD_SURROGATE operators are made by hg_op_create_surrogate");
    return HG_ERR_INVALID_ARG;
  }
  if (kind != HG_OP_P1_LAPLACE && kind != HG_OP_P1_MASS) {
    set_error("operator kind %d not available in this build", kind);
    return HG_ERR_UNSUPPORTED;
  }
  sten64.resize(h->lmax - h->lmin + 1, nullptr);
  sten32.resize(h->lmax - h->lmin + 1, nullptr);
  pattern.assign(h->lmax - h->lmin + 1, 0);
  for (int l = h->lmin; l <= h->lmax; ++l) {
    const int n = 1 << l;
    std::vector<double> s64(256 * h->mesh->nc);
    std::vector<float> s32(256 * h->mesh->nc);
    bool pat7 = true;
    for (int64_t c = 0; c < h->mesh->nc; ++c) {
      double S[16][16];
      p1_cell_stencils(*h->mesh, c, n, kind, S);
      for (int q = 0; q < 256; ++q) {
        s64[256 * c + q] = S[q / 16][q % 16];
        s32[256 * c + q] = (float)S[q / 16][q % 16];
      }
      // interior stencil (class 0) exactly zero outside the seven-point subset?
      for (int d = 0; d < kNDir; ++d)
        if (!((kPat7Mask >> d) & 1u) && S[0][d] != 0.0) pat7 = false;
    }
    pattern[l - h->lmin] = pat7 ? kPat7 : 0;
    if (int r = upload(&sten64[l - h->lmin], s64)) return r;
    if (int r = upload(&sten32[l - h->lmin], s32)) return r;
    // 1/diag(A) at every stored copy (sum of the copies' stencil centres)
    const LevelHost& H = h->lv[l - h->lmin];
    const LevelDev& L = H.dev;
    if (h->mesh->grid_denom) {
      std::vector<double> du(L.n_unique, 0.0);
      for (int64_t c = 0; c < h->mesh->nc; ++c)
        for (int k = 0; k <= n; ++k)
          for (int j = 0; j + k <= n; ++j)
            for (int i = 0; i + j + k <= n; ++i) {
              const int64_t q = c * L.cell_stride + tw(n + 1, i, j, k);
              du[H.canon[q]] += s64[256 * c + 16 * point_class(n, i, j, k)];
            }
      std::vector<double> inv(L.n_stored, 0.0);
      std::vector<float> inv32(L.n_stored, 0.0f);
      for (int64_t q = 0; q < L.n_stored; ++q)
        if (H.canon[q] >= 0 && du[H.canon[q]] != 0.0) {
          inv[q] = 1.0 / du[H.canon[q]];
          inv32[q] = (float)inv[q];
        }
      if (vinv[0].empty()) {
        vinv[0].assign(h->lmax - h->lmin + 1, nullptr);
        vinv[1].assign(h->lmax - h->lmin + 1, nullptr);
      }
      double* d = nullptr;
      float* f = nullptr;
      if (int r = upload(&d, inv)) return r;
      if (int r = upload(&f, inv32)) return r;
      vinv[HG_F64][l - h->lmin] = d;
      vinv[HG_F32][l - h->lmin] = f;
    }
  }
  return HG_OK;
}

// -div(k grad) with k at the vertices: per level the coefficient is the
// finest-level value at the same lattice point (injection), the element
// matrices of the six micro-cell types are computed per macro cell, and
// 1/diag(A) comes from the operator's own diagonal kernel.
int Op::build_divkgrad(const double* coeff) {
  const Hier* h = hier;
  if (!coeff) {
    set_error("HG_OP_P1_DIVKGRAD needs the coefficient at the finest-level vertices");
    return HG_ERR_INVALID_ARG;
  }
  if (!h->mesh->grid_denom) {
    set_error("HG_OP_P1_DIVKGRAD needs vertex coordinates on an exact lattice");
    return HG_ERR_UNSUPPORTED;
  }
  // -div(k grad) is elliptic only for k > 0 (a nonpositive or non-finite
  // value would make the operator indefinite or undefined)
  const int64_t nk = h->lv[h->lmax - h->lmin].dev.n_unique;
  for (int64_t u = 0; u < nk; ++u)
    if (!(coeff[u] > 0.0) || !std::isfinite(coeff[u])) {
      set_error("HG_OP_P1_DIVKGRAD: k must be positive and finite; canonical vertex %lld of level "
                "%d has %g", (long long)u, h->lmax, coeff[u]);
      return HG_ERR_INVALID_ARG;
    }
  const int nl = h->lmax - h->lmin + 1;
  for (int dt = 0; dt < 2; ++dt) {
    vk[dt].assign(nl, nullptr);
    vK[dt].assign(nl, nullptr);
    vinv[dt].assign(nl, nullptr);
  }
  const LevelHost& F = h->lv[h->lmax - h->lmin];
  const int64_t off = 1 << 20, m21 = (1 << 21) - 1;
  for (int l = h->lmin; l <= h->lmax; ++l) {
    const LevelHost& H = h->lv[l - h->lmin];
    const LevelDev& L = H.dev;
    const int shift = h->lmax - l;
    // coefficient at this level's canonical vertices, then at every stored copy
    std::vector<double> kc(L.n_unique), ks(L.n_stored, 0.0);
    for (int64_t u = 0; u < L.n_unique; ++u) {
      const int64_t key = H.canon_keys[u];
      const int64_t X = ((key & m21) - off) << shift, Y = (((key >> 21) & m21) - off) << shift,
                    Z = ((key >> 42) - off) << shift;
      const int64_t fk = ((Z + off) << 42) | ((Y + off) << 21) | (X + off);
      auto it = std::lower_bound(F.canon_keys.begin(), F.canon_keys.end(), fk);
      if (it == F.canon_keys.end() || *it != fk) {
        set_error("internal: level %d vertex not found on the finest level", l);
        return HG_ERR_INVALID_ARG;
      }
      kc[u] = coeff[it - F.canon_keys.begin()];
    }
    for (int64_t q = 0; q < L.n_stored; ++q)
      if (H.canon[q] >= 0) ks[q] = kc[H.canon[q]];
    // element-matrix rows of the 24 incidences (type t, corner a): row a of K_t
    const int n = 1 << l;
    std::vector<double> K(96 * h->mesh->nc);
    for (int64_t c = 0; c < h->mesh->nc; ++c)
      for (int t = 0; t < 6; ++t) {
        double X[4][3], Ke[4][4];
        micro_cell_coords(*h->mesh, c, n, t, X);
        p1_element_matrix(HG_OP_P1_LAPLACE, X, Ke);
        for (int a = 0; a < 4; ++a)
          for (int b = 0; b < 4; ++b) K[96 * c + 16 * t + 4 * a + b] = Ke[a][b];
      }
    std::vector<float> ks32(ks.begin(), ks.end()), K32(K.begin(), K.end());
    double* d = nullptr;
    float* f = nullptr;
    if (int r = upload(&d, ks)) return r;
    vk[HG_F64][l - h->lmin] = d;
    if (int r = upload(&d, K)) return r;
    vK[HG_F64][l - h->lmin] = d;
    if (int r = upload(&f, ks32)) return r;
    vk[HG_F32][l - h->lmin] = f;
    if (int r = upload(&f, K32)) return r;
    vK[HG_F32][l - h->lmin] = f;
    // diagonal (all DoFs, FP64) -> 1/diag where nonzero
    double* diag = nullptr;
    HG_CUDA(cudaMalloc(&diag, L.n_stored * sizeof(double)));
    HG_CUDA(cudaMemset(diag, 0, L.n_stored * sizeof(double)));
    StencilArgs a{};
    a.x = diag;  // unused by the diagonal mode, must be non-null
    a.out = diag;
    a.op = OP_DIAG;
    a.mask = HG_MASK_ALL;
    VarCoef vc{vk[HG_F64][l - h->lmin], vK[HG_F64][l - h->lmin], nullptr};
    if (int r = launch_p1_divkgrad(L, HG_F64, a, vc, 0)) return r;
    std::vector<double> dh(L.n_stored);
    HG_CUDA(cudaMemcpy(dh.data(), diag, L.n_stored * sizeof(double), cudaMemcpyDeviceToHost));
    cudaFree(diag);
    std::vector<double> inv(L.n_stored, 0.0);
    std::vector<float> inv32(L.n_stored, 0.0f);
    for (int64_t q = 0; q < L.n_stored; ++q)
      if (dh[q] != 0.0) {
        inv[q] = 1.0 / dh[q];
        inv32[q] = (float)inv[q];
      }
    if (int r = upload(&d, inv)) return r;
    vinv[HG_F64][l - h->lmin] = d;
    if (int r = upload(&f, inv32)) return r;
    vinv[HG_F32][l - h->lmin] = f;
  }
  return HG_OK;
}

// Grid-aware precomputation (Sec. 5.2): the div-k-grad stencil of every
// stored point, computed once per level in FP64 by the operator's own point
// sum and rounded to FP32 for the FP32 copy.
int Op::build_stored() {
  const Hier* h = hier;
  const int nl = h->lmax - h->lmin + 1;
  for (int dt = 0; dt < 2; ++dt) sst[dt].assign(nl, nullptr);
  for (int l = h->lmin; l <= h->lmax; ++l) {
    const int li = l - h->lmin;
    const LevelDev& L = h->lv[li].dev;
    const int64_t n = (int64_t)16 * L.n_stored;
    HG_CUDA(cudaMalloc(&sst[HG_F64][li], n * sizeof(double)));
    HG_CUDA(cudaMalloc(&sst[HG_F32][li], n * sizeof(float)));
    VarCoef vc{vk[HG_F64][li], vK[HG_F64][li], nullptr};
    if (int r = launch_divkgrad_stencil(L, HG_F64, vc, sst[HG_F64][li], 0)) return r;
    if (int r = launch_demote_scaled(n, (const double*)sst[HG_F64][li], 1.0,
                                     (float*)sst[HG_F32][li], 0))
      return r;
    HG_CUDA(cudaDeviceSynchronize());
  }
  return HG_OK;
}

// Polynomial surrogate stencils (Sec. 5.2, surrogate operators).  Per level:
// the interior points p of a cell (i, j, k >= 1, i + j + k <= n - 1, order
// k, j, i) and the polynomial basis at them, B[p][t] = xi^a eta^b zeta^c
// (xi = i/n - 1/4, ...; terms by a, then b, then c; a + b + c <= degree);
// B = Q R by modified Gram-Schmidt with a second orthogonalisation pass,
// columns that the points do not separate (residual below 1e-9 of their
// norm) dropped; the exact stencils S of every stored point (FP64, the
// operator's own point sum); on the device M = Q^T S per cell and direction;
// on the host the coefficients c = R^-1 M of the kept terms (0 for the
// dropped ones).  The fitted weights B c are the least-squares projection of
// the exact ones.  Then the surrogate's own diagonal replaces the exact one.
int Op::build_surrogate(const double* coeff, int degree) {
  const Hier* h = hier;
  if (degree < 0 || degree > kSurMaxDegree) {
    set_error("surrogate degree %d outside 0..%d", degree, kSurMaxDegree);
    return HG_ERR_INVALID_ARG;
  }
  if (h->lmax > 9) {
    set_error("surrogate: level %d beyond the row encoding", h->lmax);
    return HG_ERR_UNSUPPORTED;
  }
  if (int r = build_divkgrad(coeff)) return r;
  sdeg = degree;
  const int nt = sur_nterm(degree);
  const int nl = h->lmax - h->lmin + 1;
  const int64_t nc = h->mesh->nc;
  for (int dt = 0; dt < 2; ++dt) scoef[dt].assign(nl, nullptr);
  ssegs.assign(nl, nullptr);
  n_ssegs.assign(nl, 0);
  spat.assign(nl, 0);
  for (int l = h->lmin; l <= h->lmax; ++l) {
    const int li = l - h->lmin;
    const LevelDev& L = h->lv[li].dev;
    const int n = 1 << l, w = n + 1;
    std::vector<int> pidx, segs;
    std::vector<double> B;
    for (int k = 1; k <= n - 1; ++k)
      for (int j = 1; j + k <= n - 1; ++j) {
        if ((j - 1) % kSurRows == 0 && j + k <= n - 2)
          segs.push_back(j | (k << 10) | (std::min(j + kSurRows, n - 1 - k) << 20));
        for (int i = 1; i + j + k <= n - 1; ++i) {
          pidx.push_back((int)tw(w, i, j, k));
          const double v[3] = {(double)i / n - 0.25, (double)j / n - 0.25, (double)k / n - 0.25};
          for (int a = 0; a <= degree; ++a)
            for (int b = 0; a + b <= degree; ++b)
              for (int c = 0; a + b + c <= degree; ++c)
                B.push_back(std::pow(v[0], a) * std::pow(v[1], b) * std::pow(v[2], c));
        }
      }
    const int64_t P = (int64_t)pidx.size();
    n_ssegs[li] = (int)segs.size();
    if (!segs.empty())
      if (int r = upload(&ssegs[li], segs)) return r;
    std::vector<double> coef(nc * kNDir * nt, 0.0);
    if (P > 0) {
      // modified Gram-Schmidt on the columns of B, twice, dropping dependent ones
      std::vector<std::vector<double>> Qc;
      std::vector<int> kept;
      std::vector<std::vector<double>> Rc;  // column t' of R (length t'+1)
      for (int t = 0; t < nt; ++t) {
        std::vector<double> v(P);
        double n0 = 0.0;
        for (int64_t p = 0; p < P; ++p) {
          v[p] = B[p * nt + t];
          n0 += v[p] * v[p];
        }
        n0 = std::sqrt(n0);
        std::vector<double> rcol(Qc.size() + 1, 0.0);
        for (int pass = 0; pass < 2; ++pass)
          for (size_t s2 = 0; s2 < Qc.size(); ++s2) {
            double r = 0.0;
            for (int64_t p = 0; p < P; ++p) r += Qc[s2][p] * v[p];
            for (int64_t p = 0; p < P; ++p) v[p] -= r * Qc[s2][p];
            rcol[s2] += r;
          }
        double nv = 0.0;
        for (int64_t p = 0; p < P; ++p) nv += v[p] * v[p];
        nv = std::sqrt(nv);
        if (!(n0 > 0.0) || nv <= 1e-9 * n0) continue;
        for (int64_t p = 0; p < P; ++p) v[p] /= nv;
        rcol.back() = nv;
        Qc.push_back(std::move(v));
        Rc.push_back(std::move(rcol));
        kept.push_back(t);
      }
      const int T = (int)kept.size();
      std::vector<double> Q(P * T);
      for (int64_t p = 0; p < P; ++p)
        for (int t = 0; t < T; ++t) Q[p * T + t] = Qc[t][p];
      double *S = nullptr, *dQ = nullptr, *dM = nullptr;
      int* dp = nullptr;
      auto cleanup = [&]() {
        cudaFree(S);
        cudaFree(dQ);
        cudaFree(dM);
        cudaFree(dp);
      };
      int rc = HG_OK;
      std::vector<double> M(nc * kNDir * T);
      do {
        if (cudaMalloc(&S, (size_t)16 * L.n_stored * sizeof(double)) != cudaSuccess ||
            cudaMalloc(&dM, M.size() * sizeof(double)) != cudaSuccess) {
          set_error("surrogate: out of device memory for the fit of level %d", l);
          rc = HG_ERR_CUDA;
          break;
        }
        if ((rc = upload(&dQ, Q)) || (rc = upload(&dp, pidx))) break;
        VarCoef vc{vk[HG_F64][li], vK[HG_F64][li], nullptr};
        if ((rc = launch_divkgrad_stencil(L, HG_F64, vc, S, 0))) break;
        if ((rc = launch_surrogate_moments(L, S, dp, (int)P, dQ, T, dM, 0))) break;
        if (cudaMemcpy(M.data(), dM, M.size() * sizeof(double), cudaMemcpyDeviceToHost) !=
            cudaSuccess) {
          set_error("surrogate: %s", cudaGetErrorString(cudaGetLastError()));
          rc = HG_ERR_CUDA;
        }
      } while (0);
      cleanup();
      if (rc) return rc;
      // c = R^-1 (Q^T w) per cell and direction (back substitution)
      for (int64_t c = 0; c < nc; ++c)
        for (int d = 0; d < kNDir; ++d) {
          const double* m = &M[(c * kNDir + d) * T];
          std::vector<double> x(T);
          for (int t = T - 1; t >= 0; --t) {
            double r = m[t];
            for (int u = t + 1; u < T; ++u) r -= Rc[u][t] * x[u];
            x[t] = r / Rc[t][t];
          }
          for (int t = 0; t < T; ++t) coef[(c * kNDir + d) * nt + kept[t]] = x[t];
        }
    }
    // seven-point fit: every coefficient of the other eight directions is an
    // exact zero in every cell (the weights there are exact zeros, as on
    // Kuhn-ordered cubes)
    {
      bool pat7 = true;
      for (int64_t c = 0; c < nc && pat7; ++c)
        for (int d = 0; d < kNDir && pat7; ++d)
          if (!((kPat7Mask >> d) & 1u))
            for (int t = 0; t < nt; ++t)
              if (coef[(c * kNDir + d) * nt + t] != 0.0) {
                pat7 = false;
                break;
              }
      spat[li] = pat7 ? kPat7 : 0;
    }
    std::vector<float> coef32(coef.begin(), coef.end());
    double* d64 = nullptr;
    float* d32 = nullptr;
    if (int r = upload(&d64, coef)) return r;
    scoef[HG_F64][li] = d64;
    if (int r = upload(&d32, coef32)) return r;
    scoef[HG_F32][li] = d32;
    // the surrogate's diagonal (all DoFs, FP64) -> 1/diag where nonzero
    double* diag = nullptr;
    HG_CUDA(cudaMalloc(&diag, L.n_stored * sizeof(double)));
    HG_CUDA(cudaMemset(diag, 0, L.n_stored * sizeof(double)));
    StencilArgs a{};
    a.x = diag;  // unused by the diagonal mode, must be non-null
    a.out = diag;
    a.op = OP_DIAG;
    a.mask = HG_MASK_ALL;
    VarCoef vc{vk[HG_F64][li], vK[HG_F64][li], nullptr};
    SurCoef sc{degree, scoef[HG_F64][li], ssegs[li], n_ssegs[li], spat[li]};
    int rc = launch_p1_surrogate(L, HG_F64, a, vc, sc, 0);
    std::vector<double> dh(L.n_stored);
    if (!rc && cudaMemcpy(dh.data(), diag, L.n_stored * sizeof(double), cudaMemcpyDeviceToHost) !=
                   cudaSuccess) {
      set_error("surrogate: %s", cudaGetErrorString(cudaGetLastError()));
      rc = HG_ERR_CUDA;
    }
    cudaFree(diag);
    if (rc) return rc;
    std::vector<double> inv(L.n_stored, 0.0);
    std::vector<float> inv32(L.n_stored, 0.0f);
    for (int64_t q = 0; q < L.n_stored; ++q)
      if (dh[q] != 0.0) {
        inv[q] = 1.0 / dh[q];
        inv32[q] = (float)inv[q];
      }
    cudaFree(vinv[HG_F64][li]);
    cudaFree(vinv[HG_F32][li]);
    vinv[HG_F64][li] = vinv[HG_F32][li] = nullptr;
    if (int r = upload(&d64, inv)) return r;
    vinv[HG_F64][li] = d64;
    if (int r = upload(&d32, inv32)) return r;
    vinv[HG_F32][li] = d32;
  }
  return HG_OK;
}

int Op::launch(int level, int dtype, StencilArgs a, cudaStream_t s) const {
  if (space == HG_SPACE_P2) {
    const int li = level - lmin;
    P2Args P;
    P.n = 1 << level;
    P.ncells = (int)hier->mesh->nc;
    P.cells = p2cells[dtype][li];
    P.anchors = p2anchors[li];
    for (int c = 0; c < 9; ++c) P.anchor_off[c] = p2off[li][c];
    P.mode = p2mode;
    P.acc = p2acc[dtype][li];
    P.invdiag = p2inv[dtype][li];
    return launch_p2(dev(level), dtype, a, P, s);
  }
  const int li = level - hier->lmin;
  const LevelDev& L = hier->lv[li].dev;
  if (kind == HG_OP_P1_DIVKGRAD) {
    VarCoef vc{vk[dtype][li], vK[dtype][li], vinv[dtype][li]};
    return launch_p1_divkgrad(L, dtype, a, vc, s);
  }
  if (kind == HG_OP_P1_DIVKGRAD_SURROGATE) {
    VarCoef vc{vk[dtype][li], vK[dtype][li], vinv[dtype][li]};
    SurCoef sc{sdeg, scoef[dtype][li], ssegs[li], n_ssegs[li], spat[li]};
    return launch_p1_surrogate(L, dtype, a, vc, sc, s);
  }
  if (kind == HG_OP_P1_DIVKGRAD_STORED) {
    a.sten = nullptr;
    a.sst = sst[dtype][li];
    return launch_p1_const(L, dtype, a, s);
  }
  a.sten = dtype == HG_F64 ? (const void*)sten64[li] : (const void*)sten32[li];
  a.pattern = pattern[li];
  return launch_p1_const(L, dtype, a, s);
}

Op::~Op() {
  for (int dt = 0; dt < 2; ++dt)
    for (auto* v : {&p2cells[dt], &p2acc[dt], &p2inv[dt]})
      for (void* p : *v) cudaFree(p);
  for (auto p : p2anchors) cudaFree(p);
  for (auto p : sten64) cudaFree(p);
  for (auto p : sten32) cudaFree(p);
  for (int dt = 0; dt < 2; ++dt)
    for (auto* v : {&vk[dt], &vK[dt], &vinv[dt], &sst[dt], &scoef[dt]})
      for (void* p : *v) cudaFree(p);
  for (auto p : ssegs) cudaFree(p);
  cudaFree(n1sign);
}

}  // namespace hg

// ==================================================================== C ABI
using namespace hg;

struct hg_mesh : Mesh {};
struct hg_hier : Hier {};
struct hg_op : Op {};

#define HG_CHECK(cond, code, ...) \
  do {                            \
    if (!(cond)) {                \
      set_error(__VA_ARGS__);     \
      return code;                \
    }                             \
  } while (0)

extern "C" {

const char* hg_last_error(void) { return g_err.c_str(); }

int hg_mesh_create(const double* xyz, int64_t nv, const int64_t* cells, int64_t nc,
                   hg_mesh** out) {
  HG_CHECK(xyz && cells && out && nv >= 4 && nc >= 1, HG_ERR_INVALID_ARG,
           "hg_mesh_create: null pointer or empty mesh");
  g_err.clear();
  auto m = std::make_unique<hg_mesh>();
  if (int r = m->build(xyz, nv, cells, nc)) return r;
  *out = m.release();
  return HG_OK;
}

void hg_mesh_destroy(hg_mesh* mesh) { delete mesh; }

int hg_mesh_counts(const hg_mesh* m, int64_t counts[6]) {
  HG_CHECK(m && counts, HG_ERR_INVALID_ARG, "hg_mesh_counts: null argument");
  counts[0] = m->nv;
  counts[1] = (int64_t)m->edges.size();
  counts[2] = (int64_t)m->faces.size();
  counts[3] = m->nc;
  counts[4] = m->n_boundary_faces;
  counts[5] = (int64_t)m->faces.size() - m->n_boundary_faces;
  return HG_OK;
}

int hg_hier_create(const hg_mesh* mesh, int lmin, int lmax, hg_hier** out) {
  HG_CHECK(mesh && out, HG_ERR_INVALID_ARG, "hg_hier_create: null argument");
  HG_CHECK(0 <= lmin && lmin <= lmax && lmax <= 9, HG_ERR_LEVEL_RANGE,
           "hg_hier_create: need 0 <= lmin <= lmax <= 9, got %d..%d", lmin, lmax);
  auto h = std::make_unique<hg_hier>();
  if (int r = h->build(mesh, lmin, lmax)) return r;
  *out = h.release();
  return HG_OK;
}

void hg_hier_destroy(hg_hier* h) { delete h; }

int hg_function_size(const hg_hier* h, int space, int level, int64_t* n_stored,
                     int64_t* n_unique, int64_t* n_inner, int64_t* cell_stride) {
  HG_CHECK(h, HG_ERR_INVALID_ARG, "hg_function_size: null hierarchy");
  HG_CHECK(space == HG_SPACE_P1 || space == HG_SPACE_P2, HG_ERR_UNSUPPORTED,
           "space %d not available", space);
  const int li = lattice_index(h, space, level);
  HG_CHECK(li >= 0, HG_ERR_LEVEL_RANGE, "level %d of space %d outside the hierarchy %d..%d",
           level, space, h->lmin, h->lmax);
  const LevelDev& L = h->lv[li].dev;
  if (n_stored) *n_stored = L.n_stored;
  if (n_unique) *n_unique = L.n_unique;
  if (n_inner) *n_inner = L.n_inner;
  if (cell_stride) *cell_stride = L.cell_stride;
  return HG_OK;
}

int hg_canonical_info(const hg_hier* h, int space, int level, int64_t* s2c, double* xyz,
                      uint8_t* dirichlet) {
  HG_CHECK(h, HG_ERR_INVALID_ARG, "hg_canonical_info: null hierarchy");
  HG_CHECK(space == HG_SPACE_P1 || space == HG_SPACE_P2, HG_ERR_UNSUPPORTED,
           "space %d not available", space);
  const int li = lattice_index(h, space, level);
  HG_CHECK(li >= 0, HG_ERR_LEVEL_RANGE, "level out of range");
  HG_CHECK(h->mesh->grid_denom, HG_ERR_UNSUPPORTED,
           "canonical order needs vertex coordinates on a lattice of spacing 1/D, D <= 64");
  const LevelHost& H = h->lv[li];
  if (s2c)
    for (size_t q = 0; q < H.canon.size(); ++q) s2c[q] = H.canon[q];
  if (xyz) std::copy(H.canon_xyz.begin(), H.canon_xyz.end(), xyz);
  if (dirichlet) std::copy(H.dirichlet.begin(), H.dirichlet.end(), dirichlet);
  return HG_OK;
}

static const LevelDev* level_of(const Hier* h, int space, int level) {
  if (!h) {
    set_error("null hierarchy");
    return nullptr;
  }
  if (space != HG_SPACE_P1 && space != HG_SPACE_P2) {
    set_error("space %d not available", space);
    return nullptr;
  }
  const int li = lattice_index(h, space, level);
  if (li < 0) {
    set_error("level %d of space %d outside the hierarchy %d..%d", level, space, h->lmin,
              h->lmax);
    return nullptr;
  }
  return &h->lv[li].dev;
}

int hg_to_canonical(const hg_hier* h, int space, int level, int dtype, const void* st,
                    void* can, void* stream) {
  const LevelDev* L = level_of(h, space, level);
  if (!L) return HG_ERR_INVALID_ARG;
  HG_CHECK(h->mesh->grid_denom, HG_ERR_UNSUPPORTED, "mesh has no exact lattice");
  HG_CHECK(st && can && (dtype == HG_F32 || dtype == HG_F64), HG_ERR_INVALID_ARG,
           "hg_to_canonical: bad argument");
  return launch_to_canonical(*L, dtype, st, can, (cudaStream_t)stream);
}

int hg_from_canonical(const hg_hier* h, int space, int level, int dtype, const void* can,
                      void* st, void* stream) {
  const LevelDev* L = level_of(h, space, level);
  if (!L) return HG_ERR_INVALID_ARG;
  HG_CHECK(h->mesh->grid_denom, HG_ERR_UNSUPPORTED, "mesh has no exact lattice");
  HG_CHECK(st && can && (dtype == HG_F32 || dtype == HG_F64), HG_ERR_INVALID_ARG,
           "hg_from_canonical: bad argument");
  return launch_from_canonical(*L, dtype, can, st, (cudaStream_t)stream);
}

int hg_device_status(const hg_hier* h, void* stream) {
  HG_CHECK(h, HG_ERR_INVALID_ARG, "hg_device_status: null hierarchy");
  cudaStream_t s = (cudaStream_t)stream;
  if (int r = h->fetch_error(s)) return r;
  HG_CUDA(cudaStreamSynchronize(s));
  return h->check_error();
}

int hg_plane_tiles(int level, int* out, int* n_tiles) {
  HG_CHECK(level >= 0 && level <= 12 && n_tiles, HG_ERR_INVALID_ARG, "hg_plane_tiles: bad argument");
  const std::vector<int4> t = plane_tiles(1 << level);
  *n_tiles = (int)t.size();
  if (out)
    for (size_t q = 0; q < t.size(); ++q) {
      out[4 * q] = t[q].x;
      out[4 * q + 1] = t[q].y;
      out[4 * q + 2] = t[q].z;
      out[4 * q + 3] = t[q].w;
    }
  return HG_OK;
}

int hg_march_items(int level, int* out, int* n_items) {
  HG_CHECK(level >= 0 && level <= 12 && n_items, HG_ERR_INVALID_ARG, "hg_march_items: bad argument");
  const std::vector<int2> t = march_items(1 << level);
  *n_items = (int)t.size();
  if (out)
    for (size_t q = 0; q < t.size(); ++q) {
      out[2 * q] = t[q].x;
      out[2 * q + 1] = t[q].y;
    }
  return HG_OK;
}

int hg_set_p1_kernel(int mode) { return set_p1_kernel(mode); }

int hg_stream_plan(int level, int ncells, int nctas, int dtype, int* copies, int* items,
                   int* cta_copies, int* cta_items, int* counts) {
  HG_CHECK(level >= 0 && level <= 12 && ncells >= 1 && nctas >= 1 && counts &&
               (dtype == HG_F32 || dtype == HG_F64),
           HG_ERR_INVALID_ARG, "hg_stream_plan: bad argument");
  StreamPlanHost P;
  if (int r = stream_plan(1 << level, ncells, nctas, dtype == HG_F64 ? 8 : 4, P)) return r;
  counts[0] = (int)P.copies.size();
  counts[1] = (int)(P.items.size() / 3);
  counts[2] = P.band_rows;
  auto put = [](int* out, const std::vector<int4>& v) {
    if (out)
      for (size_t q = 0; q < v.size(); ++q) {
        out[4 * q] = v[q].x;
        out[4 * q + 1] = v[q].y;
        out[4 * q + 2] = v[q].z;
        out[4 * q + 3] = v[q].w;
      }
  };
  put(copies, P.copies);
  put(items, P.items);
  if (cta_copies) std::copy(P.cta_copies.begin(), P.cta_copies.end(), cta_copies);
  if (cta_items) std::copy(P.cta_items.begin(), P.cta_items.end(), cta_items);
  return HG_OK;
}

int hg_index_tw(int64_t w, int64_t i, int64_t j, int64_t k, int64_t* out) {
  HG_CHECK(out, HG_ERR_INVALID_ARG, "hg_index_tw: null output");
  // N_tet(w) = w (w+1) (w+2) / 6 must fit in int64: w <= 2^20
  HG_CHECK(w <= (int64_t(1) << 20), HG_ERR_INVALID_ARG,
           "hg_index_tw: w = %lld above 2^20 (N_tet(w) would overflow int64)", (long long)w);
  HG_CHECK(w >= 1 && i >= 0 && j >= 0 && k >= 0 && i + j + k < w, HG_ERR_INVALID_ARG,
           "hg_index_tw: (%lld,%lld,%lld) not in I_tet(%lld)", (long long)i, (long long)j,
           (long long)k, (long long)w);
  *out = tw(w, i, j, k);
  return HG_OK;
}

int hg_index_enumerate(int64_t w, int64_t* out, void* stream) {
  HG_CHECK(out && w >= 1 && w <= 1025, HG_ERR_INVALID_ARG, "hg_index_enumerate: bad argument");
  return launch_index_enumerate((int)w, out, (cudaStream_t)stream);
}

int hg_interface_dump(const hg_hier* h, int space, int level, int64_t* out, int64_t* n_rows,
                      int64_t* max_copies, void* stream) {
  const LevelDev* L = level_of(h, space, level);
  if (!L) return HG_ERR_INVALID_ARG;
  const LevelHost& H = h->lv[level - h->lmin];
  if (n_rows) *n_rows = H.prim_point_base.back();
  if (max_copies) *max_copies = L->max_copies;
  if (!out) return HG_OK;
  return launch_interface_dump(*L, out, (cudaStream_t)stream);
}

int hg_op_create(const hg_hier* h, int kind, const double* coeff, hg_op** out) {
  HG_CHECK(h && out, HG_ERR_INVALID_ARG, "hg_op_create: null argument");
  auto op = std::make_unique<hg_op>();
  if (int r = op->build(h, kind, coeff)) return r;
  *out = op.release();
  return HG_OK;
}

int hg_op_create_surrogate(const hg_hier* h, const double* k, int degree, hg_op** out) {
  HG_CHECK(h && out, HG_ERR_INVALID_ARG, "hg_op_create_surrogate: null argument");
  auto op = std::make_unique<hg_op>();
  op->hier = h;
  op->kind = HG_OP_P1_DIVKGRAD_SURROGATE;
  op->lmin = h->lmin;
  op->lmax = h->lmax;
  if (int r = op->build_surrogate(k, degree)) return r;
  *out = op.release();
  return HG_OK;
}

void hg_op_destroy(hg_op* op) { delete op; }

static int run_cell_op(const hg_op* op, int level, int dtype, StencilArgs a, cudaStream_t s) {
  HG_CHECK(op, HG_ERR_INVALID_ARG, "null operator");
  const LevelDev* L = level_of(op->hier, op->space, level);
  if (!L || level < op->lmin || level > op->lmax) return HG_ERR_LEVEL_RANGE;
  HG_CHECK(dtype == HG_F32 || dtype == HG_F64, HG_ERR_INVALID_ARG, "bad dtype %d", dtype);
  HG_CHECK(a.x && a.out && a.x != a.out, HG_ERR_INVALID_ARG,
           "input and output must be distinct non-null device pointers");
  HG_CHECK(((uintptr_t)a.x & 15) == 0, HG_ERR_INVALID_ARG,
           "input vector must be 16-byte aligned");
  return op->launch(level, dtype, a, s);
}

int hg_apply(const hg_op* op, int level, int dtype, const void* x, void* y, int mode, int mask,
             void* stream) {
  HG_CHECK(mode == HG_REPLACE || mode == HG_ADD, HG_ERR_INVALID_ARG, "bad mode %d", mode);
  HG_CHECK(mask == HG_MASK_INNER || mask == HG_MASK_ALL, HG_ERR_INVALID_ARG, "bad mask %d", mask);
  StencilArgs a{};
  a.x = x;
  a.out = y;
  a.op = OP_APPLY;
  a.mode = mode;
  a.mask = mask;
  return run_cell_op(op, level, dtype, a, (cudaStream_t)stream);
}

int hg_residual(const hg_op* op, int level, int dtype, const void* x, const void* b, void* r,
                void* stream) {
  HG_CHECK(b && b != r, HG_ERR_INVALID_ARG, "hg_residual: b must be distinct from r");
  StencilArgs a{};
  a.x = x;
  a.b = b;
  a.out = r;
  a.op = OP_RESID;
  a.mask = HG_MASK_INNER;
  return run_cell_op(op, level, dtype, a, (cudaStream_t)stream);
}

int hg_jacobi(const hg_op* op, int level, int dtype, double omega, const void* x, const void* b,
              void* x_out, void* stream) {
  HG_CHECK(b && b != x_out, HG_ERR_INVALID_ARG, "hg_jacobi: b must be distinct from x_out");
  StencilArgs a{};
  a.x = x;
  a.b = b;
  a.out = x_out;
  a.omega = omega;
  a.op = OP_JACOBI;
  a.mask = HG_MASK_INNER;
  return run_cell_op(op, level, dtype, a, (cudaStream_t)stream);
}

int hg_gauss_seidel(const hg_op* op, int level, int dtype, int colour, const void* x,
                    const void* b, void* x_out, void* stream) {
  HG_CHECK(op, HG_ERR_INVALID_ARG, "hg_gauss_seidel: null operator");
  HG_CHECK(op->space == HG_SPACE_P1, HG_ERR_UNSUPPORTED,
           "hg_gauss_seidel: P1 operators only (the colouring is of the P1 lattice coupling)");
  HG_CHECK(colour >= 0 && colour < 4, HG_ERR_INVALID_ARG, "hg_gauss_seidel: colour %d", colour);
  HG_CHECK(b && b != x_out, HG_ERR_INVALID_ARG, "hg_gauss_seidel: b must be distinct from x_out");
  const LevelDev* L = level_of(op->hier, op->space, level);
  HG_CHECK(L && L->colour, HG_ERR_UNSUPPORTED,
           "hg_gauss_seidel: this mesh admits no 4-colouring of the lattice");
  StencilArgs a{};
  a.x = x;
  a.b = b;
  a.out = x_out;
  a.op = OP_GS;
  a.mask = HG_MASK_INNER;
  a.colour = colour;
  return run_cell_op(op, level, dtype, a, (cudaStream_t)stream);
}

int hg_gs_colours(const hg_hier* h, int level, uint8_t* colours) {
  HG_CHECK(h && colours, HG_ERR_INVALID_ARG, "hg_gs_colours: null argument");
  const int li = lattice_index(h, HG_SPACE_P1, level);
  HG_CHECK(li >= 0, HG_ERR_LEVEL_RANGE, "hg_gs_colours: level %d", level);
  const LevelHost& H = h->lv[li];
  HG_CHECK(!H.colour.empty(), HG_ERR_UNSUPPORTED, "hg_gs_colours: no 4-colouring for this mesh");
  for (int64_t u = 0; u < H.dev.n_unique; ++u) colours[u] = H.colour[H.canon_rep[u]];
  return HG_OK;
}

int hg_restrict(const hg_hier* h, int space, int fine_level, int dtype, const void* rf, void* rc,
                void* stream) {
  const LevelDev* F = level_of(h, space, fine_level);
  const LevelDev* C = level_of(h, space, fine_level - 1);
  if (!F || !C) return HG_ERR_LEVEL_RANGE;
  HG_CHECK(rf && rc && rf != rc, HG_ERR_INVALID_ARG, "hg_restrict: bad pointers");
  if (space == HG_SPACE_P2) return launch_restrict_p2(*F, *C, dtype, rf, rc, (cudaStream_t)stream);
  return launch_restrict_p1(*F, *C, dtype, rf, rc, (cudaStream_t)stream);
}

int hg_prolong_add(const hg_hier* h, int space, int fine_level, int dtype, const void* ec,
                   void* xf, void* stream) {
  const LevelDev* F = level_of(h, space, fine_level);
  const LevelDev* C = level_of(h, space, fine_level - 1);
  if (!F || !C) return HG_ERR_LEVEL_RANGE;
  HG_CHECK(ec && xf && ec != xf, HG_ERR_INVALID_ARG, "hg_prolong_add: bad pointers");
  if (space == HG_SPACE_P2) return launch_prolong_p2(*F, *C, dtype, ec, xf, (cudaStream_t)stream);
  return launch_prolong_p1(*F, *C, dtype, ec, xf, (cudaStream_t)stream);
}

// Nedelec transfers and discrete gradient (the operator holds the cells'
// orientation signs).  N1 level l is stored on lattice l+1 (P2 storage).
static int n1_levels(const hg_op* op, int fine_level, bool gradient, const LevelDev** F,
                     const LevelDev** C, const char* fn) {
  HG_CHECK(op && op->kind == HG_OP_N1_CURLCURL, HG_ERR_INVALID_ARG, "%s: needs an N1 operator", fn);
  const int lo = gradient ? std::max(op->lmin, op->hier->lmin) : op->lmin + 1;
  if (fine_level < lo || fine_level > op->lmax) {
    set_error("%s: level %d outside %d..%d", fn, fine_level, lo, op->lmax);
    return HG_ERR_LEVEL_RANGE;
  }
  *F = &op->dev(fine_level);
  *C = gradient ? level_of(op->hier, HG_SPACE_P1, fine_level) : &op->dev(fine_level - 1);
  if (!*C) return HG_ERR_LEVEL_RANGE;
  return HG_OK;
}

int hg_n1_prolong_add(const hg_op* op, int fine_level, int dtype, const void* ec, void* xf,
                      void* stream) {
  const LevelDev *F, *C;
  if (int r = n1_levels(op, fine_level, false, &F, &C, "hg_n1_prolong_add")) return r;
  HG_CHECK(ec && xf && ec != xf, HG_ERR_INVALID_ARG, "hg_n1_prolong_add: bad pointers");
  return launch_n1_transfer(N1_PROLONG, *F, *C, dtype, op->n1sign, ec, xf, (cudaStream_t)stream);
}

int hg_n1_restrict(const hg_op* op, int fine_level, int dtype, const void* rf, void* rc,
                   void* stream) {
  const LevelDev *F, *C;
  if (int r = n1_levels(op, fine_level, false, &F, &C, "hg_n1_restrict")) return r;
  HG_CHECK(rf && rc && rf != rc, HG_ERR_INVALID_ARG, "hg_n1_restrict: bad pointers");
  return launch_n1_transfer(N1_RESTRICT, *F, *C, dtype, op->n1sign, rf, rc, (cudaStream_t)stream);
}

int hg_n1_gradient(const hg_op* op, int level, int dtype, const void* phi, void* u, void* stream) {
  const LevelDev *F, *C;
  if (int r = n1_levels(op, level, true, &F, &C, "hg_n1_gradient")) return r;
  HG_CHECK(phi && u && phi != u, HG_ERR_INVALID_ARG, "hg_n1_gradient: bad pointers");
  return launch_n1_transfer(N1_GRAD, *F, *C, dtype, op->n1sign, phi, u, (cudaStream_t)stream);
}

int hg_n1_gradient_t(const hg_op* op, int level, int dtype, const void* r, void* rp,
                     void* stream) {
  const LevelDev *F, *C;
  if (int e = n1_levels(op, level, true, &F, &C, "hg_n1_gradient_t")) return e;
  HG_CHECK(r && rp && r != rp, HG_ERR_INVALID_ARG, "hg_n1_gradient_t: bad pointers");
  return launch_n1_transfer(N1_GRADT, *F, *C, dtype, op->n1sign, r, rp, (cudaStream_t)stream);
}

int hg_dot(const hg_hier* h, int space, int level, int dtype, const void* x, const void* y,
           int mask, double* result, void* stream) {
  const LevelDev* L = level_of(h, space, level);
  if (!L) return HG_ERR_LEVEL_RANGE;
  HG_CHECK(x && y && result, HG_ERR_INVALID_ARG, "hg_dot: null pointer");
  cudaStream_t s = (cudaStream_t)stream;
  if (int r = launch_dot(*L, dtype, x, y, mask, h->dot_scratch, h->dot_result, s)) return r;
  HG_CUDA(cudaMemcpyAsync(h->dot_host, h->dot_result, sizeof(double), cudaMemcpyDeviceToHost, s));
  if (int r = h->fetch_error(s)) return r;
  HG_CUDA(cudaStreamSynchronize(s));
  *result = *h->dot_host;
  return h->check_error();
}

}  // extern "C"
