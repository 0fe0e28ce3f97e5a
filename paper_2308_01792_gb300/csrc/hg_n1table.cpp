// Class table of the lowest-order Nedelec (N1) prolongation between levels
// l-1 and l (multigrid by design, Sec. 5.1; N1 elements, Sec. 6).  Host
// only; the transfer kernels read it from constant memory.
//
// Fine N1 level l lives at the odd points q of lattice F (level l+1), coarse
// level l-1 at the odd points of lattice C (level l).  In F units the coarse
// micro-cells are anchored at multiples of 4, q = 4p + r with r in {0..3}^3.
// The fine micro-edge at q runs from q - d to q + d, with d the lattice
// direction fixed by the parity of q (d changes only the odd coordinates, so
// both ends lie in the closed cube [4p, 4p + 4]^3), and lies in one coarse
// micro-cell of anchor p.  Its DoF is the tangential line integral of the
// coarse function, which is linear in that cell:
//   u_f = sum over the coarse cell's local edges (a, b) of
//         [ l_a(m) (l_b(e1) - l_b(e0)) - l_b(m) (l_a(e1) - l_a(e0)) ] * u_(a,b)
// with e0, e1 the fine end points, m their midpoint and l the coarse
// barycentric coordinates (grad l . (e1 - e0) = l(e1) - l(e0) for affine l).
// The coordinates are multiples of 1/4, so every weight is an exact dyadic
// rational.  The table stores, per class r, the nonzero terms: the coarse DoF
// as a C-lattice offset from 2p, its lattice direction and the weight with
// the sign of the local edge (a -> b) against that direction folded in.  A
// kernel multiplies by the orientation signs of the cell (one per lattice
// direction: +1 when the direction's physical vector has a positive first
// nonzero of z, y, x, the order of the canonical keys) for the fine and the
// coarse DoF.  The restriction (the exact transpose) reads the same terms
// regrouped per coarse DoF parity class.
#include <cstring>
#include <mutex>

#include "hg_host.h"

namespace hg {

namespace {

const int kOffN1[6][4][3] = {
    {{0, 0, 0}, {1, 0, 0}, {0, 1, 0}, {0, 0, 1}},
    {{1, 1, 0}, {1, 0, 1}, {0, 1, 1}, {1, 1, 1}},
    {{0, 1, 0}, {1, 0, 1}, {1, 0, 0}, {0, 0, 1}},
    {{0, 1, 0}, {1, 0, 1}, {0, 0, 1}, {0, 1, 1}},
    {{0, 1, 0}, {1, 0, 1}, {0, 1, 1}, {1, 1, 0}},
    {{0, 1, 0}, {1, 0, 1}, {1, 1, 0}, {1, 0, 0}}};
const int kEdgeN1[6][2] = {{0, 1}, {0, 2}, {0, 3}, {1, 2}, {1, 3}, {2, 3}};

// 4 * barycentric coordinates of the quarter-unit point r4 in cell type t
// (Cramer's rule on integers); false if outside the closed cell.
bool bary_quarter(int t, const int r4[3], int l4[4]) {
  int M[3][3], rhs[3];
  for (int d = 0; d < 3; ++d) {
    for (int a = 0; a < 3; ++a) M[d][a] = kOffN1[t][a + 1][d] - kOffN1[t][0][d];
    rhs[d] = r4[d] - 4 * kOffN1[t][0][d];
  }
  auto det3 = [](const int A[3][3]) {
    return A[0][0] * (A[1][1] * A[2][2] - A[1][2] * A[2][1]) -
           A[0][1] * (A[1][0] * A[2][2] - A[1][2] * A[2][0]) +
           A[0][2] * (A[1][0] * A[2][1] - A[1][1] * A[2][0]);
  };
  const int D = det3(M);
  int sum = 0;
  for (int a = 0; a < 3; ++a) {
    int B[3][3];
    memcpy(B, M, sizeof B);
    for (int d = 0; d < 3; ++d) B[d][a] = rhs[d];
    const int num = det3(B);
    if (num % D) return false;
    l4[a + 1] = num / D;
    sum += l4[a + 1];
  }
  l4[0] = 4 - sum;
  for (int a = 0; a < 4; ++a)
    if (l4[a] < 0) return false;
  return true;
}

N1ProlongTable g_table;
std::once_flag g_once;
int g_status = HG_OK;

int build() {
  N1ProlongTable& T = g_table;
  memset(&T, 0, sizeof T);
  for (int cl = 0; cl < 64; ++cl) {
    const int r[3] = {cl & 3, (cl >> 2) & 3, cl >> 4};
    const int par = (r[0] & 1) | ((r[1] & 1) << 1) | ((r[2] & 1) << 2);
    T.fine_dir[cl] = par ? par - 1 : -1;
    if (!par) continue;
    const int* d = kN1Dir[par - 1];
    const int e0[3] = {r[0] - d[0], r[1] - d[1], r[2] - d[2]};
    const int e1[3] = {r[0] + d[0], r[1] + d[1], r[2] + d[2]};
    int t = -1, l0[4], l1[4];
    for (int tt = 0; tt < 6 && t < 0; ++tt)
      if (bary_quarter(tt, e0, l0) && bary_quarter(tt, e1, l1)) t = tt;
    if (t < 0) {
      set_error("N1 transfer table: no coarse cell holds the fine edge of class %d", cl);
      return HG_ERR_INVALID_ARG;
    }
    for (int e = 0; e < 6; ++e) {
      const int a = kEdgeN1[e][0], b = kEdgeN1[e][1];
      // in quarters: l = l4 / 4, m = (l0 + l1) / 8
      const double ma = (l0[a] + l1[a]) / 8.0, mb = (l0[b] + l1[b]) / 8.0;
      const double w = ma * (l1[b] - l0[b]) / 4.0 - mb * (l1[a] - l0[a]) / 4.0;
      if (w == 0.0) continue;
      int v[3], o[3];
      for (int k = 0; k < 3; ++k) {
        v[k] = kOffN1[t][b][k] - kOffN1[t][a][k];
        o[k] = kOffN1[t][a][k] + kOffN1[t][b][k];
      }
      int dir = -1, sgn = 0;
      for (int q = 0; q < 7 && dir < 0; ++q) {
        const int* D = kN1Dir[q];
        if (v[0] == D[0] && v[1] == D[1] && v[2] == D[2]) { dir = q; sgn = 1; }
        if (v[0] == -D[0] && v[1] == -D[1] && v[2] == -D[2]) { dir = q; sgn = -1; }
      }
      if (dir < 0 || T.n[cl] >= 6) {
        set_error("N1 transfer table: class %d has an edge outside the lattice directions", cl);
        return HG_ERR_INVALID_ARG;
      }
      const int q = T.n[cl]++;
      T.off[cl][q] = o[0] | (o[1] << 2) | (o[2] << 4);
      T.dir[cl][q] = dir;
      T.w[cl][q] = sgn * w;
    }
  }
  // transposed lists: the fine point q = 4p + r feeds the coarse DoF
  // c = 2p + o, i.e. sits at F offset r - 2o from 2c (each pair once)
  int cnt[8] = {};
  for (int cl = 0; cl < 64; ++cl)
    for (int q = 0; q < T.n[cl]; ++q) ++cnt[T.dir[cl][q] + 1];
  T.res_start[0] = T.res_start[1] = 0;
  for (int pc = 1; pc < 8; ++pc) T.res_start[pc + 1] = T.res_start[pc] + cnt[pc];
  if (T.res_start[8] > kN1MaxRes) {
    set_error("N1 transfer table: restriction lists too long");
    return HG_ERR_INVALID_ARG;
  }
  int fill[8];
  for (int pc = 0; pc < 8; ++pc) fill[pc] = T.res_start[pc];
  for (int cl = 0; cl < 64; ++cl) {
    const int r[3] = {cl & 3, (cl >> 2) & 3, cl >> 4};
    for (int q = 0; q < T.n[cl]; ++q) {
      const int o = T.off[cl][q];
      const int dx = r[0] - 2 * (o & 3), dy = r[1] - 2 * ((o >> 2) & 3), dz = r[2] - 2 * (o >> 4);
      const int e = fill[T.dir[cl][q] + 1]++;
      T.res_d[e] = (dx + 8) | ((dy + 8) << 5) | ((dz + 8) << 10);
      T.res_w[e] = T.w[cl][q];
      T.res_fdir[e] = T.fine_dir[cl];
    }
  }
  return HG_OK;
}

}  // namespace

const int kN1Dir[7][3] = {{1, 0, 0},  {0, 1, 0},  {-1, 1, 0}, {0, 0, 1},
                          {-1, 0, 1}, {0, -1, 1}, {1, -1, 1}};

int n1_prolong_table(const N1ProlongTable** out) {
  std::call_once(g_once, [] { g_status = build(); });
  if (g_status) return g_status;
  *out = &g_table;
  return HG_OK;
}

}  // namespace hg

extern "C" int hg_n1_restrict_table(int* start, int* d, double* w, int* fine_dir) {
  const hg::N1ProlongTable* T = nullptr;
  if (int r = hg::n1_prolong_table(&T)) return r;
  for (int c = 0; c < 9; ++c)
    if (start) start[c] = T->res_start[c];
  for (int e = 0; e < T->res_start[8]; ++e) {
    if (d) d[e] = T->res_d[e];
    if (w) w[e] = T->res_w[e];
    if (fine_dir) fine_dir[e] = T->res_fdir[e];
  }
  return HG_OK;
}

extern "C" int hg_n1_prolong_table(int* n, int* off, int* dir, double* w, int* fine_dir) {
  const hg::N1ProlongTable* T = nullptr;
  if (int r = hg::n1_prolong_table(&T)) return r;
  for (int c = 0; c < 64; ++c) {
    if (n) n[c] = T->n[c];
    if (fine_dir) fine_dir[c] = T->fine_dir[c];
    for (int q = 0; q < 6; ++q) {
      if (off) off[6 * c + q] = T->off[c][q];
      if (dir) dir[6 * c + q] = T->dir[c][q];
      if (w) w[6 * c + q] = T->w[c][q];
    }
  }
  return HG_OK;
}
