// P1 -div(k grad) with a vertex coefficient k: the element-wise operator of
// Sec. 5.2 (y += A^(T) x_T per element, A^(T) = k_T K_type, k_T the mean of
// the element's four vertex values, i.e. the exact integral for P1 k).
//
// The element sum is evaluated per output vertex v (gather form): v lies in
// 24 micro-cells of its macro cell, 4 of each of the six subgroups; for each
// of them k_T is formed from the four vertex values of k and row a of the
// subgroup's 4x4 element matrix (a = v's corner) is applied to the element's
// four values of x.  Interior points gather all 24; a point on a macro face,
// edge or vertex takes, in every cell that contains it, the incident
// micro-cells inside that cell, and the interface items add those partial
// sums over the copies in ascending cell order (as for constant stencils).
//
// Same launch structure as the constant-stencil kernel: interface items
// first, then plane-window tiles (30 consecutive t_w offsets of one plane per
// warp window, 16-window strips; see hg_p1.cu) that load the 7 neighbour
// rows of x and of k per window and take the shifted neighbours by shuffle.
// The cell's 24 x 4 element rows sit in a per-warp shared-memory copy and
// are read as 16-byte vectors (every lane of a warp reads the same row).
#include <cuda_runtime.h>

#include "hg_internal.h"

namespace hg {

namespace {

constexpr int kBlock = 256;
constexpr int kWarps = kBlock / 32;

// Incidence q = 4*type + corner: direction index (see dir_offset) of the
// element's vertex b seen from the output vertex (corner) v.
__device__ constexpr int kInc[24][4] = {
    {0, 1, 3, 5},   {2, 0, 7, 9},   {4, 8, 0, 11},  {6, 10, 12, 0},  {0, 11, 9, 5},  {12, 0, 7, 3},
    {10, 8, 0, 1},  {6, 4, 2, 0},   {0, 13, 8, 11}, {14, 0, 6, 2},   {7, 5, 0, 9},   {12, 1, 10, 0},
    {0, 13, 11, 5}, {14, 0, 2, 7},  {12, 1, 0, 3},  {6, 8, 4, 0},    {0, 13, 5, 1},  {14, 0, 7, 12},
    {6, 8, 0, 10},  {2, 11, 9, 0},  {0, 13, 1, 8},  {14, 0, 12, 6},  {2, 11, 0, 4},  {7, 5, 3, 0}};

// Mask of the incidences whose micro-cell lies inside the macro cell for a
// point of boundary class cls (bit f: on the face opposite local vertex f),
// one entry per class, fixed at compile time.
__host__ __device__ constexpr unsigned incidence_mask_of(int cls) {
  constexpr int off[6][4][3] = {
      {{0, 0, 0}, {1, 0, 0}, {0, 1, 0}, {0, 0, 1}}, {{1, 1, 0}, {1, 0, 1}, {0, 1, 1}, {1, 1, 1}},
      {{0, 1, 0}, {1, 0, 1}, {1, 0, 0}, {0, 0, 1}}, {{0, 1, 0}, {1, 0, 1}, {0, 0, 1}, {0, 1, 1}},
      {{0, 1, 0}, {1, 0, 1}, {0, 1, 1}, {1, 1, 0}}, {{0, 1, 0}, {1, 0, 1}, {1, 1, 0}, {1, 0, 0}}};
  constexpr int delta[6] = {0, 2, 1, 1, 1, 1};
  unsigned m = 0;
  for (int q = 0; q < 24; ++q) {
    const int t = q / 4, a = q % 4;
    const int* o = off[t][a];
    bool in = !((o[0] && (cls & 2)) || (o[1] && (cls & 4)) || (o[2] && (cls & 8)));
    if (o[0] + o[1] + o[2] == delta[t] && (cls & 1)) in = false;
    m |= in ? (1u << q) : 0u;
  }
  return m;
}
__device__ constexpr unsigned kIncMask[16] = {
    incidence_mask_of(0),  incidence_mask_of(1),  incidence_mask_of(2),  incidence_mask_of(3),
    incidence_mask_of(4),  incidence_mask_of(5),  incidence_mask_of(6),  incidence_mask_of(7),
    incidence_mask_of(8),  incidence_mask_of(9),  incidence_mask_of(10), incidence_mask_of(11),
    incidence_mask_of(12), incidence_mask_of(13), incidence_mask_of(14), incidence_mask_of(15)};
__device__ __forceinline__ unsigned incidence_mask(int cls) { return kIncMask[cls & 15]; }

// sum over incidences in `mask` of k_T * (K row . x_T); K: 24 x 4 of the cell.
template <typename T, bool FULL>
__device__ __forceinline__ T divkgrad_point(const T xv[kNDir], const T kv[kNDir],
                                            const T* __restrict__ K, unsigned mask) {
  T acc[4] = {T(0), T(0), T(0), T(0)};
#pragma unroll
  for (int q = 0; q < 24; ++q) {
    if (!FULL && !((mask >> q) & 1u)) continue;
    const T kT = T(0.25) * (kv[kInc[q][0]] + kv[kInc[q][1]] + kv[kInc[q][2]] + kv[kInc[q][3]]);
    const T r = __ldg(K + 4 * q) * xv[kInc[q][0]] + __ldg(K + 4 * q + 1) * xv[kInc[q][1]] +
                __ldg(K + 4 * q + 2) * xv[kInc[q][2]] + __ldg(K + 4 * q + 3) * xv[kInc[q][3]];
    acc[q & 3] += kT * r;
  }
  return (acc[0] + acc[1]) + (acc[2] + acc[3]);
}

// One 4-entry element row, aligned for a single vector shared-memory read.
template <typename T>
struct alignas(4 * sizeof(T)) Row4Vec {
  T x, y, z, w;
};
template <typename T>
struct Row4 {
  using type = Row4Vec<T>;
};

// Interior point (all 24 incidences), element rows from shared memory.
template <typename T>
__device__ __forceinline__ T divkgrad_point_sm(const T xv[kNDir], const T kv[kNDir],
                                               const typename Row4<T>::type* __restrict__ Ks) {
  // four partial sums (incidences q mod 4) shorten the dependent chain
  T acc[4] = {T(0), T(0), T(0), T(0)};
#pragma unroll
  for (int q = 0; q < 24; ++q) {
    const typename Row4<T>::type Kr = Ks[q];
    const T kT = T(0.25) * (kv[kInc[q][0]] + kv[kInc[q][1]] + kv[kInc[q][2]] + kv[kInc[q][3]]);
    const T r = Kr.x * xv[kInc[q][0]] + Kr.y * xv[kInc[q][1]] + Kr.z * xv[kInc[q][2]] +
                Kr.w * xv[kInc[q][3]];
    acc[q & 3] += kT * r;
  }
  return (acc[0] + acc[1]) + (acc[2] + acc[3]);
}

template <typename T>
struct VarArgs {
  int n, w;
  int64_t stride;
  const int4* tiles;  // plane-window tiles of one cell (same for every cell)
  int n_tiles_cell;
  int n_tiles;
  const int4* items;
  int n_items, nb_items;
  const IfaceCopy* copies;
  const uint2* clane;  // per item and lane: point, Dirichlet flag, cell, copies, active
  const T* x;
  const T* b;
  T* y;
  const T* kc;       // coefficient at stored vertices
  const T* K;        // [ncells][24][4] element-matrix rows
  const T* invdiag;  // stored 1/diag (Jacobi)
  T omega;
  int op, mode, mask;
  const uint8_t* colour;  // OP_GS: colour per stored point
  int gs_colour;
  T* dvec;                // OP_CHEB: direction, updated in place
  T cheb_a;               // OP_CHEB: weight of the previous direction
  // surrogate form: polynomial coefficients [ncells][15][nterm], degree and
  // the bands of interior rows of one cell (j0 | k << 10 | j1 << 20)
  const T* sc;
  int sdeg;
  const int* segs;
  int n_segs_cell, n_segs;
  int spat;  // surrogate: kPat7 when the fitted weights vanish outside the seven-point subset
};

// 15-point neighbourhood of a cell-local point from global memory (values
// outside the cell's closed lattice read as 0; their weights are 0).
template <typename T>
__device__ __forceinline__ void gather15(const T* __restrict__ x, int n, int w, int i, int j, int k,
                                         T v[kNDir]) {
  const int L = w - k - j;
  const int r0 = row_start(w, j, k);
  const int rjp = r0 + L, rjm = r0 - (L + 1);
  const int rkp = r0 + ntri32(w - k - 1) + L, rkm = r0 - ntri32(w - k) - (L + 1);
  const int rjmkp = rkp - L, rjpkm = rkm + L + 1;
  const int rows[15] = {r0, r0, r0, rjp, rjm, rkp, rkm, rjp, rjm, rkp, rkm, rjmkp, rjpkm, rjmkp, rjpkm};
#pragma unroll
  for (int d = 0; d < kNDir; ++d) {
    int di, dj, dk;
    dir_offset(d, di, dj, dk);
    const int a = i + di, b = j + dj, c = k + dk;
    v[d] = (a >= 0 && b >= 0 && c >= 0 && a + b + c <= n) ? __ldg(x + rows[d] + a) : T(0);
  }
}

// Apply item (lane = c * P + pt takes copy c of point pt, C <= 32 copies, P = 32 / C):
// each lane gathers its copy's partial, the point's C partials are summed in
// ascending cell order by lane exchange and written to every copy.
template <typename T, int OP>
__device__ void var_interface_item(const VarArgs<T>& A, int item, int lane);

// Item of a primitive with more than 32 copies: one lane per point, copies
// in turn.
template <typename T, int OP>
__device__ void var_interface_point(const VarArgs<T>& A, const int4& it, int lane) {
  const int dim = it.z & 15, ncopies = (it.z >> 4) & 255, dirichlet = (it.z >> 12) & 1;
  const int n = A.n, w = A.w;
  const int p = it.y + lane;
  if (lane >= it.w) return;
  int wts[3];
  // face points: rows b = 1..n-2 of n-1-b points (same order as the items)
  if (dim == 2) {
    int r = 0, rem = p;
    while (rem >= n - 2 - r) {
      rem -= n - 2 - r;
      ++r;
    }
    wts[1] = rem + 1;
    wts[2] = r + 1;
    wts[0] = n - wts[1] - wts[2];
  } else if (dim == 1) {
    wts[0] = n - 1 - p;
    wts[1] = p + 1;
    wts[2] = 0;
  } else {
    wts[0] = n;
    wts[1] = wts[2] = 0;
  }
  const IfaceCopy* cp = A.copies + it.x;
  int64_t idx0;
  {
    int i, j, k;
    copy_local_ijk(cp[0], dim, wts, i, j, k);
    idx0 = (int64_t)cp[0].cell * A.stride + tw32(w, i, j, k);
  }
  T v;
  if (dirichlet && (OP != OP_APPLY || A.mask == HG_MASK_INNER) && OP != OP_DIAG) {
    v = op_scaled(OP) ? A.x[idx0] : T(0);
  } else {
    T sum = T(0);
    for (int q = 0; q < ncopies; ++q) {
      int i, j, k;
      copy_local_ijk(cp[q], dim, wts, i, j, k);
      const int cell = cp[q].cell;
      T xv[kNDir], kv[kNDir];
      if (OP == OP_DIAG) {
#pragma unroll
        for (int d = 0; d < kNDir; ++d) xv[d] = d == 0 ? T(1) : T(0);
      } else {
        gather15<T>(A.x + (int64_t)cell * A.stride, n, w, i, j, k, xv);
      }
      gather15<T>(A.kc + (int64_t)cell * A.stride, n, w, i, j, k, kv);
      sum += divkgrad_point<T, false>(xv, kv, A.K + (int64_t)cell * 96,
                                      incidence_mask(point_class(n, i, j, k)));
    }
    if (OP == OP_APPLY || OP == OP_DIAG) {
      v = (OP == OP_APPLY && A.mode == HG_ADD) ? A.y[idx0] + sum : sum;
    } else if (OP == OP_RESID) {
      v = A.b[idx0] - sum;
    } else if (OP == OP_GS) {
      v = A.colour[idx0] == A.gs_colour ? A.x[idx0] + (A.b[idx0] - sum) * A.invdiag[idx0]
                                        : A.x[idx0];
    } else if (OP == OP_CHEB) {
      T dn = A.omega * (A.b[idx0] - sum) * A.invdiag[idx0];
      if (A.cheb_a != T(0)) dn += A.cheb_a * A.dvec[idx0];
      for (int q = 0; q < ncopies; ++q) {
        int i, j, k;
        copy_local_ijk(cp[q], dim, wts, i, j, k);
        A.dvec[(int64_t)cp[q].cell * A.stride + tw32(w, i, j, k)] = dn;
      }
      v = A.x[idx0] + dn;
    } else {
      v = A.x[idx0] + A.omega * (A.b[idx0] - sum) * A.invdiag[idx0];
    }
  }
  for (int q = 0; q < ncopies; ++q) {
    int i, j, k;
    copy_local_ijk(cp[q], dim, wts, i, j, k);
    A.y[(int64_t)cp[q].cell * A.stride + tw32(w, i, j, k)] = v;
  }
}

template <typename T, int OP>
__device__ void var_interface_item(const VarArgs<T>& A, int item, int lane) {
  const uint2 e = __ldg(A.clane + (int64_t)item * 32 + lane);
  const int C = (e.y >> 24) & 63;
  if (C > 32) {
    // one lane per point, copies in turn (32-point item)
    var_interface_point<T, OP>(A, A.items[item], lane);
    return;
  }
  const int n = A.n, w = A.w;
  const int P = 32 / C, pt = lane % P;  // lane = copy * P + point
  const bool act = (e.y >> 30) & 1u;
  const int dirichlet = (e.x >> 30) & 1u;
  const int cell = e.y & 0xffffff;
  const int i = e.x & 1023, j = (e.x >> 10) & 1023, k = (e.x >> 20) & 1023;
  const int64_t cbase = (int64_t)cell * A.stride;
  const int64_t g = cbase + tw32(w, i, j, k);
  T v;
  if (dirichlet && (OP != OP_APPLY || A.mask == HG_MASK_INNER) && OP != OP_DIAG) {
    v = op_scaled(OP) ? A.x[g] : T(0);
  } else {
    T xv[kNDir], kv[kNDir];
    if (OP == OP_DIAG) {
#pragma unroll
      for (int d = 0; d < kNDir; ++d) xv[d] = d == 0 ? T(1) : T(0);
    } else {
      gather15<T>(A.x + cbase, n, w, i, j, k, xv);
    }
    gather15<T>(A.kc + cbase, n, w, i, j, k, kv);
    const T part = divkgrad_point<T, false>(xv, kv, A.K + (int64_t)cell * 96,
                                            incidence_mask(point_class(n, i, j, k)));
    T sum = T(0);
    for (int q = 0; q < C; ++q) sum += __shfl_sync(0xffffffffu, part, (q * P + pt) & 31);
    if (OP == OP_APPLY || OP == OP_DIAG) {
      v = (OP == OP_APPLY && A.mode == HG_ADD) ? A.y[g] + sum : sum;
    } else if (OP == OP_RESID) {
      v = A.b[g] - sum;
    } else if (OP == OP_GS) {
      v = A.colour[g] == A.gs_colour ? A.x[g] + (A.b[g] - sum) * A.invdiag[g] : A.x[g];
    } else if (OP == OP_CHEB) {
      // every copy's lane reads and writes its own copy of d
      T dn = A.omega * (A.b[g] - sum) * A.invdiag[g];
      if (A.cheb_a != T(0) && act) dn += A.cheb_a * A.dvec[g];
      if (act) A.dvec[g] = dn;
      v = A.x[g] + dn;
    } else {
      v = A.x[g] + A.omega * (A.b[g] - sum) * A.invdiag[g];
    }
  }
  if (act) A.y[g] = v;
}

// Plane-window tile t of the variable-coefficient operator (offsets and row
// walk as in the constant-stencil kernel of hg_p1.cu): per window the lane
// loads the 7 rows of x and of k, takes the 8 shifted neighbours of each by
// shuffle, and gathers the 24 incidences.  Ks: this warp's shared copy of
// the cell's element rows.
template <typename T, int OP>
__device__ void var_plane_tile(const VarArgs<T>& A, int t, int lane,
                               typename Row4<T>::type* __restrict__ Ks) {
  const int cell = t / A.n_tiles_cell;
  const int4 tl = A.tiles[t - cell * A.n_tiles_cell];
  const int k = tl.x & 0xffff, nwin = tl.x >> 16;
  const int w = A.w, n = A.n;
  const int64_t base = (int64_t)cell * A.stride;
  const T* __restrict__ x = A.x + base;
  const T* __restrict__ kc = A.kc + base;
  {
    const T* __restrict__ K = A.K + (int64_t)cell * 96;
    T* ks = reinterpret_cast<T*>(Ks);
    for (int q = lane; q < 96; q += 32) ks[q] = __ldg(K + q);
    __syncwarp();
  }
  const int Tp = ntri32(w - k - 1), Tm = ntri32(w - k);
  const int gb = row_start(w, n - k - 2, k) + 1;
  const bool halo = lane == 0 || lane == 31;
  int j = tl.z >> 16, r = (tl.z & 0xffff) + lane, len = w - k - j;
  int g = tl.y + lane;
  // lanes are placed up to gb+1; the walk stays inside the plane and lanes
  // past gb+1 read at gb+1 (row length 3), never stored
  while (r >= len && g <= gb + 1) { r -= len; --len; ++j; }
  const unsigned F = 0xffffffffu;
  for (int q = 0; q < nwin; ++q) {
    if (q > 0) {
      g += 30;
      r += 30;
      while (r >= len && g <= gb + 1) { r -= len; --len; ++j; }
    }
    const bool in = g <= gb + 1;
    const int gq = in ? g : gb + 1, lq = in ? len : 3;
    const bool ok = in && g <= gb && !halo && r >= 1 && r <= len - 2;
    const int o[7] = {gq, gq + lq, gq - lq - 1, gq + Tp + lq, gq + Tp, gq - Tm - lq - 1, gq - Tm};
    T xr[7], kr[7];
#pragma unroll
    for (int m = 0; m < 7; ++m) {
      xr[m] = OP == OP_DIAG ? T(0) : __ldg(x + o[m]);
      kr[m] = __ldg(kc + o[m]);
    }
    // direction order: 0 c, 1 +i, 2 -i, 3 +j, 4 -j, 5 +k, 6 -k, 7 (-1,1,0),
    // 8 (1,-1,0), 9 (-1,0,1), 10 (1,0,-1), 11 (0,-1,1), 12 (0,1,-1),
    // 13 (1,-1,1), 14 (-1,1,-1); rows o: c, up, dn, p1c, p1m, m1c, m1p
    T xv[kNDir], kv[kNDir];
    kv[0] = kr[0];
    kv[1] = __shfl_down_sync(F, kr[0], 1);
    kv[2] = __shfl_up_sync(F, kr[0], 1);
    kv[3] = kr[1];
    kv[4] = kr[2];
    kv[5] = kr[3];
    kv[6] = kr[5];
    kv[7] = __shfl_up_sync(F, kr[1], 1);
    kv[8] = __shfl_down_sync(F, kr[2], 1);
    kv[9] = __shfl_up_sync(F, kr[3], 1);
    kv[10] = __shfl_down_sync(F, kr[5], 1);
    kv[11] = kr[4];
    kv[12] = kr[6];
    kv[13] = __shfl_down_sync(F, kr[4], 1);
    kv[14] = __shfl_up_sync(F, kr[6], 1);
    if (OP == OP_DIAG) {
#pragma unroll
      for (int d = 0; d < kNDir; ++d) xv[d] = d == 0 ? T(1) : T(0);
    } else {
      xv[0] = xr[0];
      xv[1] = __shfl_down_sync(F, xr[0], 1);
      xv[2] = __shfl_up_sync(F, xr[0], 1);
      xv[3] = xr[1];
      xv[4] = xr[2];
      xv[5] = xr[3];
      xv[6] = xr[5];
      xv[7] = __shfl_up_sync(F, xr[1], 1);
      xv[8] = __shfl_down_sync(F, xr[2], 1);
      xv[9] = __shfl_up_sync(F, xr[3], 1);
      xv[10] = __shfl_down_sync(F, xr[5], 1);
      xv[11] = xr[4];
      xv[12] = xr[6];
      xv[13] = __shfl_down_sync(F, xr[4], 1);
      xv[14] = __shfl_up_sync(F, xr[6], 1);
    }
    const T acc = divkgrad_point_sm<T>(xv, kv, Ks);
    if (ok) {
      const int64_t idx = base + gq;
      if (OP == OP_APPLY || OP == OP_DIAG) {
        A.y[idx] = (OP == OP_APPLY && A.mode == HG_ADD) ? A.y[idx] + acc : acc;
      } else if (OP == OP_RESID) {
        A.y[idx] = A.b[idx] - acc;
      } else if (OP == OP_GS) {
        A.y[idx] = A.colour[idx] == A.gs_colour ? xr[0] + (A.b[idx] - acc) * A.invdiag[idx] : xr[0];
      } else if (OP == OP_CHEB) {
        T dn = A.omega * (A.b[idx] - acc) * A.invdiag[idx];
        if (A.cheb_a != T(0)) dn += A.cheb_a * A.dvec[idx];
        A.dvec[idx] = dn;
        A.y[idx] = xr[0] + dn;
      } else {
        A.y[idx] = xr[0] + A.omega * (A.b[idx] - acc) * A.invdiag[idx];
      }
    }
  }
  __syncwarp();
}

// Band t of the surrogate operator (Sec. 5.2, surrogates): rows j0..j1-1 of
// plane k of one cell, cell-interior points only.  Lane d < 15 first forms
// the plane's coefficients of direction d in (xi, eta) at the plane's
// zeta = k/n - 1/4 (C2[a][b] = sum_c C[d][a,b,c] zeta^c); per row it forms
// rowc[d][m] = sum_b C2[m][b] eta^b (eta = j/n - 1/4) in shared memory, and
// every lane then evaluates its point's 15 weights by Horner's rule in
// xi = i/n - 1/4 and applies them to the 15 neighbours of x (all inside the
// cell's lattice for an interior point).  Q: the degree, fixed at compile time.
// PAT = kPat7: the directions outside the seven-point subset have exactly
// zero coefficients in every cell; their terms (exact zeros) are left out,
// which changes no sum.
template <typename T, int OP, int Q, int PAT>
__device__ void sur_band(const VarArgs<T>& A, int t, int lane, T* __restrict__ rowc) {
  constexpr int Q1 = Q + 1, NT = sur_nterm(Q);
  const int cell = t / A.n_segs_cell;
  const int sg = A.segs[t - cell * A.n_segs_cell];
  const int j0 = sg & 1023, k = (sg >> 10) & 1023, j1 = sg >> 20;
  const int n = A.n, w = A.w;
  const T inv_n = T(1) / T(n);  // n is a power of two: exact
  const T zeta = T(k) * inv_n - T(0.25);
  T c2[Q1][Q1];
#pragma unroll
  for (int a = 0; a < Q1; ++a)
#pragma unroll
    for (int b = 0; b < Q1; ++b) c2[a][b] = T(0);
  if (lane < kNDir) {
    const T* __restrict__ C = A.sc + ((int64_t)cell * kNDir + lane) * NT;
    int tt = 0;
#pragma unroll
    for (int a = 0; a <= Q; ++a)
#pragma unroll
      for (int b = 0; a + b <= Q; ++b) {
        // Horner in zeta over the terms c = 0..Q-a-b (stored in ascending c)
        T acc = T(0);
#pragma unroll
        for (int c = Q - a - b; c >= 0; --c) acc = fma(acc, zeta, __ldg(C + tt + c));
        tt += Q - a - b + 1;
        c2[a][b] = acc;
      }
  }
  const int64_t base = (int64_t)cell * A.stride;
  for (int j = j0; j < j1; ++j) {
    const T eta = T(j) * inv_n - T(0.25);
    if (lane < kNDir) {
#pragma unroll
      for (int m = 0; m <= Q; ++m) {
        T acc = T(0);
#pragma unroll
        for (int b = Q - m; b >= 0; --b) acc = fma(acc, eta, c2[m][b]);
        rowc[lane * Q1 + m] = acc;
      }
    }
    __syncwarp();
    const int len = w - k - j;
    const int r0 = row_start(w, j, k);
    const int rjp = r0 + len, rjm = r0 - (len + 1);
    const int rkp = r0 + ntri32(w - k - 1) + len, rkm = r0 - ntri32(w - k) - (len + 1);
    const int rjmkp = rkp - len, rjpkm = rkm + len + 1;
    const int rows[kNDir] = {r0,  r0,  r0,  rjp,   rjm,   rkp,   rkm,  rjp,
                             rjm, rkp, rkm, rjmkp, rjpkm, rjmkp, rjpkm};
    for (int i0 = 1; i0 <= len - 2; i0 += 32) {
      const int i = i0 + lane;
      const bool ok = i <= len - 2;
      const int ic = ok ? i : i0;  // lanes past the row's last interior point: unstored
      const T xi = T(ic) * inv_n - T(0.25);
          T acc = T(0), centre = T(0);
#pragma unroll
      for (int d = 0; d < kNDir; ++d) {
        if (PAT == kPat7 && !((kPat7Mask >> d) & 1u)) continue;
        T wd = rowc[d * Q1 + Q];
#pragma unroll
        for (int m = Q - 1; m >= 0; --m) wd = fma(wd, xi, rowc[d * Q1 + m]);
        if (d == 0) centre = wd;
        if (OP != OP_DIAG) {
          int di, dj, dk;
          dir_offset(d, di, dj, dk);
          acc = fma(wd, __ldg(A.x + base + rows[d] + ic + di), acc);
        }
      }
      if (OP == OP_DIAG) acc = centre;
      if (ok) {
        const int64_t idx = base + r0 + ic;
        if (OP == OP_APPLY || OP == OP_DIAG) {
          A.y[idx] = (OP == OP_APPLY && A.mode == HG_ADD) ? A.y[idx] + acc : acc;
        } else if (OP == OP_RESID) {
          A.y[idx] = A.b[idx] - acc;
        } else {
          const T x0 = A.x[idx];
          if (OP == OP_GS) {
            A.y[idx] = A.colour[idx] == A.gs_colour ? x0 + (A.b[idx] - acc) * A.invdiag[idx] : x0;
          } else if (OP == OP_CHEB) {
            T dn = A.omega * (A.b[idx] - acc) * A.invdiag[idx];
            if (A.cheb_a != T(0)) dn += A.cheb_a * A.dvec[idx];
            A.dvec[idx] = dn;
            A.y[idx] = x0 + dn;
          } else {
            A.y[idx] = x0 + A.omega * (A.b[idx] - acc) * A.invdiag[idx];
          }
        }
      }
    }
    __syncwarp();
  }
}

template <typename T, int OP, bool SUR>
__global__ void __launch_bounds__(kBlock) p1var_kernel(VarArgs<T> A) {
  // element rows of the cell (plane tiles) or the row coefficients of a
  // surrogate segment (15 x (degree + 1) <= 75 values)
  __shared__ typename Row4<T>::type Ks[kWarps][24];
  const int lane = threadIdx.x & 31;
  const int wg = blockIdx.x * kWarps + (threadIdx.x >> 5);
  if ((int)blockIdx.x < A.nb_items) {
    if (wg < A.n_items) var_interface_item<T, OP>(A, wg, lane);
  } else {
    const int t = wg - A.nb_items * kWarps;
    if (SUR) {
      if (t < A.n_segs) {
        T* rowc = reinterpret_cast<T*>(Ks[threadIdx.x >> 5]);
        if (A.spat == kPat7) {
          switch (A.sdeg) {
            case 0: sur_band<T, OP, 0, kPat7>(A, t, lane, rowc); break;
            case 1: sur_band<T, OP, 1, kPat7>(A, t, lane, rowc); break;
            case 2: sur_band<T, OP, 2, kPat7>(A, t, lane, rowc); break;
            case 3: sur_band<T, OP, 3, kPat7>(A, t, lane, rowc); break;
            default: sur_band<T, OP, 4, kPat7>(A, t, lane, rowc); break;
          }
        } else {
          switch (A.sdeg) {
            case 0: sur_band<T, OP, 0, 0>(A, t, lane, rowc); break;
            case 1: sur_band<T, OP, 1, 0>(A, t, lane, rowc); break;
            case 2: sur_band<T, OP, 2, 0>(A, t, lane, rowc); break;
            case 3: sur_band<T, OP, 3, 0>(A, t, lane, rowc); break;
            default: sur_band<T, OP, 4, 0>(A, t, lane, rowc); break;
          }
        }
      }
    } else if (t < A.n_tiles) {
      var_plane_tile<T, OP>(A, t, lane, Ks[threadIdx.x >> 5]);
    }
  }
}

template <typename T, int OP, bool SUR = false>
int run_var(const LevelDev& L, const StencilArgs& a, const VarCoef& vc, cudaStream_t s,
            const SurCoef* sc = nullptr) {
  VarArgs<T> A;
  A.n = L.n;
  A.w = L.w;
  A.stride = L.cell_stride;
  A.tiles = L.ptiles;
  A.n_tiles_cell = L.n_ptiles_cell;
  A.n_tiles = L.n_ptiles_cell * L.ncells;
  A.items = L.citems;
  A.n_items = L.n_citems;
  A.clane = L.clane;
  A.nb_items = (A.n_items + kWarps - 1) / kWarps;
  A.copies = L.copies;
  A.x = (const T*)a.x;
  A.b = (const T*)a.b;
  A.y = (T*)a.out;
  A.kc = (const T*)vc.k;
  A.K = (const T*)vc.K;
  A.invdiag = (const T*)vc.invdiag;
  A.omega = (T)a.omega;
  A.op = a.op;
  A.mode = a.mode;
  A.mask = a.mask;
  A.colour = L.colour;
  A.gs_colour = a.colour;
  A.dvec = (T*)a.dvec;
  A.cheb_a = (T)a.cheb_a;
  A.sc = nullptr;
  A.sdeg = 0;
  A.segs = nullptr;
  A.n_segs_cell = A.n_segs = 0;
  A.spat = 0;
  if (SUR) {
    A.spat = sc->pattern;
    A.sc = (const T*)sc->coef;
    A.sdeg = sc->degree;
    A.segs = sc->segs;
    A.n_segs_cell = sc->n_segs_cell;
    A.n_segs = sc->n_segs_cell * L.ncells;
  }
  const int work = SUR ? A.n_segs : A.n_tiles;
  const int grid = A.nb_items + (work + kWarps - 1) / kWarps;
  if (grid == 0) return HG_OK;
  p1var_kernel<T, OP, SUR><<<grid, kBlock, 0, s>>>(A);
  HG_CUDA(cudaGetLastError());
  return HG_OK;
}

template <typename T, bool SUR = false>
int run_var_op(const LevelDev& L, const StencilArgs& a, const VarCoef& vc, cudaStream_t s,
               const SurCoef* sc = nullptr) {
  switch (a.op) {
    case OP_APPLY: return run_var<T, OP_APPLY, SUR>(L, a, vc, s, sc);
    case OP_RESID: return run_var<T, OP_RESID, SUR>(L, a, vc, s, sc);
    case OP_JACOBI: return run_var<T, OP_JACOBI, SUR>(L, a, vc, s, sc);
    case OP_DIAG: return run_var<T, OP_DIAG, SUR>(L, a, vc, s, sc);
    case OP_GS: return run_var<T, OP_GS, SUR>(L, a, vc, s, sc);
    case OP_CHEB: return run_var<T, OP_CHEB, SUR>(L, a, vc, s, sc);
  }
  set_error("unknown cell operation %d", a.op);
  return HG_ERR_INVALID_ARG;
}

// Least-squares projections of the surrogate fit: block (cell, d) sums
// Q[p][t] * S_d(p) over the cell's interior points in a fixed order (thread
// strides, then a shared-memory tree), so the result is deterministic.
constexpr int kMomThreads = 256;
__global__ void __launch_bounds__(kMomThreads) surrogate_moments_kernel(
    const double* __restrict__ S, int64_t stride, const int* __restrict__ pidx, int P,
    const double* __restrict__ Q, int T, double* __restrict__ M) {
  constexpr int kMaxT = sur_nterm(kSurMaxDegree);
  __shared__ double red[kMomThreads];
  const int cell = blockIdx.x / kNDir, d = blockIdx.x - cell * kNDir;
  double acc[kMaxT];
#pragma unroll
  for (int t = 0; t < kMaxT; ++t) acc[t] = 0.0;
  for (int p = threadIdx.x; p < P; p += kMomThreads) {
    const double sv = S[16 * ((int64_t)cell * stride + pidx[p]) + d];
    const double* qp = Q + (int64_t)p * T;
#pragma unroll
    for (int t = 0; t < kMaxT; ++t)
      if (t < T) acc[t] = fma(qp[t], sv, acc[t]);
  }
#pragma unroll 1
  for (int t = 0; t < T; ++t) {
    double v = 0.0;
#pragma unroll
    for (int u = 0; u < kMaxT; ++u)
      if (u == t) v = acc[u];
    red[threadIdx.x] = v;
    __syncthreads();
    for (int h = kMomThreads / 2; h > 0; h >>= 1) {
      if ((int)threadIdx.x < h) red[threadIdx.x] += red[threadIdx.x + h];
      __syncthreads();
    }
    if (threadIdx.x == 0) M[((int64_t)cell * kNDir + d) * T + t] = red[0];
    __syncthreads();
  }
}

// Partial stencils of every stored point: one warp per lattice row of a
// cell, lanes over i; weight d = the operator's point sum applied to the
// unit vector of direction d (incidences inside the cell only); the 16th
// value is 1 / centre weight for points inside the cell, else 0.
template <typename T>
__global__ void __launch_bounds__(kBlock) divkgrad_stencil_kernel(int n, int w, int64_t stride,
                                                                  int n_rows, const T* kc,
                                                                  const T* K, T* S) {
  const int lane = threadIdx.x & 31;
  const int r = blockIdx.x * kWarps + (threadIdx.x >> 5);
  if (r >= n_rows) return;
  int cell, j, k;
  row_item(w, r, cell, j, k);
  const int64_t r0 = (int64_t)cell * stride + row_start(w, j, k);
  for (int i = lane; i + j + k <= n; i += 32) {
    T kv[kNDir];
    gather15<T>(kc + (int64_t)cell * stride, n, w, i, j, k, kv);
    const unsigned mask = incidence_mask(point_class(n, i, j, k));
    T centre = T(0);
#pragma unroll 1
    for (int d = 0; d < kNDir; ++d) {
      T xv[kNDir];
#pragma unroll
      for (int e = 0; e < kNDir; ++e) xv[e] = e == d ? T(1) : T(0);
      const T v = divkgrad_point<T, false>(xv, kv, K + (int64_t)cell * 96, mask);
      S[16 * (r0 + i) + d] = v;
      if (d == 0) centre = v;
    }
    // slot 15: inverse diagonal of points inside the cell (their stencil is complete)
    S[16 * (r0 + i) + 15] =
        (point_class(n, i, j, k) == 0 && centre != T(0)) ? T(1) / centre : T(0);
  }
}

template <typename T>
int run_stencil(const LevelDev& L, const VarCoef& vc, void* S, cudaStream_t s) {
  HG_CUDA(cudaMemsetAsync(S, 0, (size_t)16 * L.n_stored * sizeof(T), s));
  const int n_rows = L.ncells * ntri32(L.w);
  if (n_rows == 0) return HG_OK;
  divkgrad_stencil_kernel<T><<<(n_rows + kWarps - 1) / kWarps, kBlock, 0, s>>>(
      L.n, L.w, L.cell_stride, n_rows, (const T*)vc.k, (const T*)vc.K, (T*)S);
  HG_CUDA(cudaGetLastError());
  return HG_OK;
}

}  // namespace

int launch_p1_divkgrad(const LevelDev& L, int dtype, const StencilArgs& a, const VarCoef& vc,
                       cudaStream_t s) {
  return dtype == HG_F64 ? run_var_op<double>(L, a, vc, s) : run_var_op<float>(L, a, vc, s);
}

int launch_p1_surrogate(const LevelDev& L, int dtype, const StencilArgs& a, const VarCoef& vc,
                        const SurCoef& sc, cudaStream_t s) {
  if (sc.degree < 0 || sc.degree > kSurMaxDegree || L.n > 512) {
    set_error("surrogate: degree %d or level size %d outside the kernel's range", sc.degree, L.n);
    return HG_ERR_UNSUPPORTED;
  }
  return dtype == HG_F64 ? run_var_op<double, true>(L, a, vc, s, &sc)
                         : run_var_op<float, true>(L, a, vc, s, &sc);
}

int launch_surrogate_moments(const LevelDev& L, const double* S, const int* pidx, int P,
                             const double* Q, int T, double* M, cudaStream_t s) {
  if (T < 1 || T > sur_nterm(kSurMaxDegree)) {
    set_error("surrogate: %d basis functions outside 1..%d", T, sur_nterm(kSurMaxDegree));
    return HG_ERR_INVALID_ARG;
  }
  if (L.ncells == 0 || P == 0) return HG_OK;
  surrogate_moments_kernel<<<L.ncells * kNDir, kMomThreads, 0, s>>>(S, L.cell_stride, pidx, P, Q, T,
                                                                   M);
  HG_CUDA(cudaGetLastError());
  return HG_OK;
}

int launch_divkgrad_stencil(const LevelDev& L, int dtype, const VarCoef& vc, void* S,
                            cudaStream_t s) {
  return dtype == HG_F64 ? run_stencil<double>(L, vc, S, s) : run_stencil<float>(L, vc, S, s);
}

}  // namespace hg
