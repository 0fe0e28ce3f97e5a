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
// first, then interior tiles whose warps hold register windows of the 7 rows
// of x and of k that the 15-point neighbourhood touches.
#include <cuda_runtime.h>

#include "hg_internal.h"

namespace hg {

namespace {

constexpr int kBlock = 256;
constexpr int kWarps = kBlock / 32;
constexpr int kVarRows = 4;  // output rows per interior tile

// Incidence q = 4*type + corner: direction index (see dir_offset) of the
// element's vertex b seen from the output vertex (corner) v.
__device__ constexpr int kInc[24][4] = {
    {0, 1, 3, 5},   {2, 0, 7, 9},   {4, 8, 0, 11},  {6, 10, 12, 0},  {0, 11, 9, 5},  {12, 0, 7, 3},
    {10, 8, 0, 1},  {6, 4, 2, 0},   {0, 13, 8, 11}, {14, 0, 6, 2},   {7, 5, 0, 9},   {12, 1, 10, 0},
    {0, 13, 11, 5}, {14, 0, 2, 7},  {12, 1, 0, 3},  {6, 8, 4, 0},    {0, 13, 5, 1},  {14, 0, 7, 12},
    {6, 8, 0, 10},  {2, 11, 9, 0},  {0, 13, 1, 8},  {14, 0, 12, 6},  {2, 11, 0, 4},  {7, 5, 3, 0}};
// Vertex offsets of the six subgroups and their width deficit (w = n - delta).
__device__ constexpr int kOff[6][4][3] = {
    {{0, 0, 0}, {1, 0, 0}, {0, 1, 0}, {0, 0, 1}}, {{1, 1, 0}, {1, 0, 1}, {0, 1, 1}, {1, 1, 1}},
    {{0, 1, 0}, {1, 0, 1}, {1, 0, 0}, {0, 0, 1}}, {{0, 1, 0}, {1, 0, 1}, {0, 0, 1}, {0, 1, 1}},
    {{0, 1, 0}, {1, 0, 1}, {0, 1, 1}, {1, 1, 0}}, {{0, 1, 0}, {1, 0, 1}, {1, 1, 0}, {1, 0, 0}}};
__device__ constexpr int kDelta[6] = {0, 2, 1, 1, 1, 1};

// Mask of the incidences whose micro-cell lies inside the macro cell for a
// point of boundary class cls (bit f: on the face opposite local vertex f).
__device__ __forceinline__ unsigned incidence_mask(int cls) {
  unsigned m = 0;
#pragma unroll
  for (int q = 0; q < 24; ++q) {
    const int t = q / 4, a = q % 4;
    const int* o = kOff[t][a];
    bool in = !((o[0] && (cls & 2)) || (o[1] && (cls & 4)) || (o[2] && (cls & 8)));
    if (o[0] + o[1] + o[2] == kDelta[t] && (cls & 1)) in = false;
    m |= in ? (1u << q) : 0u;
  }
  return m;
}

// sum over incidences in `mask` of k_T * (K row . x_T); K: 24 x 4 of the cell.
template <typename T, bool FULL>
__device__ __forceinline__ T divkgrad_point(const T xv[kNDir], const T kv[kNDir],
                                            const T* __restrict__ K, unsigned mask) {
  T acc = T(0);
#pragma unroll
  for (int q = 0; q < 24; ++q) {
    if (!FULL && !((mask >> q) & 1u)) continue;
    const T kT = T(0.25) * (kv[kInc[q][0]] + kv[kInc[q][1]] + kv[kInc[q][2]] + kv[kInc[q][3]]);
    const T r = __ldg(K + 4 * q) * xv[kInc[q][0]] + __ldg(K + 4 * q + 1) * xv[kInc[q][1]] +
                __ldg(K + 4 * q + 2) * xv[kInc[q][2]] + __ldg(K + 4 * q + 3) * xv[kInc[q][3]];
    acc += kT * r;
  }
  return acc;
}

template <typename T>
struct VarArgs {
  int n, w;
  int64_t stride;
  const int4* tiles;
  int n_tiles;
  const int4* items;
  int n_items, nb_items;
  const IfaceCopy* copies;
  const T* x;
  const T* b;
  T* y;
  const T* kc;       // coefficient at stored vertices
  const T* K;        // [ncells][24][4] element-matrix rows
  const T* invdiag;  // stored 1/diag (Jacobi)
  T omega;
  int op, mode, mask;
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

template <typename T, int OP>
__device__ void var_interface_point(const VarArgs<T>& A, int item, int lane) {
  const int4 it = A.items[item];
  const int dim = it.z & 15, ncopies = (it.z >> 4) & 255, dirichlet = (it.z >> 12) & 1;
  const int n = A.n, w = A.w;
  const int p = it.y + lane;
  if (p >= prim_points(dim, n)) return;
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
    v = OP == OP_JACOBI ? A.x[idx0] : T(0);
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

// Register window of one lattice row set (see the constant-stencil tiles):
// plane k rows j0-1..j0+R, plane k+1 rows j0-1..j0+R-1, plane k-1 rows j0..j0+R.
template <typename T, int R>
struct Window {
  T K[R + 2], Kp[R + 1], Km[R + 1];
  __device__ __forceinline__ void load(const T* __restrict__ x, int w, int i, int j0, int k,
                                       int nr) {
    const int lk = w - k, lkp = w - k - 1, lkm = w - k + 1;
    int r = row_start(w, j0 - 1, k);
#pragma unroll
    for (int q = 0; q < R + 2; ++q) {
      const int len = lk - (j0 - 1 + q);
      K[q] = (q < nr + 2 && i >= 0 && i < len) ? __ldg(x + r + i) : T(0);
      r += len;
    }
    r = row_start(w, j0 - 1, k + 1);
#pragma unroll
    for (int q = 0; q < R + 1; ++q) {
      const int len = lkp - (j0 - 1 + q);
      Kp[q] = (q < nr + 1 && i >= 0 && i < len) ? __ldg(x + r + i) : T(0);
      r += len;
    }
    r = row_start(w, j0, k - 1);
#pragma unroll
    for (int q = 0; q < R + 1; ++q) {
      const int len = lkm - (j0 + q);
      Km[q] = (q < nr + 1 && i >= 0 && i < len) ? __ldg(x + r + i) : T(0);
      r += len;
    }
  }
  // 15 values of output row q in direction order (all lanes shuffle)
  __device__ __forceinline__ void neighbours(int q, T v[kNDir]) const {
    const unsigned F = 0xffffffffu;
    v[0] = K[q + 1];
    v[1] = __shfl_down_sync(F, K[q + 1], 1);
    v[2] = __shfl_up_sync(F, K[q + 1], 1);
    v[3] = K[q + 2];
    v[4] = K[q];
    v[5] = Kp[q + 1];
    v[6] = Km[q];
    v[7] = __shfl_up_sync(F, K[q + 2], 1);
    v[8] = __shfl_down_sync(F, K[q], 1);
    v[9] = __shfl_up_sync(F, Kp[q + 1], 1);
    v[10] = __shfl_down_sync(F, Km[q], 1);
    v[11] = Kp[q];
    v[12] = Km[q + 1];
    v[13] = __shfl_down_sync(F, Kp[q], 1);
    v[14] = __shfl_up_sync(F, Km[q + 1], 1);
  }
};

template <typename T, int OP>
__device__ void var_interior_tile(const VarArgs<T>& A, int t, int lane) {
  const int4 tl = A.tiles[t];
  const int cell = tl.x, k = tl.y, i0 = tl.z, j0 = tl.w & 0xffff, j1 = tl.w >> 16;
  const int w = A.w;
  const int64_t base = (int64_t)cell * A.stride;
  const int i = i0 - 1 + lane;
  const bool out_lane = lane >= 1 && lane <= 30;
  const T* __restrict__ K = A.K + (int64_t)cell * 96;
  // the tile table is built for kTileRows rows; process it in chunks of kVarRows
  for (int jc = j0; jc < j1; jc += kVarRows) {
    const int nr = min(kVarRows, j1 - jc);
    Window<T, kVarRows> wx, wk;
    if (OP != OP_DIAG) wx.load(A.x + base, w, i, jc, k, nr);
    wk.load(A.kc + base, w, i, jc, k, nr);
    int ry = row_start(w, jc, k);
#pragma unroll
    for (int q = 0; q < kVarRows; ++q) {
      if (q < nr) {
        const int j = jc + q;
        T xv[kNDir], kv[kNDir];
        if (OP == OP_DIAG) {
#pragma unroll
          for (int d = 0; d < kNDir; ++d) xv[d] = d == 0 ? T(1) : T(0);
        } else {
          wx.neighbours(q, xv);
        }
        wk.neighbours(q, kv);
        const T acc = divkgrad_point<T, true>(xv, kv, K, 0u);
        if (out_lane && i < (w - k) - j - 1) {
          const int64_t idx = base + ry + i;
          if (OP == OP_APPLY || OP == OP_DIAG) {
            A.y[idx] = (OP == OP_APPLY && A.mode == HG_ADD) ? A.y[idx] + acc : acc;
          } else if (OP == OP_RESID) {
            A.y[idx] = A.b[idx] - acc;
          } else {
            A.y[idx] = xv[0] + A.omega * (A.b[idx] - acc) * A.invdiag[idx];
          }
        }
        ry += (w - k) - j;
      }
    }
  }
}

template <typename T, int OP>
__global__ void __launch_bounds__(kBlock) p1var_kernel(VarArgs<T> A) {
  const int lane = threadIdx.x & 31;
  const int wg = blockIdx.x * kWarps + (threadIdx.x >> 5);
  if ((int)blockIdx.x < A.nb_items) {
    if (wg < A.n_items) var_interface_point<T, OP>(A, wg, lane);
  } else {
    const int t = wg - A.nb_items * kWarps;
    if (t < A.n_tiles) var_interior_tile<T, OP>(A, t, lane);
  }
}

template <typename T, int OP>
int run_var(const LevelDev& L, const StencilArgs& a, const VarCoef& vc, cudaStream_t s) {
  VarArgs<T> A;
  A.n = L.n;
  A.w = L.w;
  A.stride = L.cell_stride;
  A.tiles = L.tiles;
  A.n_tiles = L.n_tiles;
  A.items = L.items;
  A.n_items = (OP == OP_APPLY && a.mask == HG_MASK_INNER) ? L.n_items_inner : L.n_items;
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
  const int grid = A.nb_items + (L.n_tiles + kWarps - 1) / kWarps;
  if (grid == 0) return HG_OK;
  p1var_kernel<T, OP><<<grid, kBlock, 0, s>>>(A);
  HG_CUDA(cudaGetLastError());
  return HG_OK;
}

template <typename T>
int run_var_op(const LevelDev& L, const StencilArgs& a, const VarCoef& vc, cudaStream_t s) {
  switch (a.op) {
    case OP_APPLY: return run_var<T, OP_APPLY>(L, a, vc, s);
    case OP_RESID: return run_var<T, OP_RESID>(L, a, vc, s);
    case OP_JACOBI: return run_var<T, OP_JACOBI>(L, a, vc, s);
    case OP_DIAG: return run_var<T, OP_DIAG>(L, a, vc, s);
  }
  set_error("unknown cell operation %d", a.op);
  return HG_ERR_INVALID_ARG;
}

}  // namespace

int launch_p1_divkgrad(const LevelDev& L, int dtype, const StencilArgs& a, const VarCoef& vc,
                       cudaStream_t s) {
  return dtype == HG_F64 ? run_var_op<double>(L, a, vc, s) : run_var_op<float>(L, a, vc, s);
}

}  // namespace hg
