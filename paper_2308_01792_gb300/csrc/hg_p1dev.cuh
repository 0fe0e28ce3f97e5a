// Device pieces shared by the P1 constant-stencil kernels (hg_p1.cu,
// hg_p1stream.cu): the launch arguments, the partial stencil of one cell at
// any cell-local point, and the interface items that sum the partials of a
// macro face/edge/vertex point over the cells containing it (the ghost-layer
// exchange of Sec. 2 as an on-device gather) and write the sum to every copy.
#pragma once

#include <cuda_runtime.h>

#include "hg_internal.h"

namespace hg {
namespace {

template <typename T>
struct FusedArgs {
  int n, w;
  int64_t stride;
  const uint8_t* flags;
  const int4* tiles;  // plane-window tiles of one cell (same for every cell)
  int n_tiles_cell;
  int n_tiles;        // all cells
  const int4* items;  // apply items (first_copy, p0, dim | ncopies<<4 | dirichlet<<12, points)
  const uint2* clane;  // per item and lane: point, Dirichlet flag, cell, copies, active
  int n_items;
  int nb_items;       // blocks holding interface items (first in the grid)
  const IfacePrim* prims;
  const IfaceCopy* copies;
  const T* x;
  const T* b;
  T* y;
  const T* sten;
  const T* sst;           // stored stencils [nst][16] (ST kernels) instead of sten
  const int2* march;      // column-march items of one cell (march kernel)
  int n_march_cell, n_march;
  T omega;
  int mode, mask;
  const uint8_t* colour;  // OP_GS: colour per stored point
  int gs_colour;          // OP_GS: the colour updated
  T* dvec;                // OP_CHEB: direction, updated in place
  T cheb_a;               // OP_CHEB: weight of the previous direction
  int* err;            // device error word (bounded waits record HG_ERR_TIMEOUT)
};

// Face point p (rows b = 1..n-2 of n-1-b points) -> barycentric weights.
__device__ __forceinline__ void face_point(int n, int p, int wts[3]) {
  // row r = b-1 starts at S_r = r(2n-3-r)/2
  const float q = 2.0f * n - 3.0f;
  int r = (int)floorf((q - sqrtf(fmaxf(q * q - 8.0f * p, 0.0f))) * 0.5f);
  if (r < 0) r = 0;
  while ((r + 1) * (2 * n - 3 - (r + 1)) / 2 <= p) ++r;
  while (r * (2 * n - 3 - r) / 2 > p) --r;
  const int a = p - r * (2 * n - 3 - r) / 2 + 1;
  const int b = r + 1;
  wts[0] = n - a - b;
  wts[1] = a;
  wts[2] = b;
}

__device__ __forceinline__ void prim_weights(int dim, int n, int p, int wts[3]) {
  if (dim == 2) {
    face_point(n, p, wts);
  } else if (dim == 1) {
    wts[0] = n - 1 - p;
    wts[1] = p + 1;
    wts[2] = 0;
  } else {
    wts[0] = n;
    wts[1] = 0;
    wts[2] = 0;
  }
}

// One stored stencil: 15 weights and, in the 16th slot, 1/(centre weight)
// for points inside the cell (16-byte vector loads).
__device__ __forceinline__ void load_sten16(const float* __restrict__ p, float s[kNDir],
                                            float& inv) {
  const float4* q = reinterpret_cast<const float4*>(p);
  const float4 a = __ldg(q), b = __ldg(q + 1), c = __ldg(q + 2), d = __ldg(q + 3);
  s[0] = a.x; s[1] = a.y; s[2] = a.z; s[3] = a.w;
  s[4] = b.x; s[5] = b.y; s[6] = b.z; s[7] = b.w;
  s[8] = c.x; s[9] = c.y; s[10] = c.z; s[11] = c.w;
  s[12] = d.x; s[13] = d.y; s[14] = d.z;
  inv = d.w;
}
__device__ __forceinline__ void load_sten16(const double* __restrict__ p, double s[kNDir],
                                            double& inv) {
  const double2* q = reinterpret_cast<const double2*>(p);
#pragma unroll
  for (int v = 0; v < 7; ++v) {
    const double2 t = __ldg(q + v);
    s[2 * v] = t.x;
    s[2 * v + 1] = t.y;
  }
  const double2 t = __ldg(q + 7);
  s[14] = t.x;
  inv = t.y;
}

// Partial stencil of one cell at a cell-local point (any class).  The 7
// rows touched are found from rs(j,k) by row-length steps:
//   rs(j+-1,k), rs(j,k+1) = rs + ntri(w-k-1) + L, rs(j,k-1) = rs - ntri(w-k) - (L+1),
//   rs(j-1,k+1) = rs(j,k+1) - L, rs(j+1,k-1) = rs(j,k-1) + L + 1, L = w-k-j.
// All 15 weights and values are loaded before the sum so the loads overlap.
// S: the class stencil, or with ST the point's own stored stencil.
template <typename T, bool ST = false>
__device__ __forceinline__ void cell_partial_load(const T* __restrict__ x, const T* __restrict__ S,
                                                  int n, int w, int i, int j, int k, T sv[kNDir],
                                                  T xv[kNDir]) {
  const int L = w - k - j;
  const int r0 = row_start(w, j, k);
  const int rjp = r0 + L, rjm = r0 - (L + 1);
  const int rkp = r0 + ntri32(w - k - 1) + L, rkm = r0 - ntri32(w - k) - (L + 1);
  const int rjmkp = rkp - L, rjpkm = rkm + L + 1;
  const int rows[15] = {r0, r0, r0, rjp, rjm, rkp, rkm, rjp, rjm, rkp, rkm, rjmkp, rjpkm, rjmkp, rjpkm};
  {
    // stored stencils and the 16-value class stencils alike: 16-byte vectors
    T unused;
    load_sten16(S, sv, unused);
  }
#pragma unroll
  for (int d = 0; d < kNDir; ++d) {
    int di, dj, dk;
    dir_offset(d, di, dj, dk);
    const int a = i + di, b = j + dj, c = k + dk;
    xv[d] = (a >= 0 && b >= 0 && c >= 0 && a + b + c <= n) ? __ldg(x + rows[d] + a) : T(0);
  }
}

// 15-term dot in three independent chains (plane k, k+1, k-1 terms) for
// instruction-level parallelism; the order is fixed, so every caller with the
// same operands gets the same bits.
template <typename T>
__device__ __forceinline__ T dot15(const T sv[kNDir], const T xv[kNDir]) {
  const T a0 = sv[0] * xv[0] + sv[1] * xv[1] + sv[2] * xv[2] + sv[3] * xv[3] + sv[4] * xv[4] +
               sv[7] * xv[7] + sv[8] * xv[8];
  const T a1 = sv[5] * xv[5] + sv[9] * xv[9] + sv[11] * xv[11] + sv[13] * xv[13];
  const T a2 = sv[6] * xv[6] + sv[10] * xv[10] + sv[12] * xv[12] + sv[14] * xv[14];
  return a0 + (a1 + a2);
}

// Item of a primitive with more than 32 copies: one lane per point, copies
// in turn.
template <typename T, int OP, bool ST>
__device__ void interface_point_serial(const FusedArgs<T>& A, const int4& it, int lane) {
  const int dim = it.z & 15, ncopies = (it.z >> 4) & 255, dirichlet = (it.z >> 12) & 1;
  const int n = A.n, w = A.w;
  const int p = it.y + lane;
  if (lane >= it.w) return;
  int wts[3];
  prim_weights(dim, n, p, wts);
  const IfaceCopy* cp = A.copies + it.x;
  int64_t idx0;
  {
    int i, j, k;
    copy_local_ijk(cp[0], dim, wts, i, j, k);
    idx0 = (int64_t)cp[0].cell * A.stride + tw32(w, i, j, k);
  }
  T v;
  if (dirichlet && (OP != OP_APPLY || A.mask == HG_MASK_INNER)) {
    v = op_scaled(OP) ? A.x[idx0] : T(0);
  } else {
    T sum = T(0), diag = T(0);
    for (int q = 0; q < ncopies; ++q) {
      T sv[kNDir], xv[kNDir];
      int i, j, k;
      copy_local_ijk(cp[q], dim, wts, i, j, k);
      const int cell = cp[q].cell;
      if (ST)
        cell_partial_load<T, true>(A.x + (int64_t)cell * A.stride,
                                   A.sst + 16 * ((int64_t)cell * A.stride + tw32(w, i, j, k)), n,
                                   w, i, j, k, sv, xv);
      else
        cell_partial_load<T>(A.x + (int64_t)cell * A.stride,
                             A.sten + (int64_t)cell * 256 + point_class(n, i, j, k) * 16, n, w, i,
                             j, k, sv, xv);
      sum += dot15<T>(sv, xv);
      if (op_scaled(OP)) diag += sv[0];
    }
    if (OP == OP_APPLY) {
      v = A.mode == HG_ADD ? A.y[idx0] + sum : sum;
    } else if (OP == OP_RESID) {
      v = A.b[idx0] - sum;
    } else if (OP == OP_GS) {
      v = A.colour[idx0] == A.gs_colour ? A.x[idx0] + (A.b[idx0] - sum) / diag : A.x[idx0];
    } else if (OP == OP_CHEB) {
      T dn = A.omega * (A.b[idx0] - sum) / diag;
      if (A.cheb_a != T(0)) dn += A.cheb_a * A.dvec[idx0];
      for (int q = 0; q < ncopies; ++q) {
        int i, j, k;
        copy_local_ijk(cp[q], dim, wts, i, j, k);
        A.dvec[(int64_t)cp[q].cell * A.stride + tw32(w, i, j, k)] = dn;
      }
      v = A.x[idx0] + dn;
    } else {
      v = A.x[idx0] + A.omega * (A.b[idx0] - sum) / diag;
    }
  }
  for (int q = 0; q < ncopies; ++q) {
    int i, j, k;
    copy_local_ijk(cp[q], dim, wts, i, j, k);
    A.y[(int64_t)cp[q].cell * A.stride + tw32(w, i, j, k)] = v;
  }
}

// One lane of an apply item (lane = c * P + pt takes copy c of point pt, C <= 32
// copies, P = 32 / C points), decoded from its 8-byte entry of the lane table.
struct ItemLane {
  int C, P, pt, dirichlet, cell, i, j, k;
  bool act;
  int64_t cbase, g;
};

__device__ __forceinline__ ItemLane item_lane(const uint2 e, int lane, int w, int64_t stride) {
  ItemLane L;
  L.C = (e.y >> 24) & 63;
  L.P = 32 / (L.C > 0 && L.C <= 32 ? L.C : 32);
  L.pt = lane % L.P;
  L.act = (e.y >> 30) & 1u;
  L.dirichlet = (e.x >> 30) & 1u;
  L.cell = e.y & 0xffffff;
  L.i = e.x & 1023;
  L.j = (e.x >> 10) & 1023;
  L.k = (e.x >> 20) & 1023;
  L.cbase = (int64_t)L.cell * stride;
  L.g = L.cbase + tw32(w, L.i, L.j, L.k);
  return L;
}

// Whether the item's output is fixed by its Dirichlet primitive (no sum).
template <int OP>
__device__ __forceinline__ bool item_fixed(const ItemLane& L, int mask) {
  return L.dirichlet && (OP != OP_APPLY || mask == HG_MASK_INNER);
}

// The lane's partial stencil and neighbour values (loads only).
template <typename T, bool ST>
__device__ __forceinline__ void item_load(const FusedArgs<T>& A, const ItemLane& L, T sv[kNDir],
                                          T xv[kNDir]) {
  if (ST)
    cell_partial_load<T, true>(A.x + L.cbase, A.sst + 16 * L.g, A.n, A.w, L.i, L.j, L.k, sv, xv);
  else
    cell_partial_load<T>(A.x + L.cbase,
                         A.sten + (int64_t)L.cell * 256 + point_class(A.n, L.i, L.j, L.k) * 16,
                         A.n, A.w, L.i, L.j, L.k, sv, xv);
}

// Sum of the point's C partials in ascending copy (= cell) order by lane
// exchange, the operation's output, written to the lane's copy.
template <typename T, int OP>
__device__ __forceinline__ void item_finish(const FusedArgs<T>& A, const ItemLane& L, bool fixed,
                                            const T sv[kNDir], const T xv[kNDir]) {
  const int64_t g = L.g;
  T v;
  if (fixed) {
    v = op_scaled(OP) ? A.x[g] : T(0);
  } else {
    const T part = dot15<T>(sv, xv);
    T sum = T(0), diag = T(0);
    for (int q = 0; q < L.C; ++q) {
      const int src = (q * L.P + L.pt) & 31;
      sum += __shfl_sync(0xffffffffu, part, src);
      if (op_scaled(OP)) diag += __shfl_sync(0xffffffffu, sv[0], src);
    }
    if (OP == OP_APPLY) {
      v = A.mode == HG_ADD ? A.y[g] + sum : sum;
    } else if (OP == OP_RESID) {
      v = A.b[g] - sum;
    } else if (OP == OP_GS) {
      v = A.colour[g] == A.gs_colour ? A.x[g] + (A.b[g] - sum) / diag : A.x[g];
    } else if (OP == OP_CHEB) {
      // every copy's lane reads and writes its own copy of d
      T dn = A.omega * (A.b[g] - sum) / diag;
      if (A.cheb_a != T(0) && L.act) dn += A.cheb_a * A.dvec[g];
      if (L.act) A.dvec[g] = dn;
      v = A.x[g] + dn;
    } else {
      v = A.x[g] + A.omega * (A.b[g] - sum) / diag;
    }
  }
  if (L.act) A.y[g] = v;
}

// Apply item (C <= 32 copies: one lane per (point, copy); more: the serial path).
template <typename T, int OP, bool ST>
__device__ void interface_item(const FusedArgs<T>& A, int item, int lane) {
  const uint2 e = __ldg(A.clane + (int64_t)item * 32 + lane);
  if (((e.y >> 24) & 63) > 32) {
    interface_point_serial<T, OP, ST>(A, A.items[item], lane);
    return;
  }
  const ItemLane L = item_lane(e, lane, A.w, A.stride);
  const bool fixed = item_fixed<OP>(L, A.mask);
  T sv[kNDir], xv[kNDir];
  if (!fixed) item_load<T, ST>(A, L, sv, xv);
  item_finish<T, OP>(A, L, fixed, sv, xv);
}

}  // namespace
}  // namespace hg
