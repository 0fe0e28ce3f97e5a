// P1 kernels on the per-macro-cell vertex lattice.
//
// Storage: every macro cell holds its closed vertex lattice i+j+k <= n in
// t_{n+1} order (Sec. 4); points on macro faces/edges/vertices have one copy
// per containing cell and all copies are kept equal.
//
// An operator application (Sec. 5.2 apply(), stencil-based pattern with
// constant stencils precomputed per macro cell) is ONE launch of warp-sized
// work items of two kinds:
//  * interface items (first in the grid): points of a macro face/edge/vertex
//    (the ghost-layer exchange of Sec. 2 as an on-device gather).  Each lane
//    takes one (point, copy) pair, floor(32 / copies) points per item, and
//    loads its copy's partial stencil; the partials of a point are summed in
//    ascending cell order by lane exchanges and the sum is written to every
//    copy, so copies stay bit-identical and no second pass is needed;
//  * plane-window tiles: rows are contiguous in t_w order, so the points of
//    plane k form one run of offsets, and the i-1 / i+1 neighbours of an
//    interior point are the offsets g-1 / g+1 even where a window spans
//    several rows.  A warp takes 32 consecutive offsets (outputs at lanes
//    1..30) of one plane; relative to g, the other neighbour rows sit at
//    +len, -(len+1) (rows j+-1), +T(w-k-1)+len, +T(w-k-1) (plane k+1, rows
//    j, j-1), -(T(w-k)+len+1), -T(w-k) (plane k-1, rows j, j+1), with len the
//    lane's row length: seven coalesced loads per window, shuffles for the
//    shifted neighbours, no lanes lost to short rows beyond the halo lanes
//    and the boundary points.  A tile is a strip of up to kPlaneSteps
//    windows, software-pipelined: the next windows' loads are in flight
//    while one window is computed.
#include <cuda_runtime.h>

#include <algorithm>
#include <atomic>
#include <cmath>
#include <cstring>

#include "hg_internal.h"
#include "hg_p1dev.cuh"

namespace hg {

namespace {

constexpr int kBlock = 256;
constexpr int kWarps = kBlock / 32;

// One window of a plane tile in registers: the seven row values of the lane's
// point, its offset and whether it is an output (ST: and the point's own
// stored stencil).
template <typename T, bool ST>
struct PlaneWin {
  T c, up, dn, p1c, p1m, m1c, m1p;
  int g;
  bool ok;
  T s[ST ? kNDir : 1];
  T inv;  // ST: 1 / centre weight
};

// Lane position inside a plane: offset g, row j, column r, row length len.
struct PlanePos {
  int g, r, len, j;
};

// Advance the lane by one window (30 offsets) and issue its seven loads.
// Lanes are placed up to gb+1 (the row end after the last interior point,
// whose values the last output takes by shuffle); the row walk stays inside
// the plane and lanes past gb+1 load at gb+1 (row length 3): in bounds, never
// stored.
// PAT = kPat7: the cell stencils vanish outside the seven-point subset
// (centre, +-(1,0,0), +-(1,-1,0), +-(0,-1,1)); the rows without weights are
// not loaded (planes k+-1 then need only one row each).
template <typename T, bool ST, int PAT = 0>
__device__ __forceinline__ void plane_load(PlaneWin<T, ST>& W, const T* __restrict__ x,
                                           const T* __restrict__ sst, PlanePos& P, bool advance,
                                           int gb, int Tp, int Tm, bool halo) {
  if (advance) {
    P.g += 30;
    P.r += 30;
    while (P.r >= P.len && P.g <= gb + 1) { P.r -= P.len; --P.len; ++P.j; }
  }
  const bool in = P.g <= gb + 1;
  const int gq = in ? P.g : gb + 1, lq = in ? P.len : 3;
  W.ok = in && P.g <= gb && !halo && P.r >= 1 && P.r <= P.len - 2;
  W.g = gq;
  W.c = __ldg(x + gq);
  W.up = __ldg(x + gq + lq);
  W.dn = __ldg(x + gq - lq - 1);
  if (PAT != kPat7) W.p1c = __ldg(x + gq + Tp + lq);
  W.p1m = __ldg(x + gq + Tp);
  if (PAT != kPat7) W.m1c = __ldg(x + gq - Tm - lq - 1);
  W.m1p = __ldg(x + gq - Tm);
  if (ST) {
    // only output lanes read weights: 64 B (FP32) per point, contiguous over the window
    if (W.ok) {
      load_sten16(sst + 16 * (int64_t)gq, W.s, W.inv);
    } else {
#pragma unroll
      for (int d = 0; d < kNDir; ++d) W.s[d] = T(0);
      W.inv = T(0);
    }
  }
}

// The 15-point stencil of one window from registers and shuffles, stored.
// With PAT = kPat7 the terms of the eight zero weights are left out; adding
// an exact zero changes no sum, so the result is the same bits.
template <typename T, int OP, bool ST, int PAT = 0>
__device__ __forceinline__ void plane_compute(const FusedArgs<T>& A, const PlaneWin<T, ST>& W,
                                              const T sc[kNDir], T wdc, int64_t base,
                                              T* __restrict__ y) {
  const T* s = ST ? W.s : sc;
  const T cm = __shfl_up_sync(0xffffffffu, W.c, 1), cp = __shfl_down_sync(0xffffffffu, W.c, 1);
  const T upm = __shfl_up_sync(0xffffffffu, W.up, 1);
  const T dnp = __shfl_down_sync(0xffffffffu, W.dn, 1);
  T acc;
  if (PAT == kPat7) {
    const T a0 = s[0] * W.c + s[1] * cp + s[2] * cm + s[7] * upm + s[8] * dnp;
    acc = a0 + (s[11] * W.p1m + s[12] * W.m1p);
  } else {
    const T p1cm = __shfl_up_sync(0xffffffffu, W.p1c, 1);
    const T p1mp = __shfl_down_sync(0xffffffffu, W.p1m, 1);
    const T m1cp = __shfl_down_sync(0xffffffffu, W.m1c, 1);
    const T m1pm = __shfl_up_sync(0xffffffffu, W.m1p, 1);
    const T a0 = s[0] * W.c + s[1] * cp + s[2] * cm + s[3] * W.up + s[4] * W.dn + s[7] * upm +
                 s[8] * dnp;
    const T a1 = s[5] * W.p1c + s[9] * p1cm + s[11] * W.p1m + s[13] * p1mp;
    const T a2 = s[6] * W.m1c + s[10] * m1cp + s[12] * W.m1p + s[14] * m1pm;
    acc = a0 + (a1 + a2);
  }
  if (W.ok) {
    const int idx = W.g;
    const T wd = !ST ? wdc
                     : (OP == OP_JACOBI || OP == OP_CHEB) ? A.omega * W.inv
                     : OP == OP_GS                        ? W.inv
                                                          : T(0);
    if (OP == OP_APPLY) {
      y[idx] = A.mode == HG_ADD ? y[idx] + acc : acc;
    } else if (OP == OP_RESID) {
      y[idx] = A.b[base + idx] - acc;
    } else if (OP == OP_GS) {
      y[idx] = A.colour[base + idx] == A.gs_colour ? W.c + (A.b[base + idx] - acc) * wd : W.c;
    } else if (OP == OP_CHEB) {
      T dn = (A.b[base + idx] - acc) * wd;
      if (A.cheb_a != T(0)) dn += A.cheb_a * A.dvec[base + idx];
      A.dvec[base + idx] = dn;
      y[idx] = W.c + dn;
    } else {
      y[idx] = W.c + (A.b[base + idx] - acc) * wd;
    }
  }
}

// Plane-window tile t (see the file comment): its windows in order, the loads
// of the next D windows in flight while one is computed (D = 0, 1 or 2;
// three rotating register sets for D = 2).
template <typename T, int OP, int D, bool ST, int PAT = 0>
__device__ __forceinline__ void plane_tile(const FusedArgs<T>& A, int t, int lane) {
  const int cell = t / A.n_tiles_cell;
  const int4 tl = A.tiles[t - cell * A.n_tiles_cell];
  const int k = tl.x & 0xffff, nwin = tl.x >> 16;
  const int w = A.w, n = A.n;
  const int64_t base = (int64_t)cell * A.stride;
  const T* __restrict__ x = A.x + base;
  T* __restrict__ y = A.y + base;
  const int Tp = ntri32(w - k - 1), Tm = ntri32(w - k);
  const int gb = row_start(w, n - k - 2, k) + 1;  // last interior offset of the plane
  T s[kNDir];
  T wd = T(0);
  const T* __restrict__ sst = ST ? A.sst + 16 * base : nullptr;
  if (!ST) {
    const T* __restrict__ S = A.sten + (int64_t)cell * 256;
#pragma unroll
    for (int d = 0; d < kNDir; ++d) s[d] = __ldg(S + d);
    wd = (OP == OP_JACOBI || OP == OP_CHEB) ? A.omega / s[0] : OP == OP_GS ? T(1) / s[0] : T(0);
  }
  const bool halo = lane == 0 || lane == 31;
  PlanePos P;
  P.j = tl.z >> 16;
  P.r = (tl.z & 0xffff) + lane;
  P.len = w - k - P.j;
  P.g = tl.y + lane;
  while (P.r >= P.len && P.g <= gb + 1) { P.r -= P.len; --P.len; ++P.j; }
  PlaneWin<T, ST> W0, W1, W2;
  if (D == 0) {
    for (int q = 0; q < nwin; ++q) {
      plane_load<T, ST, PAT>(W0, x, sst, P, q > 0, gb, Tp, Tm, halo);
      plane_compute<T, OP, ST, PAT>(A, W0, s, wd, base, y);
    }
  } else if (D == 1) {
    plane_load<T, ST, PAT>(W0, x, sst, P, false, gb, Tp, Tm, halo);
    for (int q = 0; q < nwin; q += 2) {
      if (q + 1 < nwin) plane_load<T, ST, PAT>(W1, x, sst, P, true, gb, Tp, Tm, halo);
      plane_compute<T, OP, ST, PAT>(A, W0, s, wd, base, y);
      if (q + 1 < nwin) {
        if (q + 2 < nwin) plane_load<T, ST, PAT>(W0, x, sst, P, true, gb, Tp, Tm, halo);
        plane_compute<T, OP, ST, PAT>(A, W1, s, wd, base, y);
      }
    }
  } else {
    plane_load<T, ST, PAT>(W0, x, sst, P, false, gb, Tp, Tm, halo);
    if (nwin > 1) plane_load<T, ST, PAT>(W1, x, sst, P, true, gb, Tp, Tm, halo);
    for (int q = 0; q < nwin; q += 3) {
      if (q + 2 < nwin) plane_load<T, ST, PAT>(W2, x, sst, P, true, gb, Tp, Tm, halo);
      plane_compute<T, OP, ST, PAT>(A, W0, s, wd, base, y);
      if (q + 1 < nwin) {
        if (q + 3 < nwin) plane_load<T, ST, PAT>(W0, x, sst, P, true, gb, Tp, Tm, halo);
        plane_compute<T, OP, ST, PAT>(A, W1, s, wd, base, y);
      }
      if (q + 2 < nwin) {
        if (q + 4 < nwin) plane_load<T, ST, PAT>(W1, x, sst, P, true, gb, Tp, Tm, halo);
        plane_compute<T, OP, ST, PAT>(A, W2, s, wd, base, y);
      }
    }
  }
}

// Column-march item t: lane l holds interior column i = i0 + l of plane k and
// marches rows j0..j1-1.  The centre row's three values (i-1, i, i+1) of the
// next row are loaded one step ahead and rotate into the centre; the row
// below's i+1 (and i) is the previous centre; the other neighbours are one
// load each.  Columns past a row's last interior point are clamped to it:
// their loads stay on interior points' neighbourhoods (in bounds) and they
// store nothing.  The stencil sums are formed in the same order as in
// plane_compute, so both kernels give the same bits.
template <typename T, int OP, int PAT>
__device__ __forceinline__ void march_item(const FusedArgs<T>& A, int t, int lane) {
  const int cell = t / A.n_march_cell;
  const int2 it = A.march[t - cell * A.n_march_cell];
  const int k = it.x & 0xffff, i0 = it.x >> 16, j0 = it.y & 0xffff, j1 = it.y >> 16;
  const int w = A.w;
  const int64_t base = (int64_t)cell * A.stride;
  const T* __restrict__ x = A.x + base;
  T* __restrict__ y = A.y + base;
  T s[kNDir];
  {
    const T* __restrict__ S = A.sten + (int64_t)cell * 256;
#pragma unroll
    for (int d = 0; d < kNDir; ++d) s[d] = __ldg(S + d);
  }
  const T wd = (OP == OP_JACOBI || OP == OP_CHEB) ? A.omega / s[0] : OP == OP_GS ? T(1) / s[0] : T(0);
  const int Tp = ntri32(w - k - 1), Tm = ntri32(w - k);
  const int i = i0 + lane;
  int len = w - k - j0;
  int r0 = row_start(w, j0, k);
  int ic = min(i, len - 2);
  T cm = __ldg(x + r0 + ic - 1), cc = __ldg(x + r0 + ic), cp = __ldg(x + r0 + ic + 1);
  // row j0 - 1 at i and i + 1
  T dnc = __ldg(x + r0 - len - 1 + ic), dnp = __ldg(x + r0 - len + ic);
  for (int j = j0; j < j1; ++j) {
    ic = min(i, len - 2);
    const int rjp = r0 + len;
    const T nm = __ldg(x + rjp + ic - 1), nc = __ldg(x + rjp + ic), np = __ldg(x + rjp + ic + 1);
    const T p1m = __ldg(x + r0 + Tp + ic), m1p = __ldg(x + r0 - Tm + ic);
    T acc;
    if (PAT == kPat7) {
      const T a0 = s[0] * cc + s[1] * cp + s[2] * cm + s[7] * nm + s[8] * dnp;
      acc = a0 + (s[11] * p1m + s[12] * m1p);
    } else {
      const int rkp = r0 + Tp + len, rkm = r0 - Tm - len - 1;
      const T p1c = __ldg(x + rkp + ic), p1cm = __ldg(x + rkp + ic - 1);
      const T p1mp = __ldg(x + r0 + Tp + ic + 1);
      const T m1c = __ldg(x + rkm + ic), m1cp = __ldg(x + rkm + ic + 1);
      const T m1pm = __ldg(x + r0 - Tm + ic - 1);
      const T a0 = s[0] * cc + s[1] * cp + s[2] * cm + s[3] * nc + s[4] * dnc + s[7] * nm +
                   s[8] * dnp;
      const T a1 = s[5] * p1c + s[9] * p1cm + s[11] * p1m + s[13] * p1mp;
      const T a2 = s[6] * m1c + s[10] * m1cp + s[12] * m1p + s[14] * m1pm;
      acc = a0 + (a1 + a2);
    }
    if (i <= len - 2) {
      const int idx = r0 + i;
      if (OP == OP_APPLY) {
        y[idx] = A.mode == HG_ADD ? y[idx] + acc : acc;
      } else if (OP == OP_RESID) {
        y[idx] = A.b[base + idx] - acc;
      } else if (OP == OP_GS) {
        y[idx] = A.colour[base + idx] == A.gs_colour ? cc + (A.b[base + idx] - acc) * wd : cc;
      } else if (OP == OP_CHEB) {
        T dn = (A.b[base + idx] - acc) * wd;
        if (A.cheb_a != T(0)) dn += A.cheb_a * A.dvec[base + idx];
        A.dvec[base + idx] = dn;
        y[idx] = cc + dn;
      } else {
        y[idx] = cc + (A.b[base + idx] - acc) * wd;
      }
    }
    dnc = cc;
    dnp = cp;
    cm = nm;
    cc = nc;
    cp = np;
    r0 = rjp;
    --len;
  }
}

template <typename T, int OP, int PAT = 0>
__global__ void __launch_bounds__(kBlock, 4) p1_march_kernel(FusedArgs<T> A) {
  const int lane = threadIdx.x & 31;
  const int wg = blockIdx.x * kWarps + (threadIdx.x >> 5);
  if ((int)blockIdx.x < A.nb_items) {
    if (wg < A.n_items) interface_item<T, OP, false>(A, wg, lane);
  } else {
    const int t = wg - A.nb_items * kWarps;
    if (t < A.n_march) march_item<T, OP, PAT>(A, t, lane);
  }
}

// Block `blk` of one operator application: interface items first, then tiles.
template <typename T, int OP, int R, bool ST = false, int PAT = 0>
__device__ __forceinline__ void p1_block(const FusedArgs<T>& A, int blk) {
  const int lane = threadIdx.x & 31;
  const int wg = blk * kWarps + (threadIdx.x >> 5);
  if (blk < A.nb_items) {
    if (wg < A.n_items) interface_item<T, OP, ST>(A, wg, lane);
  } else {
    const int t = wg - A.nb_items * kWarps;
    if (t < A.n_tiles) plane_tile<T, OP, R, ST, PAT>(A, t, lane);
  }
}

// Windows of a plane tile whose loads are in flight while one is computed.
#ifndef HG_P1_PREFETCH
#define HG_P1_PREFETCH 1
#endif
constexpr int kPlanePrefetch = HG_P1_PREFETCH;

// Resident blocks per SM the register budget is sized for (FP32 / FP64).
#ifndef HG_P1_MIN_BLOCKS_F32
#define HG_P1_MIN_BLOCKS_F32 3
#endif
template <typename T>
constexpr int min_blocks() { return sizeof(T) == 4 ? HG_P1_MIN_BLOCKS_F32 : 2; }

template <typename T, int OP, int PAT = 0>
__global__ void __launch_bounds__(kBlock, min_blocks<T>()) p1_fused_kernel(FusedArgs<T> A) {
  p1_block<T, OP, kPlanePrefetch, false, PAT>(A, blockIdx.x);
}

// Stored-stencil form (grid-aware precomputation of a variable-coefficient
// operator): the 64 B (FP32) stencil of each output point streams from HBM
// with the window's x rows.  Prefetch depth and resident blocks per SM are
// tuning constants (the weights' registers set the budget): one window in
// flight at 3-4 blocks per SM beats two windows at 2 blocks per SM.
#ifndef HG_STORED_PREFETCH
#define HG_STORED_PREFETCH 0
#endif
#ifndef HG_STORED_MIN_BLOCKS
#define HG_STORED_MIN_BLOCKS 3
#endif
template <typename T, int OP>
__global__ void __launch_bounds__(kBlock, HG_STORED_MIN_BLOCKS) p1_stored_kernel(FusedArgs<T> A) {
  p1_block<T, OP, HG_STORED_PREFETCH, true>(A, blockIdx.x);
}

// Index of the problem owning unit u: base[p] <= u < base[p+1].
__device__ __forceinline__ int unit_problem(const int* __restrict__ base, int nprob, int u) {
  int lo = 0, hi = nprob - 1;
  while (lo < hi) {
    const int mid = (lo + hi + 1) >> 1;
    if (__ldg(base + mid) <= u) lo = mid; else hi = mid - 1;
  }
  return lo;
}

// Batched persistent form: units u (one per block of each problem's grid,
// problems concatenated) are taken in a grid-stride loop.
template <typename T, int OP, int R>
__global__ void __launch_bounds__(kBlock, min_blocks<T>()) p1_batched_kernel(
    const FusedArgs<T>* __restrict__ descs, const int* __restrict__ base, int nprob) {
  const int total = __ldg(base + nprob);
  for (int u = blockIdx.x; u < total; u += gridDim.x) {
    const int p = unit_problem(base, nprob, u);
    p1_block<T, OP, R>(descs[p], u - __ldg(base + p));
  }
}

template <typename T>
FusedArgs<T> fused_args(const LevelDev& L, const StencilArgs& a, int n_items) {
  FusedArgs<T> A;
  A.n = L.n;
  A.w = L.w;
  A.stride = L.cell_stride;
  A.flags = L.cls_flags;
  A.tiles = L.ptiles;
  A.n_tiles_cell = L.n_ptiles_cell;
  A.n_tiles = L.n_ptiles_cell * L.ncells;
  A.items = L.citems;
  A.clane = L.clane;
  A.n_items = n_items;
  A.nb_items = (n_items + kWarps - 1) / kWarps;
  A.prims = L.prims;
  A.copies = L.copies;
  A.x = (const T*)a.x;
  A.b = (const T*)a.b;
  A.y = (T*)a.out;
  A.sten = (const T*)a.sten;
  A.sst = (const T*)a.sst;
  A.omega = (T)a.omega;
  A.mode = a.mode;
  A.mask = a.mask;
  A.colour = L.colour;
  A.gs_colour = a.colour;
  A.dvec = (T*)a.dvec;
  A.cheb_a = (T)a.cheb_a;
  A.err = L.err;
  A.march = L.march;
  A.n_march_cell = L.n_march_cell;
  A.n_march = L.n_march_cell * L.ncells;
  return A;
}

template <typename T, int OP>
int run_p1(const LevelDev& L, const StencilArgs& a, cudaStream_t s, bool march) {
  const int n_items = L.n_citems;
  FusedArgs<T> A = fused_args<T>(L, a, n_items);
  if (march && !a.sst) {
    const int grid = A.nb_items + (A.n_march + kWarps - 1) / kWarps;
    if (grid == 0) return HG_OK;
    if (a.pattern == kPat7)
      p1_march_kernel<T, OP, kPat7><<<grid, kBlock, 0, s>>>(A);
    else
      p1_march_kernel<T, OP><<<grid, kBlock, 0, s>>>(A);
    HG_CUDA(cudaGetLastError());
    return HG_OK;
  }
  const int grid = A.nb_items + (A.n_tiles + kWarps - 1) / kWarps;
  if (grid == 0) return HG_OK;
  if (a.sst)
    p1_stored_kernel<T, OP><<<grid, kBlock, 0, s>>>(A);
  else if (a.pattern == kPat7)
    p1_fused_kernel<T, OP, kPat7><<<grid, kBlock, 0, s>>>(A);
  else
    p1_fused_kernel<T, OP><<<grid, kBlock, 0, s>>>(A);
  HG_CUDA(cudaGetLastError());
  return HG_OK;
}

template <typename T>
int run_p1_op(const LevelDev& L, const StencilArgs& a, cudaStream_t s, bool march = false) {
  switch (a.op) {
    case OP_APPLY: return run_p1<T, OP_APPLY>(L, a, s, march);
    case OP_RESID: return run_p1<T, OP_RESID>(L, a, s, march);
    case OP_JACOBI: return run_p1<T, OP_JACOBI>(L, a, s, march);
    case OP_GS: return run_p1<T, OP_GS>(L, a, s, march);
    case OP_CHEB: return run_p1<T, OP_CHEB>(L, a, s, march);
  }
  set_error("unknown cell operation %d", a.op);
  return HG_ERR_INVALID_ARG;
}

// ------------------------------------------------------------ row items
// Row item r of a level: cell = r / ntri(w), then plane k and row j of the
// cell's lattice.  Plane k has w-k rows; R(k) = k(2w-k+1)/2 rows precede it.

// ------------------------------------------------------------ maps / dumps
__global__ void index_enumerate_kernel(int w, int64_t* out) {
  // one warp per row item of a single lattice, lanes over i
  const int lane = threadIdx.x & 31;
  const int r = blockIdx.x * kWarps + (threadIdx.x >> 5);
  if (r >= ntri32(w)) return;
  int cell, j, k;
  row_item(w, r, cell, j, k);
  const int r0 = row_start(w, j, k);
  for (int i = lane; i + j + k <= w - 1; i += 32)
    out[r0 + i] = (int64_t)i + ((int64_t)j << 20) + ((int64_t)k << 40);
}

__global__ void interface_dump_kernel(int n, int w, const int4* items, int n_items,
                                      const int32_t* item_prim, const IfacePrim* prims,
                                      const int32_t* pbase, const IfaceCopy* copies, int maxc,
                                      int64_t* out) {
  const int lane = threadIdx.x & 31;
  const int it = blockIdx.x * kWarps + (threadIdx.x >> 5);
  if (it >= n_items) return;
  const int4 item = items[it];
  const int prim = item_prim[it];
  const IfacePrim P = prims[prim];
  const int p = item.y + lane;
  if (p >= prim_points(P.dim, n)) return;
  int wts[3];
  prim_weights(P.dim, n, p, wts);
  int64_t* row = out + (int64_t)(pbase[prim] + p) * (2 * maxc + 1);
  row[0] = P.ncopies;
  for (int q = 0; q < maxc; ++q) {
    if (q < P.ncopies) {
      int i, j, k;
      const IfaceCopy c = copies[P.first_copy + q];
      copy_local_ijk(c, P.dim, wts, i, j, k);
      row[1 + 2 * q] = c.cell;
      row[2 + 2 * q] = tw32(w, i, j, k);
    } else {
      row[1 + 2 * q] = -1;
      row[2 + 2 * q] = -1;
    }
  }
}

// Stored <-> canonical copies; S is the source and D the destination element
// type (a conversion rounds to nearest).
template <typename S, typename D>
__global__ void gather_kernel(const S* __restrict__ st, const int64_t* __restrict__ rep, int64_t nu,
                              D* __restrict__ can) {
  for (int64_t u = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; u < nu;
       u += (int64_t)gridDim.x * blockDim.x)
    can[u] = (D)st[rep[u]];
}

template <typename S, typename D>
__global__ void scatter_kernel(const S* __restrict__ can, const int32_t* __restrict__ canon,
                               int64_t ns, D* __restrict__ st) {
  for (int64_t q = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; q < ns;
       q += (int64_t)gridDim.x * blockDim.x) {
    int32_t u = canon[q];
    if (u >= 0) st[q] = (D)can[u];
  }
}

// ---------------------------------------------------------- grid transfers
// Lattice rows per warp of the transfer kernels (consecutive in row-item order).
constexpr int kXferRows = 4;

// Restriction r_c = P^T r_f.  A coarse point I collects the fine points 2I
// (weight 1) and 2I +- d (weight 1/2, the midpoints of the coarse edges at I)
// that lie in the cell and are owned by it (each unique fine DoF counted once).
template <typename T>
__device__ __forceinline__ T restrict_partial(const T* __restrict__ rf, const uint8_t* fl, int nf,
                                              int I, int J, int K) {
  const int wf = nf + 1;
  T acc = T(0);
#pragma unroll
  for (int d = 0; d < kNDir; ++d) {
    int di, dj, dk;
    dir_offset(d, di, dj, dk);
    const int a = 2 * I + di, b = 2 * J + dj, c = 2 * K + dk;
    if (a < 0 || b < 0 || c < 0 || a + b + c > nf) continue;
    if (!(fl[point_class(nf, a, b, c)] & CF_OWNER)) continue;
    const T v = rf[tw32(wf, a, b, c)];
    acc += d == 0 ? v : T(0.5) * v;
  }
  return acc;
}

// Restriction of one fine/coarse level pair (blocks [0, nb_items) take coarse
// interface items, the rest coarse rows).
template <typename T>
struct RestrictDesc {
  int nf, nc;
  int64_t fstride, cstride;
  const uint8_t* flags;
  const int4* items;
  int n_items, nb_items;
  const IfaceCopy* copies;
  int n_rows;
  const T* rf;
  T* rc;
};

template <typename T>
__device__ __forceinline__ void restrict_block(const RestrictDesc<T>& D, int blk) {
  const int lane = threadIdx.x & 31;
  const int wg = blk * kWarps + (threadIdx.x >> 5);
  const int nf = D.nf, nc = D.nc, wc = nc + 1;
  if (blk < D.nb_items) {
    if (wg >= D.n_items) return;
    const int4 it = D.items[wg];
    IfacePrim P;
    P.dim = it.z & 15;
    P.ncopies = (it.z >> 4) & 255;
    P.dirichlet = (it.z >> 12) & 1;
    const int p = it.y + lane;
    if (p >= prim_points(P.dim, nc)) return;
    int wts[3];
    prim_weights(P.dim, nc, p, wts);
    const IfaceCopy* cp = D.copies + it.x;
    T v = T(0);
    if (!P.dirichlet) {
      for (int q = 0; q < P.ncopies; ++q) {
        int I, J, K;
        copy_local_ijk(cp[q], P.dim, wts, I, J, K);
        v += restrict_partial<T>(D.rf + (int64_t)cp[q].cell * D.fstride, D.flags + cp[q].cell * 16,
                                 nf, I, J, K);
      }
    }
    for (int q = 0; q < P.ncopies; ++q) {
      int I, J, K;
      copy_local_ijk(cp[q], P.dim, wts, I, J, K);
      D.rc[(int64_t)cp[q].cell * D.cstride + tw32(wc, I, J, K)] = v;
    }
    return;
  }
  const int r = (wg - D.nb_items * kWarps) * kXferRows;
  if (r >= D.n_rows) return;
  int cell, J, K;
  row_item(wc, r, cell, J, K);
  // coarse rows r .. r + kXferRows - 1 in row-item order (J inner, then K, then cell)
  for (int q = 0; q < kXferRows && r + q < D.n_rows; ++q) {
    const T* rf = D.rf + (int64_t)cell * D.fstride;
    T* rc = D.rc + (int64_t)cell * D.cstride;
    const uint8_t* fl = D.flags + cell * 16;
    const int r0 = row_start(wc, J, K);
    for (int I = lane; I + J + K <= nc; I += 32) {
      if (point_class(nc, I, J, K) != 0) continue;  // interface points: items above
      rc[r0 + I] = restrict_partial<T>(rf, fl, nf, I, J, K);
    }
    if (++J == wc - K) {
      J = 0;
      if (++K == wc) {
        K = 0;
        ++cell;
      }
    }
  }
}

template <typename T>
__global__ void __launch_bounds__(kBlock) restrict_kernel(RestrictDesc<T> D) {
  restrict_block<T>(D, blockIdx.x);
}

// Prolongation x_f += P e_c: fine points with even coordinates copy the coarse
// value; the others are midpoints of the coarse edge picked by the parity.
template <typename T>
struct ProlongDesc {
  int nf;
  int64_t fstride, cstride;
  const uint8_t* flags;
  int n_rows;
  const T* ec;
  T* xf;
};

// Coarse-edge direction of a fine point by coordinate parity p = i&1 |
// (j&1)<<1 | (k&1)<<2, one 2-bit field (offset + 1) per parity: p = 0 maps
// to (0,0,0), whose two endpoints coincide (0.5 (a + a) = a exactly).
constexpr unsigned kParDi = (1u << 0) | (2u << 2) | (1u << 4) | (0u << 6) | (1u << 8) | (0u << 10) |
                            (1u << 12) | (2u << 14);
constexpr unsigned kParDj = (1u << 0) | (1u << 2) | (2u << 4) | (2u << 6) | (1u << 8) | (1u << 10) |
                            (0u << 12) | (0u << 14);
constexpr unsigned kParDk = (1u << 0) | (1u << 2) | (1u << 4) | (1u << 6) | (2u << 8) | (2u << 10) |
                            (2u << 12) | (2u << 14);

template <typename T>
__device__ __forceinline__ void prolong_block(const ProlongDesc<T>& D, int blk) {
  const int lane = threadIdx.x & 31;
  const int r = (blk * kWarps + (threadIdx.x >> 5)) * kXferRows;
  const int nf = D.nf, wf = nf + 1, wc = nf / 2 + 1;
  if (r >= D.n_rows) return;
  int cell, j, k;
  row_item(wf, r, cell, j, k);
  // rows r .. r + kXferRows - 1 in row-item order (j inner, then k, then cell)
  for (int q = 0; q < kXferRows && r + q < D.n_rows; ++q) {
    const T* ec = D.ec + (int64_t)cell * D.cstride;
    T* xf = D.xf + (int64_t)cell * D.fstride;
    const uint8_t* fl = D.flags + cell * 16;
    const int r0 = row_start(wf, j, k);
    for (int i = lane; i + j + k <= nf; i += 32) {
      if (fl[point_class(nf, i, j, k)] & CF_DIRICHLET) continue;
      const int par2 = 2 * ((i & 1) | ((j & 1) << 1) | ((k & 1) << 2));
      const int di = (int)((kParDi >> par2) & 3u) - 1, dj = (int)((kParDj >> par2) & 3u) - 1,
                dk = (int)((kParDk >> par2) & 3u) - 1;
      const T a = ec[tw32(wc, (i - di) >> 1, (j - dj) >> 1, (k - dk) >> 1)];
      const T b = ec[tw32(wc, (i + di) >> 1, (j + dj) >> 1, (k + dk) >> 1)];
      xf[r0 + i] += T(0.5) * (a + b);
    }
    if (++j == wf - k) {
      j = 0;
      if (++k == wf) {
        k = 0;
        ++cell;
      }
    }
  }
}

template <typename T>
__global__ void __launch_bounds__(kBlock) prolong_kernel(ProlongDesc<T> D) {
  prolong_block<T>(D, blockIdx.x);
}

template <typename T>
__global__ void __launch_bounds__(kBlock) restrict_batched_kernel(
    const RestrictDesc<T>* __restrict__ descs, const int* __restrict__ base, int nprob) {
  const int total = __ldg(base + nprob);
  for (int u = blockIdx.x; u < total; u += gridDim.x) {
    const int p = unit_problem(base, nprob, u);
    restrict_block<T>(descs[p], u - __ldg(base + p));
  }
}

template <typename T>
__global__ void __launch_bounds__(kBlock) prolong_batched_kernel(
    const ProlongDesc<T>* __restrict__ descs, const int* __restrict__ base, int nprob) {
  const int total = __ldg(base + nprob);
  for (int u = blockIdx.x; u < total; u += gridDim.x) {
    const int p = unit_problem(base, nprob, u);
    prolong_block<T>(descs[p], u - __ldg(base + p));
  }
}

// ------------------------------------------------------------- reductions
// Deterministic FP64 dot over owned points: a fixed grid of kDotBlocks blocks
// strides over row items; one partial per block; one block adds the partials
// in a fixed tree order.
constexpr int kDotBlocks = 608;

template <typename T>
__global__ void __launch_bounds__(kBlock) dot_partial_kernel(int n, int64_t stride,
                                                             const uint8_t* flags, int n_rows,
                                                             const T* __restrict__ X,
                                                             const T* __restrict__ Y, int mask,
                                                             double* partial) {
  const int w = n + 1;
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  double acc = 0.0;
  for (int r = blockIdx.x * kWarps + warp; r < n_rows; r += gridDim.x * kWarps) {
    int cell, j, k;
    row_item(w, r, cell, j, k);
    const int64_t r0 = (int64_t)cell * stride + row_start(w, j, k);
    const uint8_t* fl = flags + cell * 16;
    for (int i = lane; i + j + k <= n; i += 32) {
      const uint8_t f = fl[point_class(n, i, j, k)];
      if (!(f & CF_OWNER)) continue;
      if (mask == HG_MASK_INNER && (f & CF_DIRICHLET)) continue;
      acc += (double)X[r0 + i] * (double)Y[r0 + i];
    }
  }
  __shared__ double red[kWarps];
  for (int o = 16; o > 0; o >>= 1) acc += __shfl_down_sync(0xffffffffu, acc, o);
  if (lane == 0) red[warp] = acc;
  __syncthreads();
  if (threadIdx.x == 0) {
    double t = 0.0;
    for (int q = 0; q < kWarps; ++q) t += red[q];
    partial[blockIdx.x] = t;
  }
}

__global__ void __launch_bounds__(1024) sum_partials_kernel(const double* partial, int np,
                                                            double* result) {
  __shared__ double red[1024];
  double acc = 0.0;
  for (int q = threadIdx.x; q < np; q += blockDim.x) acc += partial[q];
  red[threadIdx.x] = acc;
  __syncthreads();
  for (int o = blockDim.x / 2; o > 0; o >>= 1) {
    if (threadIdx.x < o) red[threadIdx.x] += red[threadIdx.x + o];
    __syncthreads();
  }
  if (threadIdx.x == 0) *result = red[0];
}

int grid_for(int64_t n) {
  int64_t g = (n + kBlock - 1) / kBlock;
  return (int)(g < 152 * 16 ? (g > 0 ? g : 1) : 152 * 16);
}

int blocks_for_warps(int64_t nw) { return (int)((nw + kWarps - 1) / kWarps); }
// Warps of the row part of one transfer launch (kXferRows rows each).
int64_t xfer_warps(int64_t n_rows) { return (n_rows + kXferRows - 1) / kXferRows; }

}  // namespace

namespace {
std::atomic<int> g_p1_kernel{HG_P1_KERNEL_AUTO};
// Stored points from which the streaming kernel pays off in AUTO mode
// (measured on GB300: 113 vs 134 us per apply at 18 M stored points, 20.6 vs
// 15.1 us at 2.2 M, FP64 slower at both).
constexpr int64_t kStreamAutoPoints = int64_t(8) << 20;
}  // namespace

int set_p1_kernel(int mode) {
  if (mode != HG_P1_KERNEL_AUTO && mode != HG_P1_KERNEL_WINDOWS && mode != HG_P1_KERNEL_STREAM &&
      mode != HG_P1_KERNEL_MARCH) {
    set_error("hg_set_p1_kernel: unknown mode %d", mode);
    return HG_ERR_INVALID_ARG;
  }
  g_p1_kernel.store(mode);
  return HG_OK;
}

int launch_p1_const(const LevelDev& L, int dtype, const StencilArgs& a, cudaStream_t s) {
  // constant stencils: the streaming kernel or the plane windows (see
  // hg_set_p1_kernel); stored stencils: the plane windows
  const int mode = g_p1_kernel.load();
  const bool stream = !a.sst && p1_stream_fits(L.w, dtype) &&
                      (mode == HG_P1_KERNEL_STREAM ||
                       (mode == HG_P1_KERNEL_AUTO && dtype == HG_F32 && L.n_stored >= kStreamAutoPoints));
  if (stream) return launch_p1_stream(L, dtype, a, s);
  const bool march = mode == HG_P1_KERNEL_MARCH;
  return dtype == HG_F64 ? run_p1_op<double>(L, a, s, march) : run_p1_op<float>(L, a, s, march);
}

int launch_index_enumerate(int w, int64_t* out, cudaStream_t s) {
  index_enumerate_kernel<<<blocks_for_warps(ntri32(w)), kBlock, 0, s>>>(w, out);
  HG_CUDA(cudaGetLastError());
  return HG_OK;
}

int launch_interface_dump(const LevelDev& L, int64_t* out, cudaStream_t s) {
  if (L.n_items == 0) return HG_OK;
  interface_dump_kernel<<<blocks_for_warps(L.n_items), kBlock, 0, s>>>(
      L.n, L.w, L.items, L.n_items, L.item_prim, L.prims, L.prim_point_base, L.copies,
      L.max_copies, out);
  HG_CUDA(cudaGetLastError());
  return HG_OK;
}

int launch_to_canonical(const LevelDev& L, int dtype, const void* st, void* can, cudaStream_t s,
                        int can_dtype) {
  if (can_dtype < 0) can_dtype = dtype;
  const int g = grid_for(L.n_unique);
  const int64_t* rep = L.canon_rep;
  const int64_t nu = L.n_unique;
  if (dtype == HG_F64 && can_dtype == HG_F64)
    gather_kernel<<<g, kBlock, 0, s>>>((const double*)st, rep, nu, (double*)can);
  else if (dtype == HG_F64)
    gather_kernel<<<g, kBlock, 0, s>>>((const double*)st, rep, nu, (float*)can);
  else if (can_dtype == HG_F64)
    gather_kernel<<<g, kBlock, 0, s>>>((const float*)st, rep, nu, (double*)can);
  else
    gather_kernel<<<g, kBlock, 0, s>>>((const float*)st, rep, nu, (float*)can);
  HG_CUDA(cudaGetLastError());
  return HG_OK;
}

int launch_from_canonical(const LevelDev& L, int dtype, const void* can, void* st,
                          cudaStream_t s, int can_dtype) {
  if (can_dtype < 0) can_dtype = dtype;
  const int g = grid_for(L.n_stored);
  const int32_t* cn = L.canon;
  const int64_t ns = L.n_stored;
  if (dtype == HG_F64 && can_dtype == HG_F64)
    scatter_kernel<<<g, kBlock, 0, s>>>((const double*)can, cn, ns, (double*)st);
  else if (dtype == HG_F64)
    scatter_kernel<<<g, kBlock, 0, s>>>((const float*)can, cn, ns, (double*)st);
  else if (can_dtype == HG_F64)
    scatter_kernel<<<g, kBlock, 0, s>>>((const double*)can, cn, ns, (float*)st);
  else
    scatter_kernel<<<g, kBlock, 0, s>>>((const float*)can, cn, ns, (float*)st);
  HG_CUDA(cudaGetLastError());
  return HG_OK;
}

template <typename T>
RestrictDesc<T> restrict_desc(const LevelDev& F, const LevelDev& C, const void* rf, void* rc) {
  RestrictDesc<T> D;
  D.nf = F.n;
  D.nc = C.n;
  D.fstride = F.cell_stride;
  D.cstride = C.cell_stride;
  D.flags = F.cls_flags;
  D.items = C.items;
  D.n_items = C.n_items;
  D.nb_items = blocks_for_warps(C.n_items);
  D.copies = C.copies;
  D.n_rows = C.ncells * ntri32(C.w);
  D.rf = (const T*)rf;
  D.rc = (T*)rc;
  return D;
}

template <typename T>
ProlongDesc<T> prolong_desc(const LevelDev& F, const LevelDev& C, const void* ec, void* xf) {
  ProlongDesc<T> D;
  D.nf = F.n;
  D.fstride = F.cell_stride;
  D.cstride = C.cell_stride;
  D.flags = F.cls_flags;
  D.n_rows = F.ncells * ntri32(F.w);
  D.ec = (const T*)ec;
  D.xf = (T*)xf;
  return D;
}

template <typename T>
static int run_restrict(const LevelDev& F, const LevelDev& C, const void* rf, void* rc,
                        cudaStream_t s) {
  const RestrictDesc<T> D = restrict_desc<T>(F, C, rf, rc);
  restrict_kernel<T><<<D.nb_items + blocks_for_warps(xfer_warps(D.n_rows)), kBlock, 0, s>>>(D);
  HG_CUDA(cudaGetLastError());
  return HG_OK;
}

int launch_restrict_p1(const LevelDev& F, const LevelDev& C, int dtype, const void* rf, void* rc,
                       cudaStream_t s) {
  return dtype == HG_F64 ? run_restrict<double>(F, C, rf, rc, s)
                         : run_restrict<float>(F, C, rf, rc, s);
}

int launch_prolong_p1(const LevelDev& F, const LevelDev& C, int dtype, const void* ec, void* xf,
                      cudaStream_t s) {
  if (dtype == HG_F64) {
    const ProlongDesc<double> D = prolong_desc<double>(F, C, ec, xf);
    prolong_kernel<double><<<blocks_for_warps(xfer_warps(D.n_rows)), kBlock, 0, s>>>(D);
  } else {
    const ProlongDesc<float> D = prolong_desc<float>(F, C, ec, xf);
    prolong_kernel<float><<<blocks_for_warps(xfer_warps(D.n_rows)), kBlock, 0, s>>>(D);
  }
  HG_CUDA(cudaGetLastError());
  return HG_OK;
}

// ------------------------------------------------------ batched descriptors
size_t p1_desc_bytes(int dtype) {
  return dtype == HG_F64 ? sizeof(FusedArgs<double>) : sizeof(FusedArgs<float>);
}

int p1_make_desc(const LevelDev& L, int dtype, const StencilArgs& a, void* dst, int* units) {
  const int n_items = L.n_citems;
  if (dtype == HG_F64) {
    const FusedArgs<double> A = fused_args<double>(L, a, n_items);
    memcpy(dst, &A, sizeof A);
    *units = A.nb_items + (A.n_tiles + kWarps - 1) / kWarps;
  } else {
    const FusedArgs<float> A = fused_args<float>(L, a, n_items);
    memcpy(dst, &A, sizeof A);
    *units = A.nb_items + (A.n_tiles + kWarps - 1) / kWarps;
  }
  return HG_OK;
}

size_t restrict_desc_bytes(int dtype) {
  return dtype == HG_F64 ? sizeof(RestrictDesc<double>) : sizeof(RestrictDesc<float>);
}

int restrict_make_desc(const LevelDev& F, const LevelDev& C, int dtype, const void* rf, void* rc,
                       void* dst, int* units) {
  if (dtype == HG_F64) {
    const RestrictDesc<double> D = restrict_desc<double>(F, C, rf, rc);
    memcpy(dst, &D, sizeof D);
    *units = D.nb_items + blocks_for_warps(xfer_warps(D.n_rows));
  } else {
    const RestrictDesc<float> D = restrict_desc<float>(F, C, rf, rc);
    memcpy(dst, &D, sizeof D);
    *units = D.nb_items + blocks_for_warps(xfer_warps(D.n_rows));
  }
  return HG_OK;
}

size_t prolong_desc_bytes(int dtype) {
  return dtype == HG_F64 ? sizeof(ProlongDesc<double>) : sizeof(ProlongDesc<float>);
}

int prolong_make_desc(const LevelDev& F, const LevelDev& C, int dtype, const void* ec, void* xf,
                      void* dst, int* units) {
  if (dtype == HG_F64) {
    const ProlongDesc<double> D = prolong_desc<double>(F, C, ec, xf);
    memcpy(dst, &D, sizeof D);
    *units = blocks_for_warps(xfer_warps(D.n_rows));
  } else {
    const ProlongDesc<float> D = prolong_desc<float>(F, C, ec, xf);
    memcpy(dst, &D, sizeof D);
    *units = blocks_for_warps(xfer_warps(D.n_rows));
  }
  return HG_OK;
}

template <typename T, int OP>
static void p1_batched_rows(int rows, const void* d, const int* base, int nprob, int grid,
                            cudaStream_t s) {
  const FusedArgs<T>* D = (const FusedArgs<T>*)d;
  if (rows <= 0)
    p1_batched_kernel<T, OP, 0><<<grid, kBlock, 0, s>>>(D, base, nprob);
  else if (rows <= 1)
    p1_batched_kernel<T, OP, 1><<<grid, kBlock, 0, s>>>(D, base, nprob);
  else
    p1_batched_kernel<T, OP, 2><<<grid, kBlock, 0, s>>>(D, base, nprob);
}

int launch_p1_batched(int dtype, int op, int rows, const void* descs, const int* base, int nprob,
                      int grid, cudaStream_t s) {
  if (nprob <= 0) return HG_OK;
  if (dtype == HG_F64) {
    if (op == OP_APPLY) p1_batched_rows<double, OP_APPLY>(rows, descs, base, nprob, grid, s);
    else if (op == OP_RESID) p1_batched_rows<double, OP_RESID>(rows, descs, base, nprob, grid, s);
    else p1_batched_rows<double, OP_JACOBI>(rows, descs, base, nprob, grid, s);
  } else {
    if (op == OP_APPLY) p1_batched_rows<float, OP_APPLY>(rows, descs, base, nprob, grid, s);
    else if (op == OP_RESID) p1_batched_rows<float, OP_RESID>(rows, descs, base, nprob, grid, s);
    else p1_batched_rows<float, OP_JACOBI>(rows, descs, base, nprob, grid, s);
  }
  HG_CUDA(cudaGetLastError());
  return HG_OK;
}

int launch_restrict_batched(int dtype, const void* descs, const int* base, int nprob, int grid,
                            cudaStream_t s) {
  if (nprob <= 0) return HG_OK;
  if (dtype == HG_F64)
    restrict_batched_kernel<double><<<grid, kBlock, 0, s>>>((const RestrictDesc<double>*)descs,
                                                            base, nprob);
  else
    restrict_batched_kernel<float><<<grid, kBlock, 0, s>>>((const RestrictDesc<float>*)descs,
                                                           base, nprob);
  HG_CUDA(cudaGetLastError());
  return HG_OK;
}

int launch_prolong_batched(int dtype, const void* descs, const int* base, int nprob, int grid,
                           cudaStream_t s) {
  if (nprob <= 0) return HG_OK;
  if (dtype == HG_F64)
    prolong_batched_kernel<double><<<grid, kBlock, 0, s>>>((const ProlongDesc<double>*)descs,
                                                           base, nprob);
  else
    prolong_batched_kernel<float><<<grid, kBlock, 0, s>>>((const ProlongDesc<float>*)descs, base,
                                                          nprob);
  HG_CUDA(cudaGetLastError());
  return HG_OK;
}

int64_t dot_scratch_len(const LevelDev&) { return kDotBlocks; }

int launch_dot(const LevelDev& L, int dtype, const void* x, const void* y, int mask,
               double* scratch, double* result_dev, cudaStream_t s) {
  const int n_rows = L.ncells * ntri32(L.w);
  if (dtype == HG_F64)
    dot_partial_kernel<double><<<kDotBlocks, kBlock, 0, s>>>(
        L.n, L.cell_stride, L.cls_flags, n_rows, (const double*)x, (const double*)y, mask,
        scratch);
  else
    dot_partial_kernel<float><<<kDotBlocks, kBlock, 0, s>>>(
        L.n, L.cell_stride, L.cls_flags, n_rows, (const float*)x, (const float*)y, mask, scratch);
  HG_CUDA(cudaGetLastError());
  sum_partials_kernel<<<1, 1024, 0, s>>>(scratch, kDotBlocks, result_dev);
  HG_CUDA(cudaGetLastError());
  return HG_OK;
}

}  // namespace hg
