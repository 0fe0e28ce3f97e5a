// P2 grid transfers (multigrid by design, Sec. 5.1: nested P2 spaces on the
// refinement hierarchy).  Prolongation is quadratic interpolation: a fine P2
// DoF takes the value of the coarse P2 function at its point; restriction is
// the exact transpose, r_c = P^T r_f.
//
// Fine P2 level l lives on lattice F (level l+1), coarse level l-1 on lattice
// C (level l).  In F units the coarse micro-cells are anchored at multiples of
// 4, so a fine point f = 4p + r, r in {0..3}^3, lies in one coarse micro-cell
// anchored at p chosen by r alone: the unit cube [p, p+1]^3 splits into the
// I-up cell (|r| <= 4), the octahedron (4 < |r| <= 8, four cells around the
// inner edge) and the I-down cell (|r| > 8), Sec. 3.2.  Its barycentric
// coordinates are multiples of 1/4, so every weight phi(f) is an exact dyadic
// rational.  The host builds, once, per class r the nonzero coarse basis
// values (<= 10 terms, coarse DoFs as C-lattice offsets from 2p) and, per
// parity class of a coarse DoF, the transposed list of (fine offset from 2c,
// weight); every fine point with a nonzero weight lies in its containing
// coarse cell, which makes the lists complete.
//
// Interface points: prolongation values of macro-interface fine points are
// computed once (from the first copy's cell) and added to every copy;
// restriction partials of macro-interface coarse DoFs count each fine point
// in its owner cell only and are summed over the copies in ascending cell
// order -- copies stay bit-identical in both.
#include <cuda_runtime.h>

#include <cstring>
#include <mutex>
#include <string>

#include "hg_internal.h"

namespace hg {

namespace {

constexpr int kXBlock = 256;
constexpr int kXWarps = kXBlock / 32;
constexpr int kMaxRes = 320;  // 290 entries for the 14-point P2 structure

__constant__ int c_pro_n[64];
__constant__ int c_pro_off[64][10];  // dx | dy << 2 | dz << 4 (C units, 0..2)
__constant__ double c_pro_w64[64][10];
__constant__ float c_pro_w32[64][10];
__constant__ int c_res_start[9];     // per parity class (x | y << 1 | z << 2)
__constant__ int c_res_delta[kMaxRes];  // (dx+8) | (dy+8) << 5 | (dz+8) << 10 (F units)
__constant__ double c_res_w64[kMaxRes];
__constant__ float c_res_w32[kMaxRes];

template <typename T>
__device__ __forceinline__ T pro_w(int c, int t);
template <>
__device__ __forceinline__ double pro_w<double>(int c, int t) { return c_pro_w64[c][t]; }
template <>
__device__ __forceinline__ float pro_w<float>(int c, int t) { return c_pro_w32[c][t]; }
template <typename T>
__device__ __forceinline__ T res_w(int e);
template <>
__device__ __forceinline__ double res_w<double>(int e) { return c_res_w64[e]; }
template <>
__device__ __forceinline__ float res_w<float>(int e) { return c_res_w32[e]; }

const int kOff[6][4][3] = {
    {{0, 0, 0}, {1, 0, 0}, {0, 1, 0}, {0, 0, 1}},
    {{1, 1, 0}, {1, 0, 1}, {0, 1, 1}, {1, 1, 1}},
    {{0, 1, 0}, {1, 0, 1}, {1, 0, 0}, {0, 0, 1}},
    {{0, 1, 0}, {1, 0, 1}, {0, 0, 1}, {0, 1, 1}},
    {{0, 1, 0}, {1, 0, 1}, {0, 1, 1}, {1, 1, 0}},
    {{0, 1, 0}, {1, 0, 1}, {1, 1, 0}, {1, 0, 0}}};
const int kEdgeV[6][2] = {{0, 1}, {0, 2}, {0, 3}, {1, 2}, {1, 3}, {2, 3}};

// 4 * barycentric coordinates of 4r (r in quarter units) in cell type t, by
// Cramer's rule on integers; false if the point is outside the cell.
bool bary4(int t, const int r4[3], int l4[4]) {
  int M[3][3], rhs[3];
  for (int d = 0; d < 3; ++d) {
    for (int a = 0; a < 3; ++a) M[d][a] = kOff[t][a + 1][d] - kOff[t][0][d];
    rhs[d] = r4[d] - 4 * kOff[t][0][d];
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
    if (num % D) return false;  // cannot happen for quarter points
    l4[a + 1] = num / D;
    sum += l4[a + 1];
  }
  l4[0] = 4 - sum;
  for (int a = 0; a < 4; ++a)
    if (l4[a] < 0) return false;
  return true;
}

std::once_flag g_tables_once;
int g_tables_status = HG_OK;

int build_tables() {
  int pn[64] = {}, poff[64][10] = {};
  double pw[64][10] = {};
  for (int cz = 0; cz < 4; ++cz)
    for (int cy = 0; cy < 4; ++cy)
      for (int cx = 0; cx < 4; ++cx) {
        const int cl = cx + 4 * cy + 16 * cz, r4[3] = {cx, cy, cz}, s = cx + cy + cz;
        int t0 = 0, t1 = 0;
        if (s <= 4) t0 = t1 = 0;
        else if (s > 8) t0 = t1 = 1;
        else { t0 = 2; t1 = 5; }
        int t = -1, l4[4];
        for (int tt = t0; tt <= t1 && t < 0; ++tt)
          if (bary4(tt, r4, l4)) t = tt;
        if (t < 0) {
          set_error("P2 transfer table: no coarse cell for class %d", cl);
          return HG_ERR_INVALID_ARG;
        }
        double wsum = 0.0;
        auto add = [&](const int o[3], double w) {
          if (w == 0.0) return;
          poff[cl][pn[cl]] = o[0] | (o[1] << 2) | (o[2] << 4);
          pw[cl][pn[cl]] = w;
          ++pn[cl];
          wsum += w;
        };
        for (int a = 0; a < 4; ++a) {
          const int o[3] = {2 * kOff[t][a][0], 2 * kOff[t][a][1], 2 * kOff[t][a][2]};
          add(o, l4[a] * (l4[a] - 2) / 8.0);  // l (2l - 1) with l = l4 / 4
        }
        for (int e = 0; e < 6; ++e) {
          const int a = kEdgeV[e][0], b = kEdgeV[e][1];
          const int o[3] = {kOff[t][a][0] + kOff[t][b][0], kOff[t][a][1] + kOff[t][b][1],
                            kOff[t][a][2] + kOff[t][b][2]};
          add(o, l4[a] * l4[b] / 4.0);  // 4 l_a l_b
        }
        if (wsum != 1.0) {
          set_error("P2 transfer table: weights of class %d do not sum to 1", cl);
          return HG_ERR_INVALID_ARG;
        }
      }
  // transposed lists per coarse parity class
  std::vector<int> rd[8];
  std::vector<double> rw[8];
  for (int cl = 0; cl < 64; ++cl)
    for (int q = 0; q < pn[cl]; ++q) {
      const int o = poff[cl][q];
      const int ox = o & 3, oy = (o >> 2) & 3, oz = (o >> 4) & 3;
      const int par = (ox & 1) | ((oy & 1) << 1) | ((oz & 1) << 2);
      const int dx = (cl & 3) - 2 * ox, dy = ((cl >> 2) & 3) - 2 * oy, dz = (cl >> 4) - 2 * oz;
      rd[par].push_back((dx + 8) | ((dy + 8) << 5) | ((dz + 8) << 10));
      rw[par].push_back(pw[cl][q]);
    }
  int start[9] = {0}, delta[kMaxRes] = {};
  double w64[kMaxRes] = {};
  float w32[kMaxRes] = {};
  for (int p = 0; p < 8; ++p) {
    start[p + 1] = start[p] + (int)rd[p].size();
    if (start[p + 1] > kMaxRes) {
      set_error("P2 transfer table: restriction lists too long");
      return HG_ERR_INVALID_ARG;
    }
    for (size_t q = 0; q < rd[p].size(); ++q) {
      delta[start[p] + q] = rd[p][q];
      w64[start[p] + q] = rw[p][q];
      w32[start[p] + q] = (float)rw[p][q];
    }
  }
  float pw32[64][10];
  for (int c = 0; c < 64; ++c)
    for (int q = 0; q < 10; ++q) pw32[c][q] = (float)pw[c][q];
  HG_CUDA(cudaMemcpyToSymbol(c_pro_n, pn, sizeof pn));
  HG_CUDA(cudaMemcpyToSymbol(c_pro_off, poff, sizeof poff));
  HG_CUDA(cudaMemcpyToSymbol(c_pro_w64, pw, sizeof pw));
  HG_CUDA(cudaMemcpyToSymbol(c_pro_w32, pw32, sizeof pw32));
  HG_CUDA(cudaMemcpyToSymbol(c_res_start, start, sizeof start));
  HG_CUDA(cudaMemcpyToSymbol(c_res_delta, delta, sizeof delta));
  HG_CUDA(cudaMemcpyToSymbol(c_res_w64, w64, sizeof w64));
  HG_CUDA(cudaMemcpyToSymbol(c_res_w32, w32, sizeof w32));
  return HG_OK;
}

int ensure_tables() {
  static std::string msg;
  std::call_once(g_tables_once, [] {
    g_tables_status = build_tables();
    if (g_tables_status) msg = hg_last_error();
  });
  if (g_tables_status) set_error("P2 transfer tables could not be built: %s", msg.c_str());
  return g_tables_status;
}

template <typename T>
struct XDesc {
  int nf, nc;                 // intervals of the F and C lattices
  int64_t fstride, cstride;
  const uint8_t* fflags;      // per (cell, class) flags of F
  const int4* items;          // interface items (32 points) of the lattice swept
  int n_items, nb_items;
  const IfaceCopy* copies;
  int n_rows;                 // rows of the lattice swept (all cells)
  const T* src;
  T* dst;
};

// Value of the coarse P2 function at fine point (I,J,K) of one cell.
template <typename T>
__device__ __forceinline__ T p2_interp(const T* __restrict__ ec, int wc, int I, int J, int K) {
  const int cl = (I & 3) | ((J & 3) << 2) | ((K & 3) << 4);
  const int px = 2 * (I >> 2), py = 2 * (J >> 2), pz = 2 * (K >> 2);
  const int nt = c_pro_n[cl];
  T v = T(0);
  for (int q = 0; q < nt; ++q) {
    const int o = c_pro_off[cl][q];
    v += pro_w<T>(cl, q) * ec[tw32(wc, px + (o & 3), py + ((o >> 2) & 3), pz + ((o >> 4) & 3))];
  }
  return v;
}

// Partial of coarse DoF (i,j,k) of one cell: owned fine points of the cell.
template <typename T>
__device__ __forceinline__ T p2_restrict_partial(const T* __restrict__ rf, const uint8_t* fl,
                                                 int nf, int i, int j, int k) {
  const int par = (i & 1) | ((j & 1) << 1) | ((k & 1) << 2);
  const int wf = nf + 1;
  T v = T(0);
  for (int e = c_res_start[par]; e < c_res_start[par + 1]; ++e) {
    const int d = c_res_delta[e];
    const int I = 2 * i + (d & 31) - 8, J = 2 * j + ((d >> 5) & 31) - 8, K = 2 * k + (d >> 10) - 8;
    if (I < 0 || J < 0 || K < 0 || I + J + K > nf) continue;
    if (!(fl[point_class(nf, I, J, K)] & CF_OWNER)) continue;
    v += res_w<T>(e) * rf[tw32(wf, I, J, K)];
  }
  return v;
}

template <typename T>
__global__ void __launch_bounds__(kXBlock) prolong_p2_kernel(XDesc<T> D) {
  const int lane = threadIdx.x & 31;
  const int wg = blockIdx.x * kXWarps + (threadIdx.x >> 5);
  const int nf = D.nf, wf = nf + 1, wc = D.nc + 1;
  if ((int)blockIdx.x < D.nb_items) {
    if (wg >= D.n_items) return;
    const int4 it = D.items[wg];
    const int dim = it.z & 15, ncopies = (it.z >> 4) & 255, dirichlet = (it.z >> 12) & 1;
    const int p = it.y + lane;
    if (dirichlet || p >= prim_points(dim, nf)) return;
    int wts[3];
    prim_point_weights(dim, nf, p, wts);
    const IfaceCopy* cp = D.copies + it.x;
    int I, J, K;
    copy_local_ijk(cp[0], dim, wts, I, J, K);
    const T v = p2_interp<T>(D.src + (int64_t)cp[0].cell * D.cstride, wc, I, J, K);
    for (int q = 0; q < ncopies; ++q) {
      copy_local_ijk(cp[q], dim, wts, I, J, K);
      D.dst[(int64_t)cp[q].cell * D.fstride + tw32(wf, I, J, K)] += v;
    }
    return;
  }
  const int r = wg - D.nb_items * kXWarps;
  if (r >= D.n_rows) return;
  int cell, j, k;
  row_item(wf, r, cell, j, k);
  if (j == 0 || k == 0) return;
  const T* ec = D.src + (int64_t)cell * D.cstride;
  T* xf = D.dst + (int64_t)cell * D.fstride + row_start(wf, j, k);
  for (int i = 1 + lane; i + j + k < nf; i += 32) xf[i] += p2_interp<T>(ec, wc, i, j, k);
}

template <typename T>
__global__ void __launch_bounds__(kXBlock) restrict_p2_kernel(XDesc<T> D) {
  const int lane = threadIdx.x & 31;
  const int wg = blockIdx.x * kXWarps + (threadIdx.x >> 5);
  const int nf = D.nf, nc = D.nc, wc = nc + 1;
  if ((int)blockIdx.x < D.nb_items) {
    if (wg >= D.n_items) return;
    const int4 it = D.items[wg];
    const int dim = it.z & 15, ncopies = (it.z >> 4) & 255, dirichlet = (it.z >> 12) & 1;
    const int p = it.y + lane;
    if (p >= prim_points(dim, nc)) return;
    int wts[3];
    prim_point_weights(dim, nc, p, wts);
    const IfaceCopy* cp = D.copies + it.x;
    T v = T(0);
    if (!dirichlet)
      for (int q = 0; q < ncopies; ++q) {
        int i, j, k;
        copy_local_ijk(cp[q], dim, wts, i, j, k);
        v += p2_restrict_partial<T>(D.src + (int64_t)cp[q].cell * D.fstride,
                                    D.fflags + cp[q].cell * 16, nf, i, j, k);
      }
    for (int q = 0; q < ncopies; ++q) {
      int i, j, k;
      copy_local_ijk(cp[q], dim, wts, i, j, k);
      D.dst[(int64_t)cp[q].cell * D.cstride + tw32(wc, i, j, k)] = v;
    }
    return;
  }
  const int r = wg - D.nb_items * kXWarps;
  if (r >= D.n_rows) return;
  int cell, j, k;
  row_item(wc, r, cell, j, k);
  if (j == 0 || k == 0) return;
  const T* rf = D.src + (int64_t)cell * D.fstride;
  const uint8_t* fl = D.fflags + cell * 16;
  T* rc = D.dst + (int64_t)cell * D.cstride + row_start(wc, j, k);
  for (int i = 1 + lane; i + j + k < nc; i += 32) rc[i] = p2_restrict_partial<T>(rf, fl, nf, i, j, k);
}

int blocks_of(int64_t warps) { return (int)((warps + kXWarps - 1) / kXWarps); }

template <typename T>
int run_prolong(const LevelDev& F, const LevelDev& C, const void* ec, void* xf, cudaStream_t s) {
  XDesc<T> D;
  D.nf = F.n;
  D.nc = C.n;
  D.fstride = F.cell_stride;
  D.cstride = C.cell_stride;
  D.fflags = F.cls_flags;
  D.items = F.items;
  D.n_items = F.n_items;
  D.nb_items = blocks_of(F.n_items);
  D.copies = F.copies;
  D.n_rows = F.ncells * ntri32(F.w);
  D.src = (const T*)ec;
  D.dst = (T*)xf;
  prolong_p2_kernel<T><<<D.nb_items + blocks_of(D.n_rows), kXBlock, 0, s>>>(D);
  HG_CUDA(cudaGetLastError());
  return HG_OK;
}

template <typename T>
int run_restrict(const LevelDev& F, const LevelDev& C, const void* rf, void* rc, cudaStream_t s) {
  XDesc<T> D;
  D.nf = F.n;
  D.nc = C.n;
  D.fstride = F.cell_stride;
  D.cstride = C.cell_stride;
  D.fflags = F.cls_flags;
  D.items = C.items;
  D.n_items = C.n_items;
  D.nb_items = blocks_of(C.n_items);
  D.copies = C.copies;
  D.n_rows = C.ncells * ntri32(C.w);
  D.src = (const T*)rf;
  D.dst = (T*)rc;
  restrict_p2_kernel<T><<<D.nb_items + blocks_of(D.n_rows), kXBlock, 0, s>>>(D);
  HG_CUDA(cudaGetLastError());
  return HG_OK;
}

}  // namespace

int launch_prolong_p2(const LevelDev& F, const LevelDev& C, int dtype, const void* ec, void* xf,
                      cudaStream_t s) {
  if (int r = ensure_tables()) return r;
  if (F.n != 2 * C.n) {
    set_error("P2 prolongation: lattices are not consecutive levels");
    return HG_ERR_INVALID_ARG;
  }
  return dtype == HG_F64 ? run_prolong<double>(F, C, ec, xf, s) : run_prolong<float>(F, C, ec, xf, s);
}

int launch_restrict_p2(const LevelDev& F, const LevelDev& C, int dtype, const void* rf, void* rc,
                       cudaStream_t s) {
  if (int r = ensure_tables()) return r;
  if (F.n != 2 * C.n) {
    set_error("P2 restriction: lattices are not consecutive levels");
    return HG_ERR_INVALID_ARG;
  }
  return dtype == HG_F64 ? run_restrict<double>(F, C, rf, rc, s) : run_restrict<float>(F, C, rf, rc, s);
}

}  // namespace hg
