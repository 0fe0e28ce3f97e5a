// Lowest-order Nedelec (N1) grid transfers and the discrete gradient
// (multigrid by design, Sec. 5.1; N1 elements and Hiptmair's hybrid smoother,
// Sec. 6).
//
// Fine N1 level l lives at the odd points of lattice F (level l+1), coarse
// level l-1 at the odd points of lattice C (level l).  The prolongation reads
// the class table of hg_n1table.cpp (per fine class the coarse DoFs and
// exact dyadic weights) and the cell's orientation signs (one per lattice
// direction); restriction is the exact transpose with the same per-class
// terms regrouped per coarse parity class.  Interface points follow the P2
// transfers: prolongation values are computed once from the first copy's
// cell (the global DoF is the same in every copy) and added to every copy;
// restriction partials count each fine point in its owner cell only and are
// summed over the copies in ascending cell order.
//
// The discrete gradient maps a P1 function of level l (lattice C = level l)
// to N1 level l (lattice F = level l+1): (G phi)(q) = s_d (phi(b) - phi(a))
// for the edge q = (a + b) in F units of direction d = b - a, zero at vertex
// points and at boundary edges.  Its transpose collects, at every vertex v,
// the 14 edges 2v +- d: weight -s_d for 2v + d (v is the lower end), +s_d for
// 2v - d, owned fine points only, summed over the vertex's copies.
#include <cuda_runtime.h>

#include <mutex>
#include <string>

#include "hg_host.h"

namespace hg {

namespace {

constexpr int kNBlock = 256;
constexpr int kNWarps = kNBlock / 32;

// The 7 lattice edge directions (index = parity class of the midpoints - 1).
__device__ constexpr int kN1DirDev[7][3] = {{1, 0, 0},  {0, 1, 0},  {-1, 1, 0}, {0, 0, 1},
                                            {-1, 0, 1}, {0, -1, 1}, {1, -1, 1}};

__constant__ int c_n1_n[64];
__constant__ int c_n1_off[64][6];
__constant__ int c_n1_dir[64][6];
__constant__ double c_n1_w64[64][6];
__constant__ float c_n1_w32[64][6];
__constant__ int c_n1_fdir[64];
__constant__ int c_n1_rstart[9];
__constant__ int c_n1_rd[kN1MaxRes];
__constant__ int c_n1_rfdir[kN1MaxRes];
__constant__ double c_n1_rw64[kN1MaxRes];
__constant__ float c_n1_rw32[kN1MaxRes];

template <typename T>
__device__ __forceinline__ T n1_w(int c, int t);
template <>
__device__ __forceinline__ double n1_w<double>(int c, int t) { return c_n1_w64[c][t]; }
template <>
__device__ __forceinline__ float n1_w<float>(int c, int t) { return c_n1_w32[c][t]; }
template <typename T>
__device__ __forceinline__ T n1_rw(int e);
template <>
__device__ __forceinline__ double n1_rw<double>(int e) { return c_n1_rw64[e]; }
template <>
__device__ __forceinline__ float n1_rw<float>(int e) { return c_n1_rw32[e]; }

std::once_flag g_once;
int g_status = HG_OK;

int upload_tables() {
  const N1ProlongTable* T = nullptr;
  if (int r = n1_prolong_table(&T)) return r;
  float w32[64][6], rw32[kN1MaxRes] = {};
  for (int c = 0; c < 64; ++c)
    for (int q = 0; q < 6; ++q) w32[c][q] = (float)T->w[c][q];
  for (int e = 0; e < kN1MaxRes; ++e) rw32[e] = (float)T->res_w[e];
  HG_CUDA(cudaMemcpyToSymbol(c_n1_n, T->n, sizeof T->n));
  HG_CUDA(cudaMemcpyToSymbol(c_n1_off, T->off, sizeof T->off));
  HG_CUDA(cudaMemcpyToSymbol(c_n1_dir, T->dir, sizeof T->dir));
  HG_CUDA(cudaMemcpyToSymbol(c_n1_w64, T->w, sizeof T->w));
  HG_CUDA(cudaMemcpyToSymbol(c_n1_w32, w32, sizeof w32));
  HG_CUDA(cudaMemcpyToSymbol(c_n1_fdir, T->fine_dir, sizeof T->fine_dir));
  HG_CUDA(cudaMemcpyToSymbol(c_n1_rstart, T->res_start, sizeof T->res_start));
  HG_CUDA(cudaMemcpyToSymbol(c_n1_rd, T->res_d, sizeof T->res_d));
  HG_CUDA(cudaMemcpyToSymbol(c_n1_rfdir, T->res_fdir, sizeof T->res_fdir));
  HG_CUDA(cudaMemcpyToSymbol(c_n1_rw64, T->res_w, sizeof T->res_w));
  HG_CUDA(cudaMemcpyToSymbol(c_n1_rw32, rw32, sizeof rw32));
  return HG_OK;
}

int ensure_n1_tables() {
  static std::string msg;
  std::call_once(g_once, [] {
    g_status = upload_tables();
    if (g_status) msg = hg_last_error();
  });
  if (g_status) set_error("N1 transfer tables could not be set up: %s", msg.c_str());
  return g_status;
}

template <typename T>
struct NDesc {
  int nf, nc;                 // intervals of the F and C lattices
  int64_t fstride, cstride;
  const uint8_t* fflags;      // per (cell, class) flags of F
  const uint8_t* cflags;      // per (cell, class) flags of C
  const int4* items;          // interface items (32 points) of the lattice swept
  int n_items, nb_items;
  const IfaceCopy* copies;
  int n_rows;                 // rows of the lattice swept (all cells)
  const int8_t* sign;         // [ncells][8] orientation sign per lattice direction
  const T* src;
  T* dst;
  T scale;                    // N1_GRAD_ADD: u += scale * G phi
};

// Coarse N1 function's DoF at fine point (I,J,K) of one cell (0 at vertex points).
template <typename T>
__device__ __forceinline__ T n1_interp(const T* __restrict__ ec, const int8_t* s, int wc, int I,
                                       int J, int K) {
  const int cl = (I & 3) | ((J & 3) << 2) | ((K & 3) << 4);
  const int fd = c_n1_fdir[cl];
  if (fd < 0) return T(0);
  const int px = 2 * (I >> 2), py = 2 * (J >> 2), pz = 2 * (K >> 2);
  T v = T(0);
  for (int q = 0; q < c_n1_n[cl]; ++q) {
    const int o = c_n1_off[cl][q];
    v += n1_w<T>(cl, q) * T(s[c_n1_dir[cl][q]]) *
         ec[tw32(wc, px + (o & 3), py + ((o >> 2) & 3), pz + ((o >> 4) & 3))];
  }
  return T(s[fd]) * v;
}

// Partial of coarse DoF (i,j,k) of one cell: owned fine points of the cell.
template <typename T>
__device__ __forceinline__ T n1_restrict_partial(const T* __restrict__ rf, const uint8_t* fl,
                                                 const int8_t* s, int nf, int i, int j, int k) {
  const int par = (i & 1) | ((j & 1) << 1) | ((k & 1) << 2);
  if (par == 0) return T(0);
  const int wf = nf + 1;
  T v = T(0);
  for (int e = c_n1_rstart[par]; e < c_n1_rstart[par + 1]; ++e) {
    const int d = c_n1_rd[e];
    const int I = 2 * i + (d & 31) - 8, J = 2 * j + ((d >> 5) & 31) - 8, K = 2 * k + (d >> 10) - 8;
    if (I < 0 || J < 0 || K < 0 || I + J + K > nf) continue;
    if (!(fl[point_class(nf, I, J, K)] & CF_OWNER)) continue;
    v += n1_rw<T>(e) * T(s[c_n1_rfdir[e]]) * rf[tw32(wf, I, J, K)];
  }
  return T(s[par - 1]) * v;
}

template <typename T>
__global__ void __launch_bounds__(kNBlock) n1_prolong_kernel(NDesc<T> D) {
  const int lane = threadIdx.x & 31;
  const int wg = blockIdx.x * kNWarps + (threadIdx.x >> 5);
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
    const T v = n1_interp<T>(D.src + (int64_t)cp[0].cell * D.cstride, D.sign + 8 * cp[0].cell, wc,
                             I, J, K);
    for (int q = 0; q < ncopies; ++q) {
      copy_local_ijk(cp[q], dim, wts, I, J, K);
      D.dst[(int64_t)cp[q].cell * D.fstride + tw32(wf, I, J, K)] += v;
    }
    return;
  }
  const int r = wg - D.nb_items * kNWarps;
  if (r >= D.n_rows) return;
  int cell, j, k;
  row_item(wf, r, cell, j, k);
  if (j == 0 || k == 0) return;
  const T* ec = D.src + (int64_t)cell * D.cstride;
  const int8_t* s = D.sign + 8 * cell;
  T* xf = D.dst + (int64_t)cell * D.fstride + row_start(wf, j, k);
  for (int i = 1 + lane; i + j + k < nf; i += 32) xf[i] += n1_interp<T>(ec, s, wc, i, j, k);
}

template <typename T>
__global__ void __launch_bounds__(kNBlock) n1_restrict_kernel(NDesc<T> D) {
  const int lane = threadIdx.x & 31;
  const int wg = blockIdx.x * kNWarps + (threadIdx.x >> 5);
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
        v += n1_restrict_partial<T>(D.src + (int64_t)cp[q].cell * D.fstride,
                                    D.fflags + cp[q].cell * 16, D.sign + 8 * cp[q].cell, nf, i,
                                    j, k);
      }
    for (int q = 0; q < ncopies; ++q) {
      int i, j, k;
      copy_local_ijk(cp[q], dim, wts, i, j, k);
      D.dst[(int64_t)cp[q].cell * D.cstride + tw32(wc, i, j, k)] = v;
    }
    return;
  }
  const int r = wg - D.nb_items * kNWarps;
  if (r >= D.n_rows) return;
  int cell, j, k;
  row_item(wc, r, cell, j, k);
  if (j == 0 || k == 0) return;
  const T* rf = D.src + (int64_t)cell * D.fstride;
  const uint8_t* fl = D.fflags + cell * 16;
  const int8_t* s = D.sign + 8 * cell;
  T* rc = D.dst + (int64_t)cell * D.cstride + row_start(wc, j, k);
  for (int i = 1 + lane; i + j + k < nc; i += 32)
    rc[i] = n1_restrict_partial<T>(rf, fl, s, nf, i, j, k);
}

// (G phi) at every point of every cell of F (one warp per row, lanes over i);
// ADD: u += G phi (vertex points and boundary edges unchanged).
template <typename T, bool ADD>
__global__ void __launch_bounds__(kNBlock) n1_grad_kernel(NDesc<T> D) {
  const int lane = threadIdx.x & 31;
  const int r = blockIdx.x * kNWarps + (threadIdx.x >> 5);
  const int nf = D.nf, wf = nf + 1, wc = D.nc + 1;
  if (r >= D.n_rows) return;
  int cell, j, k;
  row_item(wf, r, cell, j, k);
  const T* phi = D.src + (int64_t)cell * D.cstride;
  const int8_t* s = D.sign + 8 * cell;
  const uint8_t* fl = D.fflags + cell * 16;
  T* u = D.dst + (int64_t)cell * D.fstride + row_start(wf, j, k);
  for (int i = lane; i + j + k <= nf; i += 32) {
    const int par = (i & 1) | ((j & 1) << 1) | ((k & 1) << 2);
    T v = T(0);
    if (par != 0 && !(fl[point_class(nf, i, j, k)] & CF_DIRICHLET)) {
      const int* d = kN1DirDev[par - 1];
      const T a = phi[tw32(wc, (i - d[0]) >> 1, (j - d[1]) >> 1, (k - d[2]) >> 1)];
      const T b = phi[tw32(wc, (i + d[0]) >> 1, (j + d[1]) >> 1, (k + d[2]) >> 1)];
      v = T(s[par - 1]) * (b - a);
    }
    u[i] = ADD ? u[i] + D.scale * v : v;
  }
}

// Partial of (G^T r) at coarse vertex (i,j,k) of one cell: owned fine edges.
template <typename T>
__device__ __forceinline__ T n1_gradt_partial(const T* __restrict__ rf, const uint8_t* fl,
                                              const int8_t* s, int nf, int i, int j, int k) {
  const int wf = nf + 1;
  T v = T(0);
#pragma unroll
  for (int q = 0; q < 7; ++q) {
    const int* d = kN1DirDev[q];
#pragma unroll
    for (int h = 0; h < 2; ++h) {
      const int sg = h == 0 ? 1 : -1;   // 2v + d: v is the lower end (weight -s); 2v - d: +s
      const int I = 2 * i + sg * d[0], J = 2 * j + sg * d[1], K = 2 * k + sg * d[2];
      if (I < 0 || J < 0 || K < 0 || I + J + K > nf) continue;
      if (!(fl[point_class(nf, I, J, K)] & CF_OWNER)) continue;
      v += T(-sg * s[q]) * rf[tw32(wf, I, J, K)];
    }
  }
  return v;
}

template <typename T>
__global__ void __launch_bounds__(kNBlock) n1_gradt_kernel(NDesc<T> D) {
  const int lane = threadIdx.x & 31;
  const int wg = blockIdx.x * kNWarps + (threadIdx.x >> 5);
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
        v += n1_gradt_partial<T>(D.src + (int64_t)cp[q].cell * D.fstride,
                                 D.fflags + cp[q].cell * 16, D.sign + 8 * cp[q].cell, nf, i, j, k);
      }
    for (int q = 0; q < ncopies; ++q) {
      int i, j, k;
      copy_local_ijk(cp[q], dim, wts, i, j, k);
      D.dst[(int64_t)cp[q].cell * D.cstride + tw32(wc, i, j, k)] = v;
    }
    return;
  }
  const int r = wg - D.nb_items * kNWarps;
  if (r >= D.n_rows) return;
  int cell, j, k;
  row_item(wc, r, cell, j, k);
  if (j == 0 || k == 0) return;
  const T* rf = D.src + (int64_t)cell * D.fstride;
  const uint8_t* fl = D.fflags + cell * 16;
  const int8_t* s = D.sign + 8 * cell;
  T* rc = D.dst + (int64_t)cell * D.cstride + row_start(wc, j, k);
  for (int i = 1 + lane; i + j + k < nc; i += 32) rc[i] = n1_gradt_partial<T>(rf, fl, s, nf, i, j, k);
}

int blocks_of(int64_t warps) { return (int)((warps + kNWarps - 1) / kNWarps); }

template <typename T>
NDesc<T> ndesc(const LevelDev& F, const LevelDev& C, const LevelDev& swept, const int8_t* sign,
               const void* src, void* dst) {
  NDesc<T> D;
  D.nf = F.n;
  D.nc = C.n;
  D.fstride = F.cell_stride;
  D.cstride = C.cell_stride;
  D.fflags = F.cls_flags;
  D.cflags = C.cls_flags;
  D.items = swept.items;
  D.n_items = swept.n_items;
  D.nb_items = blocks_of(swept.n_items);
  D.copies = swept.copies;
  D.n_rows = swept.ncells * ntri32(swept.w);
  D.sign = sign;
  D.src = (const T*)src;
  D.dst = (T*)dst;
  D.scale = T(1);
  return D;
}

template <typename T>
int run(int which, const LevelDev& F, const LevelDev& C, const int8_t* sign, const void* src,
        void* dst, cudaStream_t s, double scale) {
  switch (which) {
    case 0: {  // prolongation: sweep F
      const NDesc<T> D = ndesc<T>(F, C, F, sign, src, dst);
      n1_prolong_kernel<T><<<D.nb_items + blocks_of(D.n_rows), kNBlock, 0, s>>>(D);
      break;
    }
    case 1: {  // restriction: sweep C
      const NDesc<T> D = ndesc<T>(F, C, C, sign, src, dst);
      n1_restrict_kernel<T><<<D.nb_items + blocks_of(D.n_rows), kNBlock, 0, s>>>(D);
      break;
    }
    case 2:
    case 4: {  // gradient (4: added): every row of F, no items
      NDesc<T> D = ndesc<T>(F, C, F, sign, src, dst);
      D.nb_items = 0;
      D.scale = (T)scale;
      if (which == 2)
        n1_grad_kernel<T, false><<<blocks_of(D.n_rows), kNBlock, 0, s>>>(D);
      else
        n1_grad_kernel<T, true><<<blocks_of(D.n_rows), kNBlock, 0, s>>>(D);
      break;
    }
    default: {  // gradient transpose: sweep C
      const NDesc<T> D = ndesc<T>(F, C, C, sign, src, dst);
      n1_gradt_kernel<T><<<D.nb_items + blocks_of(D.n_rows), kNBlock, 0, s>>>(D);
      break;
    }
  }
  HG_CUDA(cudaGetLastError());
  return HG_OK;
}

}  // namespace

int launch_n1_transfer(int which, const LevelDev& F, const LevelDev& C, int dtype,
                       const int8_t* sign, const void* src, void* dst, cudaStream_t s,
                       double scale) {
  if (int r = ensure_n1_tables()) return r;
  if (F.n != 2 * C.n) {
    set_error("N1 transfer: lattices are not consecutive levels");
    return HG_ERR_INVALID_ARG;
  }
  return dtype == HG_F64 ? run<double>(which, F, C, sign, src, dst, s, scale)
                         : run<float>(which, F, C, sign, src, dst, s, scale);
}

}  // namespace hg
