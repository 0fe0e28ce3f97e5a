// P1 kernels on the per-macro-cell vertex lattice.
//
// Storage: every macro cell holds its closed vertex lattice i+j+k <= n in
// t_{n+1} order (Sec. 4), so points on macro faces/edges/vertices have one
// copy per containing cell.  An operator application is two kernels:
//  * the cell kernel evaluates, for every point of every cell, the sum of the
//    cell's own micro-element contributions with the cell's precomputed
//    15-point stencil of the point's boundary class (Sec. 5.2, stencil-based
//    pattern with per-macro-primitive constant stencils); interior points
//    are complete, interface points hold a per-cell partial sum;
//  * the interface kernel (the ghost-layer exchange between macro
//    primitives, Sec. 2) adds the partial sums of all copies of every
//    macro face/edge/vertex point in ascending cell order and writes the
//    result to every copy, so all copies stay bit-identical.
#include <cuda_runtime.h>

#include "hg_internal.h"

namespace hg {

namespace {

constexpr int kBlock = 256;

template <typename T>
struct LevelArgs {
  int n, w;
  int64_t stride;
  const uint8_t* flags;
};

// Sum of one cell's stencil of class `cls` at (i,j,k), neighbours read through
// the t_w index (slow path for cell-boundary points).
template <typename T>
__device__ T boundary_stencil(const T* __restrict__ x, const T* __restrict__ S, int n, int w,
                              int i, int j, int k) {
  T acc = T(0);
#pragma unroll
  for (int d = 0; d < kNDir; ++d) {
    T s = S[d];
    if (s != T(0)) {
      int di, dj, dk;
      dir_offset(d, di, dj, dk);
      int a = i + di, b = j + dj, c = k + dk;
      if (a >= 0 && b >= 0 && c >= 0 && a + b + c <= n) acc += s * x[tw32(w, a, b, c)];
    }
  }
  return acc;
}

// Cell kernel: one block per (macro cell, plane k); warps over rows j, lanes
// over i (the x-lines of Sec. 4).
template <typename T, int OP>
__global__ void __launch_bounds__(kBlock) p1_cell_kernel(LevelArgs<T> L, const T* __restrict__ X,
                                                         const T* __restrict__ B, T* __restrict__ Y,
                                                         const T* __restrict__ sten, T omega,
                                                         int mode, int mask) {
  const int cell = blockIdx.x / L.w;
  const int k = blockIdx.x % L.w;
  const int n = L.n, w = L.w;
  const int64_t base = (int64_t)cell * L.stride;
  const T* x = X + base;
  const T* b = B ? B + base : nullptr;
  T* y = Y + base;
  const T* S = sten + (int64_t)cell * 256;
  const uint8_t* fl = L.flags + cell * 16;
  T s[kNDir];
#pragma unroll
  for (int d = 0; d < kNDir; ++d) s[d] = S[d];
  const int m = n - k;
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nw = blockDim.x >> 5;
  for (int j = warp; j <= m; j += nw) {
    const int r0 = row_start(w, j, k);
    const bool inner_row = j >= 1 && k >= 1 && j + k <= n - 1;
    int rjp = 0, rjm = 0, rkp = 0, rkm = 0, rjmkp = 0, rjpkm = 0;
    if (inner_row) {
      rjp = row_start(w, j + 1, k);
      rjm = row_start(w, j - 1, k);
      rkp = row_start(w, j, k + 1);
      rkm = row_start(w, j, k - 1);
      rjmkp = row_start(w, j - 1, k + 1);
      rjpkm = row_start(w, j + 1, k - 1);
    }
    for (int i = lane; i <= m - j; i += 32) {
      const int cls = point_class(n, i, j, k);
      const int idx = r0 + i;
      T acc;
      if (cls == 0) {
        acc = s[0] * x[idx] + s[1] * x[idx + 1] + s[2] * x[idx - 1] + s[3] * x[rjp + i] +
              s[4] * x[rjm + i] + s[5] * x[rkp + i] + s[6] * x[rkm + i] + s[7] * x[rjp + i - 1] +
              s[8] * x[rjm + i + 1] + s[9] * x[rkp + i - 1] + s[10] * x[rkm + i + 1] +
              s[11] * x[rjmkp + i] + s[12] * x[rjpkm + i] + s[13] * x[rjmkp + i + 1] +
              s[14] * x[rjpkm + i - 1];
        if (OP == OP_APPLY) {
          y[idx] = mode == HG_ADD ? y[idx] + acc : acc;
        } else if (OP == OP_RESID) {
          y[idx] = b[idx] - acc;
        } else {
          y[idx] = x[idx] + omega * (b[idx] - acc) / s[0];
        }
      } else {
        const uint8_t f = fl[cls];
        const bool dir = (f & CF_DIRICHLET) != 0;
        if (dir && (OP != OP_APPLY || mask == HG_MASK_INNER)) {
          if (OP == OP_RESID) y[idx] = T(0);
          if (OP == OP_JACOBI) y[idx] = x[idx];
          continue;
        }
        acc = boundary_stencil<T>(x, S + cls * 16, n, w, i, j, k);
        if (OP == OP_APPLY && mode == HG_ADD && (f & CF_OWNER)) acc = y[idx] + acc;
        y[idx] = acc;  // partial sum, completed by the interface kernel
      }
    }
  }
}

// Interface kernel: one block per macro primitive.
template <typename T, int OP>
__global__ void __launch_bounds__(kBlock) p1_iface_kernel(LevelArgs<T> L, const IfacePrim* prims,
                                                          const IfaceCopy* copies,
                                                          const T* __restrict__ X,
                                                          const T* __restrict__ B, T* Y,
                                                          const T* __restrict__ sten, T omega) {
  const IfacePrim P = prims[blockIdx.x];
  const int n = L.n, w = L.w;
  const int npts = prim_points(P.dim, n);
  const IfaceCopy* cp = copies + P.first_copy;
  for (int p = threadIdx.x; p < npts; p += blockDim.x) {
    int wts[3];
    if (P.dim == 2) {
      // row b has n-1-b points; find the row of p
      int b = 1, rem = p;
      while (rem >= n - 1 - b) {
        rem -= n - 1 - b;
        ++b;
      }
      wts[0] = n - (rem + 1) - b;
      wts[1] = rem + 1;
      wts[2] = b;
    } else {
      prim_point_weights(P.dim, n, p, wts);
    }
    T sum = T(0), diag = T(0);
    int64_t idx0 = 0;
    for (int q = 0; q < P.ncopies; ++q) {
      int i, j, k;
      copy_local_ijk(cp[q], P.dim, wts, i, j, k);
      const int64_t idx = (int64_t)cp[q].cell * L.stride + tw32(w, i, j, k);
      if (q == 0) idx0 = idx;
      sum += Y[idx];
      if (OP == OP_JACOBI)
        diag += sten[(int64_t)cp[q].cell * 256 + point_class(n, i, j, k) * 16];
    }
    T v;
    if (OP == OP_APPLY) {
      v = sum;
    } else if (OP == OP_RESID) {
      v = B[idx0] - sum;
    } else {
      v = X[idx0] + omega * (B[idx0] - sum) / diag;
    }
    for (int q = 0; q < P.ncopies; ++q) {
      int i, j, k;
      copy_local_ijk(cp[q], P.dim, wts, i, j, k);
      Y[(int64_t)cp[q].cell * L.stride + tw32(w, i, j, k)] = v;
    }
  }
}

template <typename T>
LevelArgs<T> level_args(const LevelDev& L) {
  LevelArgs<T> a;
  a.n = L.n;
  a.w = L.w;
  a.stride = L.cell_stride;
  a.flags = L.cls_flags;
  return a;
}

template <typename T, int OP>
int run_p1(const LevelDev& L, const StencilArgs& a, cudaStream_t s) {
  LevelArgs<T> la = level_args<T>(L);
  const int grid = L.ncells * L.w;
  p1_cell_kernel<T, OP><<<grid, kBlock, 0, s>>>(la, (const T*)a.x, (const T*)a.b, (T*)a.out,
                                                (const T*)a.sten, (T)a.omega, a.mode, a.mask);
  HG_CUDA(cudaGetLastError());
  const int np = (OP == OP_APPLY && a.mask == HG_MASK_ALL) ? L.n_prims : L.n_prims_inner;
  if (np > 0) {
    p1_iface_kernel<T, OP><<<np, kBlock, 0, s>>>(la, L.prims, L.copies, (const T*)a.x,
                                                 (const T*)a.b, (T*)a.out, (const T*)a.sten,
                                                 (T)a.omega);
    HG_CUDA(cudaGetLastError());
  }
  return HG_OK;
}

template <typename T>
int run_p1_op(const LevelDev& L, const StencilArgs& a, cudaStream_t s) {
  switch (a.op) {
    case OP_APPLY: return run_p1<T, OP_APPLY>(L, a, s);
    case OP_RESID: return run_p1<T, OP_RESID>(L, a, s);
    case OP_JACOBI: return run_p1<T, OP_JACOBI>(L, a, s);
  }
  set_error("unknown cell operation %d", a.op);
  return HG_ERR_INVALID_ARG;
}

// ------------------------------------------------------------ maps / dumps
__global__ void index_enumerate_kernel(int w, int64_t* out) {
  const int k = blockIdx.x;
  const int m = w - 1 - k;
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nw = blockDim.x >> 5;
  for (int j = warp; j <= m; j += nw) {
    const int r0 = row_start(w, j, k);
    for (int i = lane; i <= m - j; i += 32)
      out[r0 + i] = (int64_t)i + ((int64_t)j << 20) + ((int64_t)k << 40);
  }
}

__global__ void interface_dump_kernel(int n, int w, int64_t stride, const IfacePrim* prims,
                                      int nprims, const int32_t* pbase, const IfaceCopy* copies,
                                      int maxc, int64_t* out) {
  const int prim = blockIdx.x;
  if (prim >= nprims) return;
  const IfacePrim P = prims[prim];
  const int npts = prim_points(P.dim, n);
  for (int p = threadIdx.x; p < npts; p += blockDim.x) {
    int wts[3];
    prim_point_weights(P.dim, n, p, wts);
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
  (void)stride;
}

template <typename T>
__global__ void gather_kernel(const T* __restrict__ st, const int64_t* __restrict__ rep, int64_t nu,
                              T* __restrict__ can) {
  for (int64_t u = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; u < nu;
       u += (int64_t)gridDim.x * blockDim.x)
    can[u] = st[rep[u]];
}

template <typename T>
__global__ void scatter_kernel(const T* __restrict__ can, const int32_t* __restrict__ canon,
                               int64_t ns, T* __restrict__ st) {
  for (int64_t q = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; q < ns;
       q += (int64_t)gridDim.x * blockDim.x) {
    int32_t u = canon[q];
    if (u >= 0) st[q] = can[u];
  }
}

// ---------------------------------------------------------- grid transfers
// Restriction r_c = P^T r_f: coarse point I sums the fine points 2I (weight 1)
// and 2I +- d (weight 1/2) that lie in the cell and are owned by it; partial
// sums on coarse interface points are completed by the interface kernel.
template <typename T>
__global__ void __launch_bounds__(kBlock) restrict_kernel(int nf, int64_t fstride,
                                                          const uint8_t* flags, int nc,
                                                          int64_t cstride,
                                                          const T* __restrict__ RF,
                                                          T* __restrict__ RC) {
  const int wc = nc + 1, wf = nf + 1;
  const int cell = blockIdx.x / wc;
  const int K = blockIdx.x % wc;
  const T* rf = RF + (int64_t)cell * fstride;
  T* rc = RC + (int64_t)cell * cstride;
  const uint8_t* fl = flags + cell * 16;
  const int m = nc - K;
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nw = blockDim.x >> 5;
  for (int J = warp; J <= m; J += nw) {
    for (int I = lane; I <= m - J; I += 32) {
      const int ccls = point_class(nc, I, J, K);
      const int cidx = row_start(wc, J, K) + I;
      if (fl[ccls] & CF_DIRICHLET) {
        rc[cidx] = T(0);
        continue;
      }
      const int fi = 2 * I, fj = 2 * J, fk = 2 * K;
      T acc = T(0);
      for (int d = 0; d < kNDir; ++d) {
        int di, dj, dk;
        dir_offset(d, di, dj, dk);
        const int a = fi + di, b = fj + dj, c = fk + dk;
        if (a < 0 || b < 0 || c < 0 || a + b + c > nf) continue;
        const int fcls = point_class(nf, a, b, c);
        if (!(fl[fcls] & CF_OWNER)) continue;
        const T v = rf[tw32(wf, a, b, c)];
        acc += d == 0 ? v : T(0.5) * v;
      }
      rc[cidx] = acc;
    }
  }
}

// Prolongation x_f += P e_c: fine points with even coordinates copy the coarse
// value, the others are midpoints of the coarse edge selected by the parity.
template <typename T>
__global__ void __launch_bounds__(kBlock) prolong_kernel(int nf, int64_t fstride,
                                                         const uint8_t* flags, int64_t cstride,
                                                         const T* __restrict__ EC,
                                                         T* __restrict__ XF) {
  const int wf = nf + 1, nc = nf / 2, wc = nc + 1;
  const int cell = blockIdx.x / wf;
  const int k = blockIdx.x % wf;
  const T* ec = EC + (int64_t)cell * cstride;
  T* xf = XF + (int64_t)cell * fstride;
  const uint8_t* fl = flags + cell * 16;
  const int m = nf - k;
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nw = blockDim.x >> 5;
  for (int j = warp; j <= m; j += nw) {
    for (int i = lane; i <= m - j; i += 32) {
      if (fl[point_class(nf, i, j, k)] & CF_DIRICHLET) continue;
      const int par = (i & 1) | ((j & 1) << 1) | ((k & 1) << 2);
      T v;
      if (par == 0) {
        v = ec[tw32(wc, i >> 1, j >> 1, k >> 1)];
      } else {
        // direction d of the coarse edge whose midpoint has this parity
        int di = 0, dj = 0, dk = 0;
        switch (par) {
          case 1: di = 1; break;
          case 2: dj = 1; break;
          case 4: dk = 1; break;
          case 3: di = -1; dj = 1; break;
          case 5: di = -1; dk = 1; break;
          case 6: dj = -1; dk = 1; break;
          default: di = 1; dj = -1; dk = 1; break;
        }
        const T a = ec[tw32(wc, (i - di) >> 1, (j - dj) >> 1, (k - dk) >> 1)];
        const T b = ec[tw32(wc, (i + di) >> 1, (j + dj) >> 1, (k + dk) >> 1)];
        v = T(0.5) * (a + b);
      }
      xf[row_start(wf, j, k) + i] += v;
    }
  }
}

// ------------------------------------------------------------- reductions
// Deterministic FP64 dot: one partial per (cell, plane) block in a fixed
// shape, then a single block adds the partials in a fixed tree order.
template <typename T>
__global__ void __launch_bounds__(kBlock) dot_partial_kernel(int n, int64_t stride,
                                                             const uint8_t* flags,
                                                             const T* __restrict__ X,
                                                             const T* __restrict__ Y, int mask,
                                                             double* partial) {
  const int w = n + 1;
  const int cell = blockIdx.x / w;
  const int k = blockIdx.x % w;
  const T* x = X + (int64_t)cell * stride;
  const T* y = Y + (int64_t)cell * stride;
  const uint8_t* fl = flags + cell * 16;
  const int m = n - k;
  double acc = 0.0;
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nw = blockDim.x >> 5;
  for (int j = warp; j <= m; j += nw) {
    const int r0 = row_start(w, j, k);
    for (int i = lane; i <= m - j; i += 32) {
      const uint8_t f = fl[point_class(n, i, j, k)];
      if (!(f & CF_OWNER)) continue;
      if (mask == HG_MASK_INNER && (f & CF_DIRICHLET)) continue;
      acc += (double)x[r0 + i] * (double)y[r0 + i];
    }
  }
  __shared__ double red[kBlock / 32];
  for (int o = 16; o > 0; o >>= 1) acc += __shfl_down_sync(0xffffffffu, acc, o);
  if (lane == 0) red[warp] = acc;
  __syncthreads();
  if (threadIdx.x == 0) {
    double t = 0.0;
    for (int q = 0; q < nw; ++q) t += red[q];
    partial[blockIdx.x] = t;
  }
}

__global__ void __launch_bounds__(1024) sum_partials_kernel(const double* partial, int64_t np,
                                                            double* result) {
  __shared__ double red[1024];
  double acc = 0.0;
  for (int64_t q = threadIdx.x; q < np; q += blockDim.x) acc += partial[q];
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

}  // namespace

int launch_p1_const(const LevelDev& L, int dtype, const StencilArgs& a, cudaStream_t s) {
  return dtype == HG_F64 ? run_p1_op<double>(L, a, s) : run_p1_op<float>(L, a, s);
}

int launch_index_enumerate(int w, int64_t* out, cudaStream_t s) {
  index_enumerate_kernel<<<w, kBlock, 0, s>>>(w, out);
  HG_CUDA(cudaGetLastError());
  return HG_OK;
}

int launch_interface_dump(const LevelDev& L, int64_t* out, cudaStream_t s) {
  if (L.n_prims == 0) return HG_OK;
  interface_dump_kernel<<<L.n_prims, kBlock, 0, s>>>(L.n, L.w, L.cell_stride, L.prims, L.n_prims,
                                                     L.prim_point_base, L.copies, L.max_copies,
                                                     out);
  HG_CUDA(cudaGetLastError());
  return HG_OK;
}

int launch_to_canonical(const LevelDev& L, int dtype, const void* st, void* can, cudaStream_t s) {
  const int g = grid_for(L.n_unique);
  if (dtype == HG_F64)
    gather_kernel<double><<<g, kBlock, 0, s>>>((const double*)st, L.canon_rep, L.n_unique,
                                               (double*)can);
  else
    gather_kernel<float><<<g, kBlock, 0, s>>>((const float*)st, L.canon_rep, L.n_unique,
                                              (float*)can);
  HG_CUDA(cudaGetLastError());
  return HG_OK;
}

int launch_from_canonical(const LevelDev& L, int dtype, const void* can, void* st,
                          cudaStream_t s) {
  const int g = grid_for(L.n_stored);
  if (dtype == HG_F64)
    scatter_kernel<double><<<g, kBlock, 0, s>>>((const double*)can, L.canon, L.n_stored,
                                                (double*)st);
  else
    scatter_kernel<float><<<g, kBlock, 0, s>>>((const float*)can, L.canon, L.n_stored,
                                               (float*)st);
  HG_CUDA(cudaGetLastError());
  return HG_OK;
}

template <typename T>
static int run_restrict(const LevelDev& F, const LevelDev& C, const void* rf, void* rc,
                        cudaStream_t s) {
  restrict_kernel<T><<<C.ncells * C.w, kBlock, 0, s>>>(F.n, F.cell_stride, F.cls_flags, C.n,
                                                      C.cell_stride, (const T*)rf, (T*)rc);
  HG_CUDA(cudaGetLastError());
  if (C.n_prims_inner > 0) {
    LevelArgs<T> la = level_args<T>(C);
    p1_iface_kernel<T, OP_APPLY><<<C.n_prims_inner, kBlock, 0, s>>>(
        la, C.prims, C.copies, nullptr, nullptr, (T*)rc, nullptr, T(0));
    HG_CUDA(cudaGetLastError());
  }
  return HG_OK;
}

int launch_restrict_p1(const LevelDev& F, const LevelDev& C, int dtype, const void* rf, void* rc,
                       cudaStream_t s) {
  return dtype == HG_F64 ? run_restrict<double>(F, C, rf, rc, s)
                         : run_restrict<float>(F, C, rf, rc, s);
}

int launch_prolong_p1(const LevelDev& F, const LevelDev& C, int dtype, const void* ec, void* xf,
                      cudaStream_t s) {
  const int grid = F.ncells * F.w;
  if (dtype == HG_F64)
    prolong_kernel<double><<<grid, kBlock, 0, s>>>(F.n, F.cell_stride, F.cls_flags, C.cell_stride,
                                                   (const double*)ec, (double*)xf);
  else
    prolong_kernel<float><<<grid, kBlock, 0, s>>>(F.n, F.cell_stride, F.cls_flags, C.cell_stride,
                                                  (const float*)ec, (float*)xf);
  HG_CUDA(cudaGetLastError());
  return HG_OK;
}

int64_t dot_scratch_len(const LevelDev& L) { return (int64_t)L.ncells * L.w; }

int launch_dot(const LevelDev& L, int dtype, const void* x, const void* y, int mask,
               double* scratch, double* result_dev, cudaStream_t s) {
  const int grid = L.ncells * L.w;
  if (dtype == HG_F64)
    dot_partial_kernel<double><<<grid, kBlock, 0, s>>>(L.n, L.cell_stride, L.cls_flags,
                                                       (const double*)x, (const double*)y, mask,
                                                       scratch);
  else
    dot_partial_kernel<float><<<grid, kBlock, 0, s>>>(L.n, L.cell_stride, L.cls_flags,
                                                      (const float*)x, (const float*)y, mask,
                                                      scratch);
  HG_CUDA(cudaGetLastError());
  sum_partials_kernel<<<1, 1024, 0, s>>>(scratch, grid, result_dev);
  HG_CUDA(cudaGetLastError());
  return HG_OK;
}

}  // namespace hg
