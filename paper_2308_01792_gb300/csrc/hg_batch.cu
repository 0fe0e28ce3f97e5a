// Batched persistent stages over many independent problems: element-wise
// steps of the refinement loop, per-problem FP64 dots, and the dense coarse
// solves.  Each problem contributes a number of units (blocks); a grid-stride
// loop over the concatenated units locates its problem by binary search.
#include <cuda_runtime.h>

#include <algorithm>

#include "hg_internal.h"

namespace hg {

namespace {

constexpr int kB = 256;
constexpr int kEwPerUnit = kB * 4;   // elements per element-wise unit

__device__ __forceinline__ int find_problem(const int* __restrict__ base, int nprob, int u) {
  int lo = 0, hi = nprob - 1;
  while (lo < hi) {
    const int mid = (lo + hi + 1) >> 1;
    if (__ldg(base + mid) <= u) lo = mid; else hi = mid - 1;
  }
  return lo;
}

template <int OP>
__global__ void __launch_bounds__(kB) ew_batched_kernel(const EwDesc* __restrict__ d,
                                                        const int* __restrict__ base, int nprob) {
  const int total = __ldg(base + nprob);
  for (int u = blockIdx.x; u < total; u += gridDim.x) {
    const int p = find_problem(base, nprob, u);
    const EwDesc D = d[p];
    const int64_t e0 = (int64_t)(u - __ldg(base + p)) * kEwPerUnit;
    const int64_t e1 = D.n < e0 + kEwPerUnit ? D.n : e0 + kEwPerUnit;
    if (OP == EW_DEMOTE || OP == EW_PROMOTE) {
      const double rr = *D.rr;
      const double nr = rr > 0.0 ? sqrt(rr) : 0.0;
      if (OP == EW_DEMOTE) {
        const double sc = nr > 0.0 ? 1.0 / nr : 0.0;
        for (int64_t q = e0 + threadIdx.x; q < e1; q += kB)
          ((float*)D.a)[q] = (float)(((const double*)D.b)[q] * sc);
      } else {
        for (int64_t q = e0 + threadIdx.x; q < e1; q += kB)
          ((double*)D.a)[q] += nr * (double)((const float*)D.b)[q];
      }
    } else if (D.dtype == HG_F64) {
      for (int64_t q = e0 + threadIdx.x; q < e1; q += kB)
        ((double*)D.a)[q] = OP == EW_ZERO ? 0.0 : ((const double*)D.b)[q];
    } else {
      for (int64_t q = e0 + threadIdx.x; q < e1; q += kB)
        ((float*)D.a)[q] = OP == EW_ZERO ? 0.f : ((const float*)D.b)[q];
    }
  }
}

// Unit u of problem p covers lattice rows [b*kDotRowsPerUnit, +kDotRowsPerUnit)
// of that problem (b = u - base[p]), one warp per row in turn; each unit
// writes one partial and a second kernel adds each problem's partials in
// unit order, so the result does not depend on the grid.
template <typename T>
__global__ void __launch_bounds__(kB) dot_batched_kernel(const DotDesc* __restrict__ d,
                                                         const int* __restrict__ base, int nprob,
                                                         double* __restrict__ partial) {
  const int total = __ldg(base + nprob);
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  __shared__ double red[kB / 32];
  for (int u = blockIdx.x; u < total; u += gridDim.x) {
    const int p = find_problem(base, nprob, u);
    const DotDesc D = d[p];
    const int w = D.n + 1;
    const int r0 = (u - __ldg(base + p)) * kDotRowsPerUnit;
    const int r1 = D.n_rows < r0 + kDotRowsPerUnit ? D.n_rows : r0 + kDotRowsPerUnit;
    double acc = 0.0;
    for (int r = r0 + warp; r < r1; r += kB / 32) {
      int cell, j, k;
      row_item(w, r, cell, j, k);
      const int64_t rs = (int64_t)cell * D.stride + row_start(w, j, k);
      const uint8_t* fl = D.flags + cell * 16;
      for (int i = lane; i + j + k <= D.n; i += 32) {
        const uint8_t f = fl[point_class(D.n, i, j, k)];
        if (!(f & CF_OWNER) || (f & CF_DIRICHLET)) continue;
        acc += (double)((const T*)D.x)[rs + i] * (double)((const T*)D.y)[rs + i];
      }
    }
    for (int o = 16; o > 0; o >>= 1) acc += __shfl_down_sync(0xffffffffu, acc, o);
    if (lane == 0) red[warp] = acc;
    __syncthreads();
    if (threadIdx.x == 0) {
      double t = 0.0;
      for (int q = 0; q < kB / 32; ++q) t += red[q];
      partial[u] = t;
    }
    __syncthreads();
  }
}

__global__ void dot_batched_sum_kernel(const double* __restrict__ partial,
                                       const int* __restrict__ base, int nprob,
                                       double* __restrict__ rr) {
  const int p = blockIdx.x * blockDim.x + threadIdx.x;
  if (p >= nprob) return;
  double s = 0.0;
  for (int u = base[p]; u < base[p + 1]; ++u) s += partial[u];
  rr[p] = s;
}

// Coarse solve, phase 1: x_int = A^-1 b_int, one warp per row.
template <typename T>
__global__ void __launch_bounds__(kB) coarse_mv_batched_kernel(const CoarseBDesc* __restrict__ d,
                                                              const int* __restrict__ base,
                                                              int nprob) {
  const int total = __ldg(base + nprob);
  const int lane = threadIdx.x & 31;
  for (int u = blockIdx.x; u < total; u += gridDim.x) {
    const int p = find_problem(base, nprob, u);
    const CoarseBDesc D = d[p];
    const int row = (u - __ldg(base + p)) * (kB / 32) + (threadIdx.x >> 5);
    if (row >= D.nint) continue;
    double acc = 0.0;
    for (int c = lane; c < D.nint; c += 32)
      acc += D.ainv[(int64_t)row * D.nint + c] * (double)((const T*)D.b)[D.rep[c]];
    for (int o = 16; o > 0; o >>= 1) acc += __shfl_down_sync(0xffffffffu, acc, o);
    if (lane == 0) D.xint[row] = acc;
  }
}

// Coarse solve, phase 2: every stored copy of an interior unknown.
template <typename T>
__global__ void __launch_bounds__(kB) coarse_sc_batched_kernel(const CoarseBDesc* __restrict__ d,
                                                              const int* __restrict__ base,
                                                              int nprob) {
  const int total = __ldg(base + nprob);
  for (int u = blockIdx.x; u < total; u += gridDim.x) {
    const int p = find_problem(base, nprob, u);
    const CoarseBDesc D = d[p];
    const int64_t e0 = (int64_t)(u - __ldg(base + p)) * kEwPerUnit;
    const int64_t e1 = D.n_stored < e0 + kEwPerUnit ? D.n_stored : e0 + kEwPerUnit;
    for (int64_t q = e0 + threadIdx.x; q < e1; q += kB) {
      const int32_t c = D.canon[q];
      if (c < 0) continue;
      const int32_t iu = D.ioc[c];
      if (iu >= 0) ((T*)D.x)[q] = (T)D.xint[iu];
    }
  }
}

}  // namespace

int64_t ew_units(int64_t n) { return (n + kEwPerUnit - 1) / kEwPerUnit; }
int64_t coarse_units_mv(int nint) { return (nint + kB / 32 - 1) / (kB / 32); }
int64_t coarse_units_sc(int64_t n_stored) { return ew_units(n_stored); }

int launch_batched_ew(int op, const EwDesc* d, const int* base, int nprob, int grid,
                      cudaStream_t s) {
  if (nprob <= 0) return HG_OK;
  switch (op) {
    case EW_ZERO: ew_batched_kernel<EW_ZERO><<<grid, kB, 0, s>>>(d, base, nprob); break;
    case EW_COPY: ew_batched_kernel<EW_COPY><<<grid, kB, 0, s>>>(d, base, nprob); break;
    case EW_DEMOTE: ew_batched_kernel<EW_DEMOTE><<<grid, kB, 0, s>>>(d, base, nprob); break;
    default: ew_batched_kernel<EW_PROMOTE><<<grid, kB, 0, s>>>(d, base, nprob); break;
  }
  HG_CUDA(cudaGetLastError());
  return HG_OK;
}

int64_t dot_units(int n_rows) { return (n_rows + kDotRowsPerUnit - 1) / kDotRowsPerUnit; }

int launch_batched_dot(int dtype, const DotDesc* d, const int* base, int nprob, int grid,
                       double* partial, double* rr, cudaStream_t s) {
  if (nprob <= 0) return HG_OK;
  if (dtype == HG_F64)
    dot_batched_kernel<double><<<grid, kB, 0, s>>>(d, base, nprob, partial);
  else
    dot_batched_kernel<float><<<grid, kB, 0, s>>>(d, base, nprob, partial);
  HG_CUDA(cudaGetLastError());
  dot_batched_sum_kernel<<<(nprob + 255) / 256, 256, 0, s>>>(partial, base, nprob, rr);
  HG_CUDA(cudaGetLastError());
  return HG_OK;
}

int launch_batched_coarse(int dtype, const CoarseBDesc* d, const int* base_mv, const int* base_sc,
                          int nprob, int grid, cudaStream_t s) {
  if (nprob <= 0) return HG_OK;
  if (dtype == HG_F64) {
    coarse_mv_batched_kernel<double><<<grid, kB, 0, s>>>(d, base_mv, nprob);
    coarse_sc_batched_kernel<double><<<grid, kB, 0, s>>>(d, base_sc, nprob);
  } else {
    coarse_mv_batched_kernel<float><<<grid, kB, 0, s>>>(d, base_mv, nprob);
    coarse_sc_batched_kernel<float><<<grid, kB, 0, s>>>(d, base_sc, nprob);
  }
  HG_CUDA(cudaGetLastError());
  return HG_OK;
}

}  // namespace hg
