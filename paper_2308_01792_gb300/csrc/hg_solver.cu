// Solver kernels: the dense FP64 coarse-grid solve and the element-wise
// steps of mixed-precision iterative refinement.
#include <cuda_runtime.h>

#include "hg_internal.h"

namespace hg {

namespace {

constexpr int kBlock = 256;

// x_int = A_c^-1 b_int: one warp per row of the row-major inverse, b gathered
// from the owner copies of the interior unknowns.
template <typename T>
__global__ void __launch_bounds__(kBlock) coarse_matvec_kernel(int n, const double* __restrict__ ainv,
                                                               const int64_t* __restrict__ rep,
                                                               const T* __restrict__ b,
                                                               double* __restrict__ xint) {
  const int lane = threadIdx.x & 31;
  const int row = blockIdx.x * (kBlock / 32) + (threadIdx.x >> 5);
  if (row >= n) return;
  double acc = 0.0;
  for (int c = lane; c < n; c += 32) acc += ainv[(int64_t)row * n + c] * (double)b[rep[c]];
  for (int o = 16; o > 0; o >>= 1) acc += __shfl_down_sync(0xffffffffu, acc, o);
  if (lane == 0) xint[row] = acc;
}

// Every stored copy of an interior unknown receives its value.
template <typename T>
__global__ void coarse_scatter_kernel(int64_t ns, const int32_t* __restrict__ canon,
                                      const int32_t* __restrict__ int_of_canon,
                                      const double* __restrict__ xint, T* __restrict__ x) {
  for (int64_t q = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; q < ns;
       q += (int64_t)gridDim.x * blockDim.x) {
    const int32_t u = canon[q];
    if (u < 0) continue;
    const int32_t iu = int_of_canon[u];
    if (iu >= 0) x[q] = (T)xint[iu];
  }
}

// r32 = r64 * scale (FP64 residual to the scaled FP32 right-hand side).
__global__ void demote_scaled_kernel(int64_t n, const double* __restrict__ r, double scale,
                                     float* __restrict__ out) {
  for (int64_t q = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; q < n;
       q += (int64_t)gridDim.x * blockDim.x)
    out[q] = (float)(r[q] * scale);
}

// x64 += alpha * d32 (correction from the FP32 inner solve).
__global__ void promote_axpy_kernel(int64_t n, double alpha, const float* __restrict__ d,
                                    double* __restrict__ x) {
  for (int64_t q = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; q < n;
       q += (int64_t)gridDim.x * blockDim.x)
    x[q] += alpha * (double)d[q];
}

int grid_flat(int64_t n) {
  int64_t g = (n + kBlock - 1) / kBlock;
  return (int)(g < 152 * 8 ? (g > 0 ? g : 1) : 152 * 8);
}

}  // namespace

int launch_coarse_solve(const LevelDev& L, const CoarseDev& C, int dtype, const void* b, void* x,
                        cudaStream_t s) {
  if (C.n <= 0) return HG_OK;
  const int g = (C.n + kBlock / 32 - 1) / (kBlock / 32);
  if (dtype == HG_F64) {
    coarse_matvec_kernel<double><<<g, kBlock, 0, s>>>(C.n, C.ainv, C.stored_rep, (const double*)b,
                                                      C.xint);
    HG_CUDA(cudaGetLastError());
    coarse_scatter_kernel<double><<<grid_flat(L.n_stored), kBlock, 0, s>>>(
        L.n_stored, L.canon, C.int_of_canon, C.xint, (double*)x);
  } else {
    coarse_matvec_kernel<float><<<g, kBlock, 0, s>>>(C.n, C.ainv, C.stored_rep, (const float*)b,
                                                     C.xint);
    HG_CUDA(cudaGetLastError());
    coarse_scatter_kernel<float><<<grid_flat(L.n_stored), kBlock, 0, s>>>(
        L.n_stored, L.canon, C.int_of_canon, C.xint, (float*)x);
  }
  HG_CUDA(cudaGetLastError());
  return HG_OK;
}

int launch_demote_scaled(int64_t n, const double* r, double scale, float* out, cudaStream_t s) {
  demote_scaled_kernel<<<grid_flat(n), kBlock, 0, s>>>(n, r, scale, out);
  HG_CUDA(cudaGetLastError());
  return HG_OK;
}

int launch_promote_axpy(int64_t n, double alpha, const float* d, double* x, cudaStream_t s) {
  promote_axpy_kernel<<<grid_flat(n), kBlock, 0, s>>>(n, alpha, d, x);
  HG_CUDA(cudaGetLastError());
  return HG_OK;
}

}  // namespace hg
