// Dot product that allocates nothing, for callers that cannot call cudaMalloc.
//
// Some callers may not allocate device memory at the point where they need a
// norm: code running inside a memory pool or arena that owns all of the
// device memory, code that must not synchronise the device the way
// cudaMalloc/cudaFree can, or code on a path where allocation is forbidden.
// hg_dot keeps its per-block partial sums in buffers the hierarchy allocated
// at creation; hg_dot_noalloc computes the same deterministic FP64 dot but
// keeps the partial sums in the fixed array below and writes the result to a
// device pointer the caller supplies.
//
// The array lives in every GPU that loads this library until the process
// exits.  All calls share it: two calls that overlap on the GPU (different
// streams, or different host threads) race on it and give wrong results.
// Every call rewrites every partial it reads, so nothing needs clearing.
#include <cuda_runtime.h>

#include <mutex>

#include "hg_host.h"

namespace hg {
namespace {

// One partial per block, kNoAllocRowsPerBlock lattice rows per block.
constexpr int kNoAllocMaxBlocks = 512;
constexpr int kNoAllocRowsPerBlock = 256;
constexpr int kNoAllocThreads = 256;

}  // namespace
}  // namespace hg

static __device__ __align__(256) double g_noalloc_partials[hg::kNoAllocMaxBlocks];

namespace hg {
namespace {

template <typename T>
__global__ void __launch_bounds__(kNoAllocThreads) noalloc_dot_partial(
    int n, int64_t stride, const uint8_t* __restrict__ flags, int n_rows, const T* __restrict__ X,
    const T* __restrict__ Y, int mask, double* __restrict__ partials) {
  const int w = n + 1;
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  constexpr int kW = kNoAllocThreads / 32;
  double acc = 0.0;
  const int r_end = min(n_rows, (int)(blockIdx.x + 1) * kNoAllocRowsPerBlock);
  for (int r = blockIdx.x * kNoAllocRowsPerBlock + warp; r < r_end; r += kW) {
    int cell, j, k;
    row_item(w, r, cell, j, k);
    const int64_t r0 = (int64_t)cell * stride + row_start(w, j, k);
    const uint8_t* fl = flags + cell * 16;
    for (int i = lane; i + j + k <= n; i += 32) {
      const uint8_t f = fl[point_class(n, i, j, k)];
      if (!(f & CF_OWNER)) continue;                     // each unique DoF once
      if (mask == HG_MASK_INNER && (f & CF_DIRICHLET)) continue;
      acc += (double)X[r0 + i] * (double)Y[r0 + i];
    }
  }
  __shared__ double red[kW];
  for (int o = 16; o > 0; o >>= 1) acc += __shfl_down_sync(0xffffffffu, acc, o);
  if (lane == 0) red[warp] = acc;
  __syncthreads();
  if (threadIdx.x == 0) {
    double t = 0.0;
    for (int q = 0; q < kW; ++q) t += red[q];
    partials[blockIdx.x] = t;
  }
}

// Fixed-order tree sum of the nb partials into *out (device).
__global__ void __launch_bounds__(kNoAllocMaxBlocks) noalloc_dot_final(
    const double* __restrict__ partials, int nb, double* __restrict__ out) {
  __shared__ double red[kNoAllocMaxBlocks];
  red[threadIdx.x] = (int)threadIdx.x < nb ? partials[threadIdx.x] : 0.0;
  __syncthreads();
  for (int o = kNoAllocMaxBlocks / 2; o > 0; o >>= 1) {
    if ((int)threadIdx.x < o) red[threadIdx.x] += red[threadIdx.x + o];
    __syncthreads();
  }
  if (threadIdx.x == 0) *out = red[0];
}

// Device address of g_noalloc_partials, looked up once per device (with that
// device current) on the first call made on it, and kept for the life of the
// process.  The cached address does not survive a reset of the device's
// context (cudaDeviceReset): after one, this library must not be used again in
// the same process.
constexpr int kMaxDevices = 64;
std::mutex g_noalloc_mu;
double* g_noalloc_ptr[kMaxDevices] = {};

int noalloc_scratch(double** out) {
  int dev = 0;
  HG_CUDA(cudaGetDevice(&dev));
  if (dev < 0 || dev >= kMaxDevices) {
    set_error("hg_dot_noalloc: device %d beyond the %d supported", dev, kMaxDevices);
    return HG_ERR_UNSUPPORTED;
  }
  std::lock_guard<std::mutex> lock(g_noalloc_mu);
  if (!g_noalloc_ptr[dev]) {
    void* p = nullptr;
    const cudaError_t e = cudaGetSymbolAddress(&p, g_noalloc_partials);
    if (e != cudaSuccess) return cuda_fail(e, "cudaGetSymbolAddress(g_noalloc_partials)");
    g_noalloc_ptr[dev] = static_cast<double*>(p);
  }
  *out = g_noalloc_ptr[dev];
  return HG_OK;
}

}  // namespace
}  // namespace hg

using namespace hg;

struct hg_hier : Hier {};

extern "C" int hg_dot_noalloc(const hg_hier* h, int space, int level, int dtype, const void* x,
                              const void* y, int mask, double* result, void* stream) {
  if (!h || !x || !y || !result) {
    set_error("hg_dot_noalloc: null argument");
    return HG_ERR_INVALID_ARG;
  }
  if (space != HG_SPACE_P1 || (dtype != HG_F32 && dtype != HG_F64) ||
      (mask != HG_MASK_INNER && mask != HG_MASK_ALL)) {
    set_error("hg_dot_noalloc: unsupported space %d / dtype %d / mask %d", space, dtype, mask);
    return HG_ERR_INVALID_ARG;
  }
  if (level < h->lmin || level > h->lmax) {
    set_error("hg_dot_noalloc: level %d outside %d..%d", level, h->lmin, h->lmax);
    return HG_ERR_LEVEL_RANGE;
  }
  const LevelDev& L = h->lv[level - h->lmin].dev;
  const int64_t n_rows = (int64_t)L.ncells * ntri(L.w);
  const int64_t nb = (n_rows + kNoAllocRowsPerBlock - 1) / kNoAllocRowsPerBlock;
  if (nb > kNoAllocMaxBlocks) {
    set_error(
        "hg_dot_noalloc: level %d has %lld lattice rows; the fixed scratch holds %d partials of "
        "%d rows, i.e. at most %d rows",
        level, (long long)n_rows, kNoAllocMaxBlocks, kNoAllocRowsPerBlock,
        kNoAllocMaxBlocks * kNoAllocRowsPerBlock);
    return HG_ERR_INVALID_ARG;
  }
  double* scratch = nullptr;
  if (int r = noalloc_scratch(&scratch)) return r;
  cudaStream_t s = (cudaStream_t)stream;
  if (nb > 0) {
    if (dtype == HG_F64)
      noalloc_dot_partial<double><<<(int)nb, kNoAllocThreads, 0, s>>>(
          L.n, L.cell_stride, L.cls_flags, (int)n_rows, (const double*)x, (const double*)y, mask,
          scratch);
    else
      noalloc_dot_partial<float><<<(int)nb, kNoAllocThreads, 0, s>>>(
          L.n, L.cell_stride, L.cls_flags, (int)n_rows, (const float*)x, (const float*)y, mask,
          scratch);
    HG_CUDA(cudaGetLastError());
  }
  noalloc_dot_final<<<1, kNoAllocMaxBlocks, 0, s>>>(scratch, (int)nb, result);
  HG_CUDA(cudaGetLastError());
  return HG_OK;
}
