// Functions on a level range (Sec. 5.1: a finite-element function owns one
// vector per level of the hierarchy) and their copies from and to host
// memory in the canonical DoF order.  The vectors are caller-owned device
// buffers bound level by level; the library owns only the staging buffers
// of the host copies.
#include <cuda_runtime.h>

#include <memory>

#include "hg_host.h"
#include "hytet.h"

namespace hg {

void* Func::data(int level) const {
  const int li = lattice_index(hier, space, level);
  if (li < 0) {
    set_error("level %d of space %d outside the hierarchy %d..%d", level, space, hier->lmin,
              hier->lmax);
    return nullptr;
  }
  if (!ptr[li]) {
    set_error("function has no vector bound on level %d", level);
    return nullptr;
  }
  return ptr[li];
}

Func::~Func() {
  for (void* p : stage)
    if (p) cudaFree(p);
}

}  // namespace hg

using namespace hg;

struct hg_hier : Hier {};
struct hg_op : Op {};
struct hg_func : Func {};

extern "C" {

int hg_function_create(const hg_hier* h, int space, int dtype, hg_func** out) {
  if (!h || !out) {
    set_error("hg_function_create: null argument");
    return HG_ERR_INVALID_ARG;
  }
  if (space != HG_SPACE_P1 && space != HG_SPACE_P2) {
    set_error("hg_function_create: space %d not available", space);
    return HG_ERR_UNSUPPORTED;
  }
  if (dtype != HG_F32 && dtype != HG_F64) {
    set_error("hg_function_create: dtype %d not available", dtype);
    return HG_ERR_INVALID_ARG;
  }
  auto f = std::make_unique<hg_func>();
  f->hier = h;
  f->space = space;
  f->dtype = dtype;
  f->ptr.assign(h->lv.size(), nullptr);
  f->stage.assign(h->lv.size(), nullptr);
  *out = f.release();
  return HG_OK;
}

void hg_function_destroy(hg_func* f) { delete f; }

int hg_function_bind(hg_func* f, int level, void* dev_ptr, int64_t nbytes) {
  if (!f) {
    set_error("hg_function_bind: null function");
    return HG_ERR_INVALID_ARG;
  }
  const int li = lattice_index(f->hier, f->space, level);
  if (li < 0) {
    set_error("hg_function_bind: level %d of space %d outside the hierarchy", level, f->space);
    return HG_ERR_LEVEL_RANGE;
  }
  if (dev_ptr) {
    const int64_t need = f->hier->lv[li].dev.n_stored * (f->dtype == HG_F64 ? 8 : 4);
    if (nbytes < need || (uintptr_t)dev_ptr % 16) {
      set_error("hg_function_bind: level %d needs %lld bytes at a 16-byte boundary, got %lld",
                level, (long long)need, (long long)nbytes);
      return HG_ERR_INVALID_ARG;
    }
  }
  f->ptr[li] = dev_ptr;
  return HG_OK;
}

int hg_function_data(const hg_func* f, int level, void** dev_ptr) {
  if (!f || !dev_ptr) {
    set_error("hg_function_data: null argument");
    return HG_ERR_INVALID_ARG;
  }
  const int li = lattice_index(f->hier, f->space, level);
  if (li < 0) {
    set_error("hg_function_data: level %d of space %d outside the hierarchy", level, f->space);
    return HG_ERR_LEVEL_RANGE;
  }
  *dev_ptr = f->ptr[li];
  return HG_OK;
}

int hg_function_copy_canonical(hg_func* f, int level, void* host, int host_dtype, int64_t n,
                               int dir, void* stream) {
  if (!f || !host) {
    set_error("hg_function_copy_canonical: null argument");
    return HG_ERR_INVALID_ARG;
  }
  if ((host_dtype != HG_F32 && host_dtype != HG_F64) ||
      (dir != HG_COPY_TO_HOST && dir != HG_COPY_FROM_HOST)) {
    set_error("hg_function_copy_canonical: bad host dtype %d or direction %d", host_dtype, dir);
    return HG_ERR_INVALID_ARG;
  }
  if (!f->hier->mesh->grid_denom) {
    set_error("hg_function_copy_canonical: mesh has no exact lattice");
    return HG_ERR_UNSUPPORTED;
  }
  void* st = f->data(level);
  if (!st) return lattice_index(f->hier, f->space, level) < 0 ? HG_ERR_LEVEL_RANGE
                                                               : HG_ERR_INVALID_ARG;
  const int li = lattice_index(f->hier, f->space, level);
  const LevelDev& L = f->hier->lv[li].dev;
  if (n != L.n_unique) {
    set_error("hg_function_copy_canonical: level %d has %lld unique DoFs, got n = %lld", level,
              (long long)L.n_unique, (long long)n);
    return HG_ERR_INVALID_ARG;
  }
  if (!f->stage[li] && n > 0) {
    cudaError_t e = cudaMalloc(&f->stage[li], (size_t)n * 8);
    if (e != cudaSuccess) {
      f->stage[li] = nullptr;
      set_error("hg_function_copy_canonical: %s", cudaGetErrorString(e));
      return HG_ERR_CUDA;
    }
  }
  if (n == 0) return HG_OK;
  cudaStream_t s = (cudaStream_t)stream;
  const size_t bytes = (size_t)n * (host_dtype == HG_F64 ? 8 : 4);
  if (dir == HG_COPY_FROM_HOST) {
    cudaError_t e = cudaMemcpyAsync(f->stage[li], host, bytes, cudaMemcpyHostToDevice, s);
    if (e != cudaSuccess) {
      set_error("hg_function_copy_canonical: %s", cudaGetErrorString(e));
      return HG_ERR_CUDA;
    }
    return launch_from_canonical(L, f->dtype, f->stage[li], st, s, host_dtype);
  }
  if (int r = launch_to_canonical(L, f->dtype, st, f->stage[li], s, host_dtype)) return r;
  cudaError_t e = cudaMemcpyAsync(host, f->stage[li], bytes, cudaMemcpyDeviceToHost, s);
  if (e != cudaSuccess) {
    set_error("hg_function_copy_canonical: %s", cudaGetErrorString(e));
    return HG_ERR_CUDA;
  }
  return HG_OK;
}

int hg_apply_function(const hg_op* op, int level, const hg_func* x, hg_func* y, int mode, int mask,
                      void* stream) {
  if (!op || !x || !y || x == y) {
    set_error("hg_apply_function: null or identical functions");
    return HG_ERR_INVALID_ARG;
  }
  if (x->hier != op->hier || y->hier != op->hier || x->space != op->space ||
      y->space != op->space || x->dtype != y->dtype) {
    set_error("hg_apply_function: functions of another hierarchy, space or element type");
    return HG_ERR_INVALID_ARG;
  }
  const void* xp = x->data(level);
  void* yp = y->data(level);
  if (!xp || !yp) return HG_ERR_INVALID_ARG;
  return hg_apply(op, level, x->dtype, xp, yp, mode, mask, stream);
}

}  // extern "C"
