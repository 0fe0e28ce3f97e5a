// Learned local smoother: network handle, training (forward/backward/Adam on
// the GPU) and the sampling of training pairs.  Host orchestration only; the
// arithmetic is in hg_mlp.cu.
#include <cuda_runtime.h>

#include <algorithm>
#include <cstring>
#include <memory>
#include <vector>

#include "hg_host.h"

namespace hg {

int Mlp::build() {
  partial_blocks = mlp_grad_blocks(int64_t(1) << 40);
  HG_CUDA(cudaMalloc(&params, kMlpParams * sizeof(float)));
  HG_CUDA(cudaMalloc(&grad, kMlpParams * sizeof(float)));
  HG_CUDA(cudaMalloc(&m, kMlpParams * sizeof(float)));
  HG_CUDA(cudaMalloc(&v, kMlpParams * sizeof(float)));
  HG_CUDA(cudaMalloc(&partial, (size_t)partial_blocks * kMlpParams * sizeof(float)));
  HG_CUDA(cudaMalloc(&lpart, partial_blocks * sizeof(double)));
  HG_CUDA(cudaMalloc(&loss, sizeof(double)));
  HG_CUDA(cudaMallocHost(&loss_host, sizeof(double)));
  HG_CUDA(cudaMemset(params, 0, kMlpParams * sizeof(float)));
  HG_CUDA(cudaMemset(m, 0, kMlpParams * sizeof(float)));
  HG_CUDA(cudaMemset(v, 0, kMlpParams * sizeof(float)));
  return HG_OK;
}

Mlp::~Mlp() {
  cudaFree(params);
  cudaFree(grad);
  cudaFree(m);
  cudaFree(v);
  cudaFree(partial);
  cudaFree(lpart);
  cudaFree(loss);
  if (loss_host) cudaFreeHost(loss_host);
}

}  // namespace hg

using namespace hg;

struct hg_mlp : Mlp {};
struct hg_op : Op {};

#define HG_CHECK(cond, code, ...) \
  do {                            \
    if (!(cond)) {                \
      set_error(__VA_ARGS__);     \
      return code;                \
    }                             \
  } while (0)

extern "C" {

int hg_mlp_create(hg_mlp** out) {
  HG_CHECK(out, HG_ERR_INVALID_ARG, "hg_mlp_create: null argument");
  auto m = std::make_unique<hg_mlp>();
  if (int r = m->build()) return r;
  *out = m.release();
  return HG_OK;
}

void hg_mlp_destroy(hg_mlp* m) { delete m; }

int hg_mlp_set_params(hg_mlp* m, const float* host) {
  HG_CHECK(m && host, HG_ERR_INVALID_ARG, "hg_mlp_set_params: null argument");
  HG_CUDA(cudaMemcpy(m->params, host, kMlpParams * sizeof(float), cudaMemcpyHostToDevice));
  HG_CUDA(cudaMemset(m->m, 0, kMlpParams * sizeof(float)));
  HG_CUDA(cudaMemset(m->v, 0, kMlpParams * sizeof(float)));
  m->step = 0;
  return HG_OK;
}

int hg_mlp_get_params(const hg_mlp* m, float* host) {
  HG_CHECK(m && host, HG_ERR_INVALID_ARG, "hg_mlp_get_params: null argument");
  HG_CUDA(cudaMemcpy(host, m->params, kMlpParams * sizeof(float), cudaMemcpyDeviceToHost));
  return HG_OK;
}

int hg_mlp_forward(const hg_mlp* m, const float* X, int64_t n, float* out, void* stream) {
  HG_CHECK(m && X && out && n >= 0, HG_ERR_INVALID_ARG, "hg_mlp_forward: bad argument");
  return launch_mlp_forward(X, n, m->params, m->params + 512, m->params + 1536, out,
                            (cudaStream_t)stream);
}

int hg_mlp_grad(hg_mlp* m, const void* Xbf16, const float* t, int64_t n, float* grad_host,
                double* loss_host, void* stream) {
  HG_CHECK(m && Xbf16 && t && n > 0 && ((uintptr_t)Xbf16 & 15) == 0, HG_ERR_INVALID_ARG,
           "hg_mlp_grad: bad argument (samples must be 16-byte aligned)");
  cudaStream_t s = (cudaStream_t)stream;
  if (int r = launch_mlp_grad(Xbf16, t, n, 0, n, m->params, m->params + 512, m->params + 1536,
                              m->partial, m->lpart, m->grad, m->loss, s))
    return r;
  if (grad_host)
    HG_CUDA(cudaMemcpyAsync(grad_host, m->grad, kMlpParams * sizeof(float),
                            cudaMemcpyDeviceToHost, s));
  HG_CUDA(cudaMemcpyAsync(m->loss_host, m->loss, sizeof(double), cudaMemcpyDeviceToHost, s));
  HG_CUDA(cudaStreamSynchronize(s));
  if (loss_host) *loss_host = *m->loss_host;
  return HG_OK;
}

int hg_mlp_train(hg_mlp* m, const void* Xbf16, const float* t, int64_t n, int steps,
                 int64_t batch, double lr, double* final_loss, void* stream) {
  HG_CHECK(m && Xbf16 && t && n > 0 && steps >= 0 && batch > 0 && lr > 0 &&
               ((uintptr_t)Xbf16 & 15) == 0,
           HG_ERR_INVALID_ARG, "hg_mlp_train: bad argument");
  cudaStream_t s = (cudaStream_t)stream;
  batch = std::min(batch, n);
  int64_t first = 0;
  for (int q = 0; q < steps; ++q) {
    if (first + batch > n) first = 0;
    if (int r = launch_mlp_grad(Xbf16, t, n, first, batch, m->params, m->params + 512,
                                m->params + 1536, m->partial, m->lpart, m->grad, m->loss, s))
      return r;
    if (int r = launch_mlp_adam(m->params, m->grad, m->m, m->v, (float)lr, ++m->step, s)) return r;
    first += batch;
  }
  if (final_loss) {
    if (int r = launch_mlp_grad(Xbf16, t, n, 0, n, m->params, m->params + 512, m->params + 1536,
                                m->partial, m->lpart, m->grad, m->loss, s))
      return r;
    HG_CUDA(cudaMemcpyAsync(m->loss_host, m->loss, sizeof(double), cudaMemcpyDeviceToHost, s));
    HG_CUDA(cudaStreamSynchronize(s));
    *final_loss = *m->loss_host;
  }
  return HG_OK;
}

int hg_learned_step(const hg_op* op, const hg_mlp* mlp, int level, const float* x,
                    const float* r, double omega, float* x_out, void* stream) {
  HG_CHECK(op && mlp && x && r && x_out, HG_ERR_INVALID_ARG, "hg_learned_step: null argument");
  HG_CHECK(x_out != x && x_out != r, HG_ERR_INVALID_ARG, "hg_learned_step: x_out aliases an input");
  const Hier* h = op->hier;
  HG_CHECK(op->space == HG_SPACE_P1, HG_ERR_UNSUPPORTED, "hg_learned_step: P1 operators only");
  HG_CHECK(level >= h->lmin && level <= h->lmax, HG_ERR_LEVEL_RANGE, "level out of range");
  HG_CHECK(!op->vinv[HG_F32].empty(), HG_ERR_UNSUPPORTED,
           "hg_learned_step: operator has no stored diagonal");
  const LevelDev& L = h->lv[level - h->lmin].dev;
  return launch_learned_step(L, x, r, (const float*)op->vinv[HG_F32][level - h->lmin],
                             (float)omega, mlp->params, x_out, (cudaStream_t)stream);
}

int hg_learn_samples(const hg_op* op, int level, const float* r, const float* xstar,
                     const float* x, double omega, int stride, int offset, void* X, float* t,
                     int64_t* count, void* stream) {
  HG_CHECK(op && stride >= 1 && offset >= 0 && offset < stride, HG_ERR_INVALID_ARG,
           "hg_learn_samples: bad argument");
  const Hier* h = op->hier;
  HG_CHECK(level >= h->lmin && level <= h->lmax, HG_ERR_LEVEL_RANGE, "level out of range");
  HG_CHECK(!op->vinv[HG_F32].empty(), HG_ERR_UNSUPPORTED,
           "operator has no stored diagonal (needs an exact lattice)");
  const LevelDev& L = h->lv[level - h->lmin].dev;
  const int64_t cnt = learned_sample_count(L, stride, offset);
  if (count) *count = cnt;
  if (!X) return HG_OK;
  HG_CHECK(r && xstar && x && t, HG_ERR_INVALID_ARG, "hg_learn_samples: null vector");
  return launch_learned_sample(L, r, (const float*)op->vinv[HG_F32][level - h->lmin], xstar, x,
                               (float)omega, stride, offset, X, t, (cudaStream_t)stream);
}

}  // extern "C"
