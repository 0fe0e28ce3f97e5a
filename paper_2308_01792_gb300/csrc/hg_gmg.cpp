// Geometric multigrid on the refinement hierarchy (multigrid by design:
// functions and operators exist on every level, Sec. 5.1) and FP32/FP64
// iterative refinement.  Host orchestration only: every arithmetic step is a
// kernel launch (hg_p1.cu, hg_solver.cu).
#include <cuda_runtime.h>

#include <algorithm>
#include <cmath>
#include <cstring>
#include <memory>
#include <vector>

#include "hg_host.h"

namespace hg {

struct Gmg {
  const Op* op = nullptr;
  const Hier* hier = nullptr;
  hg_gmg_params prm{};
  int lmin = 0, lmax = 0;
  CoarseDev coarse{};
  enum { WX = 0, WB = 1, WR = 2, WT = 3 };
  std::vector<void*> work[2][4];  // [dtype][kind][level - lmin]
  double* r64 = nullptr;          // FP64 residual at lmax
  float* b32 = nullptr;           // scaled FP32 residual at lmax
  float* d32 = nullptr;           // FP32 correction at lmax
  double* dot_scratch = nullptr;
  double* dot_dev = nullptr;
  double* dot_host = nullptr;
  std::vector<double> history;
  const Mlp* learned = nullptr;   // learned smoothing on the finest FP32 level
  bool learned_active = false;
  int learned_fallbacks = 0;

  const LevelDev& L(int l) const { return hier->lv[l - hier->lmin].dev; }
  size_t bytes(int l, int dt) const { return L(l).n_stored * (dt == HG_F64 ? 8 : 4); }

  int alloc_work(int dt) {
    if (!work[dt][0].empty()) return HG_OK;
    for (int kind = 0; kind < 4; ++kind) {
      work[dt][kind].assign(lmax - lmin + 1, nullptr);
      for (int l = lmin; l <= lmax; ++l) {
        void* p = nullptr;
        HG_CUDA(cudaMalloc(&p, bytes(l, dt)));
        HG_CUDA(cudaMemset(p, 0, bytes(l, dt)));
        work[dt][kind][l - lmin] = p;
      }
    }
    return HG_OK;
  }
  void* W(int dt, int kind, int l) { return work[dt][kind][l - lmin]; }

  int dot(int l, int dt, const void* a, const void* b, double* out, cudaStream_t s) {
    if (int r = launch_dot(L(l), dt, a, b, HG_MASK_INNER, dot_scratch, dot_dev, s)) return r;
    HG_CUDA(cudaMemcpyAsync(dot_host, dot_dev, sizeof(double), cudaMemcpyDeviceToHost, s));
    if (int r = hier->fetch_error(s)) return r;
    HG_CUDA(cudaStreamSynchronize(s));
    *out = *dot_host;
    return hier->check_error();
  }

  int cell_op(int l, int dt, int opk, const void* x, const void* b, void* out, cudaStream_t s) {
    StencilArgs a{};
    a.x = x;
    a.b = b;
    a.out = out;
    a.op = opk;
    a.mode = HG_REPLACE;
    a.mask = HG_MASK_INNER;
    a.omega = prm.omega;
    return op->launch(l, dt, a, s);
  }

  int smooth(int l, int dt, void* x, const void* b, int nu, cudaStream_t s) {
    void* t = W(dt, WT, l);
    const bool learn = learned_active && dt == HG_F32 && l == lmax;
    for (int q = 0; q < nu; ++q) {
      const void* src = (q % 2 == 0) ? x : t;
      void* dst = (q % 2 == 0) ? t : x;
      if (learn) {
        // x' = x + omega s + N(s), s = D^-1 (b - A x)
        void* res = W(dt, WR, l);
        if (int r = cell_op(l, dt, OP_RESID, src, b, res, s)) return r;
        if (int r = launch_learned_step(L(l), (const float*)src, (const float*)res,
                                        (const float*)op->vinv[HG_F32][l - hier->lmin],
                                        (float)prm.omega, learned->params, (float*)dst, s))
          return r;
      } else {
        if (int r = cell_op(l, dt, OP_JACOBI, src, b, dst, s)) return r;
      }
    }
    if (nu % 2) HG_CUDA(cudaMemcpyAsync(x, t, bytes(l, dt), cudaMemcpyDeviceToDevice, s));
    return HG_OK;
  }

  int vcycle(int l, int dt, void* x, const void* b, cudaStream_t s) {
    if (l == lmin) return launch_coarse_solve(L(l), coarse, dt, b, x, s);
    if (int r = smooth(l, dt, x, b, prm.nu1, s)) return r;
    void* res = W(dt, WR, l);
    if (int r = cell_op(l, dt, OP_RESID, x, b, res, s)) return r;
    void* bc = W(dt, WB, l - 1);
    void* xc = W(dt, WX, l - 1);
    if (int r = launch_restrict_p1(L(l), L(l - 1), dt, res, bc, s)) return r;
    HG_CUDA(cudaMemsetAsync(xc, 0, bytes(l - 1, dt), s));
    if (int r = vcycle(l - 1, dt, xc, bc, s)) return r;
    if (int r = launch_prolong_p1(L(l), L(l - 1), dt, xc, x, s)) return r;
    return smooth(l, dt, x, b, prm.nu2, s);
  }

  int build_coarse();
  int solve(int precision, double* x, const double* b, double tol, int max_iter, int* iters,
            double* relres, cudaStream_t s);
  ~Gmg();
};

// Dense coarse matrix by applying the operator to unit vectors, then an FP64
// Cholesky factorisation and the explicit inverse (the coarse problem has at
// most a few thousand unknowns).
int Gmg::build_coarse() {
  const LevelHost& H = hier->lv[lmin - hier->lmin];
  const LevelDev& Lc = H.dev;
  if (!hier->mesh->grid_denom) {
    set_error("the coarse solver needs vertex coordinates on an exact lattice");
    return HG_ERR_UNSUPPORTED;
  }
  std::vector<int32_t> int_of_canon(Lc.n_unique, -1);
  std::vector<int64_t> rep;
  for (int64_t u = 0; u < Lc.n_unique; ++u)
    if (!H.dirichlet[u]) {
      int_of_canon[u] = (int32_t)rep.size();
      rep.push_back(H.canon_rep[u]);
    }
  const int n = (int)rep.size();
  coarse.n = n;
  if (n > 2048) {
    set_error("coarsest level has %d unknowns; the dense solver takes at most 2048", n);
    return HG_ERR_INVALID_ARG;
  }
  HG_CUDA(cudaMalloc(&coarse.int_of_canon, std::max<int64_t>(Lc.n_unique, 1) * sizeof(int32_t)));
  HG_CUDA(cudaMemcpy(coarse.int_of_canon, int_of_canon.data(), Lc.n_unique * sizeof(int32_t),
                     cudaMemcpyHostToDevice));
  if (n == 0) return HG_OK;
  HG_CUDA(cudaMalloc(&coarse.stored_rep, n * sizeof(int64_t)));
  HG_CUDA(cudaMemcpy(coarse.stored_rep, rep.data(), n * sizeof(int64_t), cudaMemcpyHostToDevice));
  HG_CUDA(cudaMalloc(&coarse.xint, n * sizeof(double)));
  // columns of the interior operator
  std::vector<double> A((size_t)n * n), canon(Lc.n_unique), col(Lc.n_unique);
  double *dc = nullptr, *dx = nullptr, *dy = nullptr;
  HG_CUDA(cudaMalloc(&dc, Lc.n_unique * sizeof(double)));
  HG_CUDA(cudaMalloc(&dx, Lc.n_stored * sizeof(double)));
  HG_CUDA(cudaMalloc(&dy, Lc.n_stored * sizeof(double)));
  HG_CUDA(cudaMemset(dx, 0, Lc.n_stored * sizeof(double)));
  HG_CUDA(cudaMemset(dy, 0, Lc.n_stored * sizeof(double)));
  int rc = HG_OK;
  std::vector<int64_t> interior;
  for (int64_t u = 0; u < Lc.n_unique; ++u)
    if (int_of_canon[u] >= 0) interior.push_back(u);
  for (int c = 0; c < n && rc == HG_OK; ++c) {
    std::fill(canon.begin(), canon.end(), 0.0);
    canon[interior[c]] = 1.0;
    if (cudaMemcpy(dc, canon.data(), Lc.n_unique * sizeof(double), cudaMemcpyHostToDevice)) {
      rc = cuda_fail(cudaGetLastError(), "cudaMemcpy");
      break;
    }
    if ((rc = launch_from_canonical(Lc, HG_F64, dc, dx, 0))) break;
    if ((rc = cell_op(lmin, HG_F64, OP_APPLY, dx, nullptr, dy, 0))) break;
    if ((rc = launch_to_canonical(Lc, HG_F64, dy, dc, 0))) break;
    if (cudaMemcpy(col.data(), dc, Lc.n_unique * sizeof(double), cudaMemcpyDeviceToHost)) {
      rc = cuda_fail(cudaGetLastError(), "cudaMemcpy");
      break;
    }
    for (int r = 0; r < n; ++r) A[(size_t)r * n + c] = col[interior[r]];
  }
  cudaFree(dc);
  cudaFree(dx);
  cudaFree(dy);
  if (rc) return rc;
  // Cholesky A = L L^T (lower triangle, in place)
  std::vector<double> Lm(A);
  for (int j = 0; j < n; ++j) {
    double d = Lm[(size_t)j * n + j];
    for (int k = 0; k < j; ++k) d -= Lm[(size_t)j * n + k] * Lm[(size_t)j * n + k];
    if (!(d > 0.0)) {
      set_error("coarse matrix is not positive definite (pivot %d = %g)", j, d);
      return HG_ERR_INVALID_ARG;
    }
    const double ljj = std::sqrt(d);
    Lm[(size_t)j * n + j] = ljj;
    for (int i = j + 1; i < n; ++i) {
      double v = Lm[(size_t)i * n + j];
      for (int k = 0; k < j; ++k) v -= Lm[(size_t)i * n + k] * Lm[(size_t)j * n + k];
      Lm[(size_t)i * n + j] = v / ljj;
    }
  }
  // inverse column by column: L z = e_c, L^T x = z
  std::vector<double> inv((size_t)n * n), z(n);
  for (int c = 0; c < n; ++c) {
    for (int i = 0; i < n; ++i) {
      double v = i == c ? 1.0 : 0.0;
      for (int k = 0; k < i; ++k) v -= Lm[(size_t)i * n + k] * z[k];
      z[i] = v / Lm[(size_t)i * n + i];
    }
    for (int i = n - 1; i >= 0; --i) {
      double v = z[i];
      for (int k = i + 1; k < n; ++k) v -= Lm[(size_t)k * n + i] * inv[(size_t)k * n + c];
      inv[(size_t)i * n + c] = v / Lm[(size_t)i * n + i];
    }
  }
  HG_CUDA(cudaMalloc(&coarse.ainv, (size_t)n * n * sizeof(double)));
  HG_CUDA(cudaMemcpy(coarse.ainv, inv.data(), (size_t)n * n * sizeof(double),
                     cudaMemcpyHostToDevice));
  return HG_OK;
}

int Gmg::solve(int precision, double* x, const double* b, double tol, int max_iter, int* iters,
               double* relres, cudaStream_t s) {
  history.clear();
  const int l = lmax;
  HG_CUDA(cudaMemsetAsync(x, 0, bytes(l, HG_F64), s));
  double bb;
  if (int r = dot(l, HG_F64, b, b, &bb, s)) return r;
  const double nb = std::sqrt(bb);
  int it = 0;
  double rel = 0.0;
  learned_active = learned != nullptr;
  learned_fallbacks = 0;
  double prev = 1.0;
  if (nb == 0.0) {
    history.push_back(0.0);
  } else {
    if (precision == HG_PREC_MIXED) {
      if (int r = alloc_work(HG_F32)) return r;
    }
    for (;;) {
      if (int r = cell_op(l, HG_F64, OP_RESID, x, b, r64, s)) return r;
      double rr;
      if (int r = dot(l, HG_F64, r64, r64, &rr, s)) return r;
      const double rn = std::sqrt(rr);
      rel = rn / nb;
      history.push_back(rel);
      // safeguard: if a learned cycle increased the residual, continue with the
      // plain smoother
      if (learned_active && rel > prev) {
        learned_active = false;
        ++learned_fallbacks;
      }
      prev = rel;
      if (rel <= tol || it >= max_iter) break;
      if (precision == HG_PREC_F64) {
        if (int r = vcycle(l, HG_F64, x, b, s)) return r;
      } else {
        if (int r = launch_demote_scaled(L(l).n_stored, r64, 1.0 / rn, b32, s)) return r;
        HG_CUDA(cudaMemsetAsync(d32, 0, bytes(l, HG_F32), s));
        for (int c = 0; c < std::max(prm.inner_cycles, 1); ++c)
          if (int r = vcycle(l, HG_F32, d32, b32, s)) return r;
        if (int r = launch_promote_axpy(L(l).n_stored, rn, d32, x, s)) return r;
      }
      ++it;
    }
  }
  if (iters) *iters = it;
  if (relres) *relres = rel;
  if (rel > tol) {
    set_error("not converged: relative residual %.3e after %d iterations (tol %.1e)", rel, it,
              tol);
    return HG_ERR_NOT_CONVERGED;
  }
  return HG_OK;
}

Gmg::~Gmg() {
  for (auto& per_dt : work)
    for (auto& per_kind : per_dt)
      for (void* p : per_kind) cudaFree(p);
  cudaFree(r64);
  cudaFree(b32);
  cudaFree(d32);
  cudaFree(dot_scratch);
  cudaFree(dot_dev);
  if (dot_host) cudaFreeHost(dot_host);
  cudaFree(coarse.ainv);
  cudaFree(coarse.stored_rep);
  cudaFree(coarse.int_of_canon);
  cudaFree(coarse.xint);
}

}  // namespace hg

using namespace hg;

struct hg_gmg : Gmg {};
struct hg_op : Op {};
struct hg_mlp : Mlp {};

extern "C" {

void hg_gmg_default_params(hg_gmg_params* p) {
  if (!p) return;
  memset(p, 0, sizeof *p);
  p->nu1 = 3;
  p->nu2 = 3;
  p->omega = 2.0 / 3.0;
  p->lmin = -1;
  p->inner_cycles = 1;
}

int hg_gmg_create(const hg_op* op, const hg_gmg_params* prm, hg_gmg** out) {
  if (!op || !out) {
    set_error("hg_gmg_create: null argument");
    return HG_ERR_INVALID_ARG;
  }
  auto g = std::make_unique<hg_gmg>();
  g->op = op;
  g->hier = op->hier;
  if (prm) {
    g->prm = *prm;
  } else {
    hg_gmg_default_params(&g->prm);
  }
  const Hier* h = op->hier;
  g->lmax = h->lmax;
  g->lmin = g->prm.lmin < 0 ? h->lmin : g->prm.lmin;
  if (g->lmin < h->lmin || g->lmin > h->lmax) {
    set_error("coarsest level %d outside the hierarchy %d..%d", g->lmin, h->lmin, h->lmax);
    return HG_ERR_LEVEL_RANGE;
  }
  if (g->prm.nu1 < 0 || g->prm.nu2 < 0 || !(g->prm.omega > 0.0)) {
    set_error("bad smoother parameters nu1=%d nu2=%d omega=%g", g->prm.nu1, g->prm.nu2,
              g->prm.omega);
    return HG_ERR_INVALID_ARG;
  }
  if (int r = g->alloc_work(HG_F64)) return r;
  const size_t nl = g->L(g->lmax).n_stored;
  HG_CUDA(cudaMalloc(&g->r64, nl * sizeof(double)));
  HG_CUDA(cudaMalloc(&g->b32, nl * sizeof(float)));
  HG_CUDA(cudaMalloc(&g->d32, nl * sizeof(float)));
  HG_CUDA(cudaMemset(g->r64, 0, nl * sizeof(double)));
  HG_CUDA(cudaMemset(g->b32, 0, nl * sizeof(float)));
  HG_CUDA(cudaMemset(g->d32, 0, nl * sizeof(float)));
  HG_CUDA(cudaMalloc(&g->dot_scratch, dot_scratch_len(g->L(g->lmax)) * sizeof(double)));
  HG_CUDA(cudaMalloc(&g->dot_dev, sizeof(double)));
  HG_CUDA(cudaMallocHost(&g->dot_host, sizeof(double)));
  if (int r = g->build_coarse()) return r;
  *out = g.release();
  return HG_OK;
}

void hg_gmg_destroy(hg_gmg* g) { delete g; }

int hg_vcycle(hg_gmg* g, int level, int dtype, void* x, const void* b, void* stream) {
  if (!g || !x || !b || x == b) {
    set_error("hg_vcycle: bad argument");
    return HG_ERR_INVALID_ARG;
  }
  if (level < g->lmin || level > g->lmax) {
    set_error("level %d outside %d..%d", level, g->lmin, g->lmax);
    return HG_ERR_LEVEL_RANGE;
  }
  if (dtype != HG_F32 && dtype != HG_F64) {
    set_error("bad dtype %d", dtype);
    return HG_ERR_INVALID_ARG;
  }
  if (int r = g->alloc_work(dtype)) return r;
  g->learned_active = g->learned != nullptr;
  return g->vcycle(level, dtype, x, b, (cudaStream_t)stream);
}

int hg_solve(hg_gmg* g, int precision, double* x, const double* b, double rel_tol, int max_iter,
             int* iters, double* rel_res, void* stream) {
  if (!g || !x || !b || (const void*)x == (const void*)b || max_iter < 0) {
    set_error("hg_solve: bad argument");
    return HG_ERR_INVALID_ARG;
  }
  if (precision != HG_PREC_F64 && precision != HG_PREC_MIXED) {
    set_error("hg_solve: unknown precision mode %d", precision);
    return HG_ERR_INVALID_ARG;
  }
  return g->solve(precision, x, b, rel_tol, max_iter, iters, rel_res, (cudaStream_t)stream);
}

int hg_gmg_set_learned(hg_gmg* g, const hg_mlp* mlp) {
  if (!g) {
    set_error("hg_gmg_set_learned: null handle");
    return HG_ERR_INVALID_ARG;
  }
  if (mlp && g->op->vinv[HG_F32].empty()) {
    set_error("learned smoothing needs the operator's stored diagonal (exact lattice)");
    return HG_ERR_UNSUPPORTED;
  }
  g->learned = mlp;
  return HG_OK;
}

int hg_gmg_learned_fallbacks(const hg_gmg* g, int* n) {
  if (!g || !n) {
    set_error("hg_gmg_learned_fallbacks: null argument");
    return HG_ERR_INVALID_ARG;
  }
  *n = g->learned_fallbacks;
  return HG_OK;
}

int hg_gmg_history(const hg_gmg* g, double* out, int cap, int* n) {
  if (!g) {
    set_error("hg_gmg_history: null handle");
    return HG_ERR_INVALID_ARG;
  }
  if (n) *n = (int)g->history.size();
  if (out)
    for (int q = 0; q < cap && q < (int)g->history.size(); ++q) out[q] = g->history[q];
  return HG_OK;
}

}  // extern "C"
