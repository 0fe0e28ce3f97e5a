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
  // work vectors per level: coarse correction, coarse rhs, residual,
  // smoother partner, Chebyshev direction, FMG right-hand side
  enum { WX = 0, WB = 1, WR = 2, WT = 3, WD = 4, WF = 5, NWORK = 6 };
  std::vector<void*> work[2][NWORK];  // [dtype][kind][level - lmin]
  std::vector<double> lam;         // Chebyshev: lambda_max(D^-1 A) per level - lmin
  std::vector<double> lam_p;       // Nedelec + Chebyshev: lambda_max of the potential space
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
  // Nedelec operators: Hiptmair smoothing with the P1 Laplacian of the same
  // hierarchy as the potential-space operator (G^T A G = beta K_P1)
  Op* pot = nullptr;
  // [dtype][residual, correction, zero, second iterate, direction][level - lmin]
  std::vector<void*> pwork[2][5];
  bool is_n1() const { return op->kind == HG_OP_N1_CURLCURL; }

  const LevelDev& L(int l) const { return op->dev(l); }
  size_t bytes(int l, int dt) const { return L(l).n_stored * (dt == HG_F64 ? 8 : 4); }

  int alloc_work(int dt) {
    if (!work[dt][0].empty()) return HG_OK;
    for (int kind = 0; kind < NWORK; ++kind) {
      work[dt][kind].assign(lmax - lmin + 1, nullptr);
      for (int l = lmin; l <= lmax; ++l) {
        void* p = nullptr;
        HG_CUDA(cudaMalloc(&p, bytes(l, dt)));
        HG_CUDA(cudaMemset(p, 0, bytes(l, dt)));
        work[dt][kind][l - lmin] = p;
      }
    }
    if (pot)
      if (int r = alloc_pot(dt)) return r;
    return HG_OK;
  }
  void* W(int dt, int kind, int l) { return work[dt][kind][l - lmin]; }

  int alloc_pot(int dt) {
    if (!pwork[dt][0].empty()) return HG_OK;
    for (int kind = 0; kind < 5; ++kind) {
      pwork[dt][kind].assign(lmax - lmin + 1, nullptr);
      for (int l = lmin + 1; l <= lmax; ++l) {
        const size_t nb = pot->dev(l).n_stored * (dt == HG_F64 ? 8 : 4);
        void* p = nullptr;
        HG_CUDA(cudaMalloc(&p, nb));
        HG_CUDA(cudaMemset(p, 0, nb));
        pwork[dt][kind][l - lmin] = p;
      }
    }
    return HG_OK;
  }

  int restrict_to(int l, int dt, const void* rf, void* rc, cudaStream_t s) {
    if (is_n1()) return launch_n1_transfer(N1_RESTRICT, L(l), L(l - 1), dt, op->n1sign, rf, rc, s);
    return op->space == HG_SPACE_P2 ? launch_restrict_p2(L(l), L(l - 1), dt, rf, rc, s)
                                    : launch_restrict_p1(L(l), L(l - 1), dt, rf, rc, s);
  }
  int prolong_to(int l, int dt, const void* ec, void* xf, cudaStream_t s) {
    if (is_n1()) return launch_n1_transfer(N1_PROLONG, L(l), L(l - 1), dt, op->n1sign, ec, xf, s);
    return op->space == HG_SPACE_P2 ? launch_prolong_p2(L(l), L(l - 1), dt, ec, xf, s)
                                    : launch_prolong_p1(L(l), L(l - 1), dt, ec, xf, s);
  }

  // Hiptmair hybrid smoothing (Sec. 6): per step a smoothing step on A in the
  // edge space, the residual taken to the potential space by G^T, a
  // smoothing step from zero with G^T A G = beta K_P1, and the correction
  // G e_p added; the steps ping-pong x and t.  Jacobi (weight omega; in the
  // potential space omega / beta on the P1 Laplacian, exact from zero) or,
  // with HG_SMOOTH_CHEB, cheb_order Chebyshev steps in both spaces (the
  // paper's choice).  The potential iteration runs in y = beta e_p, for which
  // it is the plain Chebyshev iteration on K_P1 y = G^T r (D^-1 A is the same
  // for beta K_P1 and K_P1), and G y / beta is added.
  int smooth_hiptmair(int l, int dt, void* x, const void* b, int nu, cudaStream_t s) {
    void* t = W(dt, WT, l);
    void* r = W(dt, WR, l);
    void* rp = pwork[dt][0][l - lmin];
    void* ep = pwork[dt][1][l - lmin];
    void* z = pwork[dt][2][l - lmin];
    const LevelDev& Lp = pot->dev(l);
    const bool cheb = prm.smoother == HG_SMOOTH_CHEB;
    for (int q = 0; q < nu; ++q) {
      const void* src = (q % 2 == 0) ? x : t;
      void* dst = (q % 2 == 0) ? t : x;
      if (cheb) {
        // the iterates alternate between r and dst so that the last lands in dst
        if (int e = cheb_poly(op, l, dt, lam[l - lmin], src, b, dst, r, W(dt, WD, l), s)) return e;
      } else {
        if (int e = cell_op(l, dt, OP_JACOBI, src, b, dst, s)) return e;
      }
      if (int e = cell_op(l, dt, OP_RESID, dst, b, r, s)) return e;
      if (int e = launch_n1_transfer(N1_GRADT, L(l), Lp, dt, op->n1sign, r, rp, s)) return e;
      if (cheb) {
        if (int e = cheb_poly(pot, l, dt, lam_p[l - lmin], z, rp, ep, pwork[dt][3][l - lmin],
                              pwork[dt][4][l - lmin], s))
          return e;
        if (int e = launch_n1_transfer(N1_GRAD_ADD, L(l), Lp, dt, op->n1sign, ep, dst, s,
                                       1.0 / op->n1beta))
          return e;
      } else {
        StencilArgs a{};
        a.x = z;
        a.b = rp;
        a.out = ep;
        a.op = OP_JACOBI;
        a.mode = HG_REPLACE;
        a.mask = HG_MASK_INNER;
        a.omega = prm.omega / op->n1beta;
        if (int e = pot->launch(l, dt, a, s)) return e;
        if (int e = launch_n1_transfer(N1_GRAD_ADD, L(l), Lp, dt, op->n1sign, ep, dst, s)) return e;
      }
    }
    if (nu % 2) HG_CUDA(cudaMemcpyAsync(x, t, bytes(l, dt), cudaMemcpyDeviceToDevice, s));
    return HG_OK;
  }

  // One Chebyshev polynomial (cheb_order steps on [cheb_lo, cheb_hi] lam) of
  // operator o from x0 towards o^-1 b; the iterates alternate between `tmp`
  // and `out` so that the last lands in `out` (x0 is only read); d: the
  // direction vector.
  int cheb_poly(const Op* o, int l, int dt, double lm, const void* x0, const void* b, void* out,
                void* tmp, void* d, cudaStream_t s) {
    const double theta = 0.5 * (prm.cheb_hi + prm.cheb_lo) * lm;
    const double delta = 0.5 * (prm.cheb_hi - prm.cheb_lo) * lm;
    const double sigma = theta / delta;
    double rho = 1.0 / sigma;
    const void* cur = x0;
    for (int k = 0; k < prm.cheb_order; ++k) {
      void* nxt = ((prm.cheb_order - 1 - k) % 2 == 0) ? out : tmp;
      double a = 0.0, beta = 1.0 / theta;
      if (k > 0) {
        const double rho_new = 1.0 / (2.0 * sigma - rho);
        a = rho_new * rho;
        beta = 2.0 * rho_new / delta;
        rho = rho_new;
      }
      if (int r = cheb_op(l, dt, cur, b, nxt, d, a, beta, s, o)) return r;
      cur = nxt;
    }
    return HG_OK;
  }

  int dot(int l, int dt, const void* a, const void* b, double* out, cudaStream_t s) {
    if (int r = launch_dot(L(l), dt, a, b, HG_MASK_INNER, dot_scratch, dot_dev, s)) return r;
    HG_CUDA(cudaMemcpyAsync(dot_host, dot_dev, sizeof(double), cudaMemcpyDeviceToHost, s));
    if (int r = hier->fetch_error(s)) return r;
    HG_CUDA(cudaStreamSynchronize(s));
    *out = *dot_host;
    return hier->check_error();
  }

  int cell_op(int l, int dt, int opk, const void* x, const void* b, void* out, cudaStream_t s,
              int colour = 0) {
    StencilArgs a{};
    a.x = x;
    a.b = b;
    a.out = out;
    a.op = opk;
    a.mode = HG_REPLACE;
    a.mask = HG_MASK_INNER;
    a.omega = prm.omega;
    a.colour = colour;
    return op->launch(l, dt, a, s);
  }

  // One Chebyshev step: d = a d + beta D^-1 (b - A x), out = x + d.
  int cheb_op(int l, int dt, const void* x, const void* b, void* out, void* d, double a,
              double beta, cudaStream_t s, const Op* o = nullptr) {
    StencilArgs st{};
    st.x = x;
    st.b = b;
    st.out = out;
    st.op = OP_CHEB;
    st.mode = HG_REPLACE;
    st.mask = HG_MASK_INNER;
    st.omega = beta;
    st.dvec = d;
    st.cheb_a = a;
    return (o ? o : op)->launch(l, dt, st, s);
  }

  // Power iteration for lambda_max(D^-1 A) on level l (FP64): v = masked v0,
  // then `iters` times w = D^-1 A v / ||v||, lambda = ||w||, v = w.  The
  // normalisation rides in the step's residual weight (b = 0, beta = -1/||v||).
  int power_lambda(int l, const double* v0, int iters, double* out, cudaStream_t s,
                   bool potential = false) {
    if (int r = alloc_work(HG_F64)) return r;
    const Op* o = potential ? pot : op;
    const LevelDev& Lv = o->dev(l);
    const size_t nb = Lv.n_stored * sizeof(double);
    double* zero = (double*)(potential ? pwork[HG_F64][2][l - lmin] : W(HG_F64, WB, l));
    double* v = (double*)(potential ? pwork[HG_F64][0][l - lmin] : W(HG_F64, WX, l));
    double* w = (double*)(potential ? pwork[HG_F64][1][l - lmin] : W(HG_F64, WD, l));
    double* scratch = (double*)(potential ? pwork[HG_F64][3][l - lmin] : W(HG_F64, WT, l));
    HG_CUDA(cudaMemsetAsync(zero, 0, nb, s));
    HG_CUDA(cudaMemsetAsync(w, 0, nb, s));
    auto dotp = [&](const double* a, const double* b, double* res) {
      if (!potential) return dot(l, HG_F64, a, b, res, s);
      if (int r = launch_dot(Lv, HG_F64, a, b, HG_MASK_INNER, dot_scratch, dot_dev, s)) return r;
      HG_CUDA(cudaMemcpyAsync(dot_host, dot_dev, sizeof(double), cudaMemcpyDeviceToHost, s));
      if (int r = hier->fetch_error(s)) return r;
      HG_CUDA(cudaStreamSynchronize(s));
      *res = *dot_host;
      return hier->check_error();
    };
    // v = v0 on the non-Dirichlet DoFs, 0 elsewhere (residual of x = 0)
    {
      StencilArgs a{};
      a.x = zero;
      a.b = v0;
      a.out = v;
      a.op = OP_RESID;
      a.mode = HG_REPLACE;
      a.mask = HG_MASK_INNER;
      if (int r = o->launch(l, HG_F64, a, s)) return r;
    }
    double vv;
    if (int r = dotp(v, v, &vv)) return r;
    if (!(vv > 0.0)) {
      set_error("power iteration: start vector is zero on the non-Dirichlet DoFs");
      return HG_ERR_INVALID_ARG;
    }
    double lam_k = 0.0;
    for (int k = 0; k < iters; ++k) {
      if (int r = cheb_op(l, HG_F64, v, zero, scratch, w, 0.0, -1.0 / std::sqrt(vv), s, o))
        return r;
      if (int r = dotp(w, w, &vv)) return r;
      lam_k = std::sqrt(vv);
      if (!(vv > 0.0)) break;
      std::swap(v, w);
    }
    *out = lam_k;
    return HG_OK;
  }

  // Default start vector of the power iteration: SplitMix64 (Steele, Lea and
  // Flood 2014) of the canonical DoF index, mapped to [-1, 1).
  int estimate_lambdas(cudaStream_t s) {
    lam.assign(lmax - lmin + 1, 0.0);
    lam_p.assign(lmax - lmin + 1, 0.0);
    for (int sp = 0; sp < (is_n1() ? 2 : 1); ++sp)
    for (int l = lmin + 1; l <= lmax; ++l) {
      const bool potential = sp == 1;
      const LevelHost& H = (potential ? pot : op)->host(l);
      std::vector<double> v(H.dev.n_stored, 0.0);
      for (int64_t q = 0; q < H.dev.n_stored; ++q) {
        const int64_t u = H.canon[q];
        if (u < 0 || H.dirichlet[u]) continue;
        uint64_t z = (uint64_t)u * 0x9e3779b97f4a7c15ull + 0x9e3779b97f4a7c15ull;
        z = (z ^ (z >> 30)) * 0xbf58476d1ce4e5b9ull;
        z = (z ^ (z >> 27)) * 0x94d049bb133111ebull;
        z ^= z >> 31;
        v[q] = (double)(z >> 11) * (2.0 / 9007199254740992.0) - 1.0;
      }
      double* dv = nullptr;
      HG_CUDA(cudaMalloc(&dv, v.size() * sizeof(double)));
      cudaError_t e = cudaMemcpy(dv, v.data(), v.size() * sizeof(double), cudaMemcpyHostToDevice);
      double* dst = potential ? &lam_p[l - lmin] : &lam[l - lmin];
      int r = e == cudaSuccess ? power_lambda(l, dv, prm.cheb_iters, dst, s, potential)
                               : cuda_fail(e, "cudaMemcpy(power start vector)");
      cudaError_t e2 = cudaStreamSynchronize(s);
      cudaFree(dv);
      if (r) return r;
      HG_CUDA(e2);
    }
    return HG_OK;
  }

  // nu Chebyshev polynomials of degree cheb_order in D^-1 A on
  // [cheb_lo, cheb_hi] lambda_max (Chebyshev semi-iteration, three-term
  // recurrence of the directions); the steps ping-pong x and t.
  int smooth_cheb(int l, int dt, void* x, const void* b, int nu, cudaStream_t s) {
    void* t = W(dt, WT, l);
    void* d = W(dt, WD, l);
    const double lm = lam[l - lmin];
    const double theta = 0.5 * (prm.cheb_hi + prm.cheb_lo) * lm;
    const double delta = 0.5 * (prm.cheb_hi - prm.cheb_lo) * lm;
    const double sigma = theta / delta;
    int steps = 0;
    for (int q = 0; q < nu; ++q) {
      double rho = 1.0 / sigma;
      for (int k = 0; k < prm.cheb_order; ++k, ++steps) {
        const void* src = (steps % 2 == 0) ? x : t;
        void* dst = (steps % 2 == 0) ? t : x;
        double a = 0.0, beta = 1.0 / theta;
        if (k > 0) {
          const double rho_new = 1.0 / (2.0 * sigma - rho);
          a = rho_new * rho;
          beta = 2.0 * rho_new / delta;
          rho = rho_new;
        }
        if (int r = cheb_op(l, dt, src, b, dst, d, a, beta, s)) return r;
      }
    }
    if (steps % 2) HG_CUDA(cudaMemcpyAsync(x, t, bytes(l, dt), cudaMemcpyDeviceToDevice, s));
    return HG_OK;
  }

  // Full multigrid (nested iteration) to `level`: rhs restricted to every
  // level, exact coarsest solve, then per finer level the prolongated
  // coarser solution followed by `cycles` V-cycles.  Level-l iterates and
  // rhs below `level` live in the WX / WF work vectors, which the V-cycle on
  // level l does not touch (it uses the vectors of level l-1 and below).
  int fmg(int level, int dt, void* x, const void* b, int cycles, cudaStream_t s) {
    auto X = [&](int l) { return l == level ? x : W(dt, WX, l); };
    auto B = [&](int l) { return l == level ? b : (const void*)W(dt, WF, l); };
    for (int l = level; l > lmin; --l)
      if (int r = restrict_to(l, dt, B(l), W(dt, WF, l - 1), s)) return r;
    HG_CUDA(cudaMemsetAsync(X(lmin), 0, bytes(lmin, dt), s));
    if (int r = launch_coarse_solve(L(lmin), coarse, dt, B(lmin), X(lmin), s)) return r;
    for (int l = lmin + 1; l <= level; ++l) {
      HG_CUDA(cudaMemsetAsync(X(l), 0, bytes(l, dt), s));
      if (int r = prolong_to(l, dt, X(l - 1), X(l), s)) return r;
      for (int c = 0; c < cycles; ++c)
        if (int r2 = vcycle(l, dt, X(l), B(l), s)) return r2;
    }
    return HG_OK;
  }

  int smooth(int l, int dt, void* x, const void* b, int nu, cudaStream_t s) {
    void* t = W(dt, WT, l);
    const bool learn = learned_active && dt == HG_F32 && l == lmax;
    if (is_n1()) return smooth_hiptmair(l, dt, x, b, nu, s);
    if (prm.smoother == HG_SMOOTH_CHEB && !learn) return smooth_cheb(l, dt, x, b, nu, s);
    if (prm.smoother == HG_SMOOTH_GS && !learn) {
      // nu 4-colour sweeps; 4 nu sub-sweeps ping-pong x and t and end in x
      for (int q = 0; q < nu; ++q)
        for (int c = 0; c < 4; ++c) {
          const void* src = (c % 2 == 0) ? x : t;
          void* dst = (c % 2 == 0) ? t : x;
          if (int r = cell_op(l, dt, OP_GS, src, b, dst, s, c)) return r;
        }
      return HG_OK;
    }
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
    if (int r = restrict_to(l, dt, res, bc, s)) return r;
    HG_CUDA(cudaMemsetAsync(xc, 0, bytes(l - 1, dt), s));
    if (int r = vcycle(l - 1, dt, xc, bc, s)) return r;
    if (int r = prolong_to(l, dt, xc, x, s)) return r;
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
  const LevelHost& H = op->host(lmin);
  const LevelDev& Lc = H.dev;
  if (!hier->mesh->grid_denom) {
    set_error("the coarse solver needs vertex coordinates on an exact lattice");
    return HG_ERR_UNSUPPORTED;
  }
  std::vector<int32_t> int_of_canon(Lc.n_unique, -1);
  std::vector<int64_t> rep;
  // N1: only the edge points (an odd lattice coordinate) are unknowns
  std::vector<uint8_t> edge_pt;
  if (is_n1()) {
    edge_pt.assign(Lc.cell_stride, 0);
    for (int k = 0; k <= Lc.n; ++k)
      for (int j = 0; j + k <= Lc.n; ++j)
        for (int i = 0; i + j + k <= Lc.n; ++i) edge_pt[tw(Lc.w, i, j, k)] = ((i | j | k) & 1) ? 1 : 0;
  }
  for (int64_t u = 0; u < Lc.n_unique; ++u)
    if (!H.dirichlet[u] && (edge_pt.empty() || edge_pt[H.canon_rep[u] % Lc.cell_stride])) {
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
  for (auto& per_dt : pwork)
    for (auto& per_kind : per_dt)
      for (void* p : per_kind) cudaFree(p);
  delete pot;
}

}  // namespace hg

using namespace hg;

struct hg_gmg : Gmg {};
struct hg_func : Func {};
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
  p->smoother = HG_SMOOTH_JACOBI;
  p->cheb_order = 2;
  p->cheb_iters = 20;
  p->cheb_lo = 0.1;
  p->cheb_hi = 1.1;
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
  g->lmax = op->lmax;
  g->lmin = g->prm.lmin < 0 ? op->lmin : g->prm.lmin;
  if (g->lmin < op->lmin || g->lmin > op->lmax) {
    set_error("coarsest level %d outside the operator's levels %d..%d", g->lmin, op->lmin,
              op->lmax);
    return HG_ERR_LEVEL_RANGE;
  }
  if (op->kind == HG_OP_N1_CURLCURL && g->prm.smoother == HG_SMOOTH_GS) {
    set_error("Nedelec multigrid: Hiptmair smoothing with weighted Jacobi or Chebyshev only");
    return HG_ERR_UNSUPPORTED;
  }
  if (op->kind == HG_OP_N1_CURLCURL && g->prm.smoother == HG_SMOOTH_JACOBI &&
      !(g->prm.omega > 0.0 && g->prm.omega <= 0.6)) {
    // lambda_max(D^-1 A) of the edge matrices exceeds 3: larger weights diverge
    set_error("Nedelec multigrid: Jacobi weight %g outside (0, 0.6]", g->prm.omega);
    return HG_ERR_INVALID_ARG;
  }
  if (g->prm.smoother != HG_SMOOTH_JACOBI && g->prm.smoother != HG_SMOOTH_GS &&
      g->prm.smoother != HG_SMOOTH_CHEB) {
    set_error("unknown smoother %d", g->prm.smoother);
    return HG_ERR_INVALID_ARG;
  }
  if (g->prm.smoother == HG_SMOOTH_GS) {
    if (op->space != HG_SPACE_P1) {
      set_error("Gauss-Seidel smoothing: P1 operators only");
      return HG_ERR_UNSUPPORTED;
    }
    for (int l = g->lmin; l <= g->lmax; ++l)
      if (!g->L(l).colour) {
        set_error("Gauss-Seidel smoothing: this mesh admits no 4-colouring of the lattice");
        return HG_ERR_UNSUPPORTED;
      }
  }
  if (g->prm.nu1 < 0 || g->prm.nu2 < 0 || !(g->prm.omega > 0.0)) {
    set_error("bad smoother parameters nu1=%d nu2=%d omega=%g", g->prm.nu1, g->prm.nu2,
              g->prm.omega);
    return HG_ERR_INVALID_ARG;
  }
  if (g->prm.smoother == HG_SMOOTH_CHEB &&
      (g->prm.cheb_order < 1 || g->prm.cheb_order > 64 || g->prm.cheb_iters < 1 ||
       g->prm.cheb_iters > 10000 || !(g->prm.cheb_lo > 0.0) ||
       !(g->prm.cheb_hi > g->prm.cheb_lo))) {
    set_error("bad Chebyshev parameters order=%d iters=%d interval [%g, %g]", g->prm.cheb_order,
              g->prm.cheb_iters, g->prm.cheb_lo, g->prm.cheb_hi);
    return HG_ERR_INVALID_ARG;
  }
  if (op->kind == HG_OP_N1_CURLCURL) {
    g->pot = new Op();
    if (int r = g->pot->build(g->hier, HG_OP_P1_LAPLACE, nullptr)) return r;
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
  if (g->prm.smoother == HG_SMOOTH_CHEB) {
    if (int r = g->estimate_lambdas(0)) return r;
  } else {
    g->lam.assign(g->lmax - g->lmin + 1, 0.0);
    g->lam_p.assign(g->lmax - g->lmin + 1, 0.0);
  }
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

int hg_solve_function(hg_gmg* g, int precision, hg_func* x, const hg_func* b, double rel_tol,
                      int max_iter, int* iters, double* rel_res, void* stream) {
  if (!g || !x || !b || x == b) {
    set_error("hg_solve_function: null or identical functions");
    return HG_ERR_INVALID_ARG;
  }
  if (x->hier != g->hier || b->hier != g->hier || x->space != g->op->space ||
      b->space != g->op->space || x->dtype != HG_F64 || b->dtype != HG_F64) {
    set_error("hg_solve_function: x and b must be FP64 functions of the operator's space");
    return HG_ERR_INVALID_ARG;
  }
  void* xp = x->data(g->lmax);
  const void* bp = b->data(g->lmax);
  if (!xp || !bp) return HG_ERR_INVALID_ARG;
  return hg_solve(g, precision, (double*)xp, (const double*)bp, rel_tol, max_iter, iters, rel_res,
                  stream);
}

int hg_gmg_set_learned(hg_gmg* g, const hg_mlp* mlp) {
  if (!g) {
    set_error("hg_gmg_set_learned: null handle");
    return HG_ERR_INVALID_ARG;
  }
  if (mlp && (g->op->space != HG_SPACE_P1 || g->op->vinv[HG_F32].empty())) {
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

static int smoothed_level(const hg_gmg* g, int level, const char* fn) {
  if (!g) {
    set_error("%s: null handle", fn);
    return HG_ERR_INVALID_ARG;
  }
  if (level <= g->lmin || level > g->lmax) {
    set_error("%s: level %d outside the smoothed levels %d..%d", fn, level, g->lmin + 1, g->lmax);
    return HG_ERR_LEVEL_RANGE;
  }
  return HG_OK;
}

int hg_gmg_lambda(const hg_gmg* g, int level, double* lam) {
  if (int r = smoothed_level(g, level, "hg_gmg_lambda")) return r;
  if (!lam) {
    set_error("hg_gmg_lambda: null output");
    return HG_ERR_INVALID_ARG;
  }
  *lam = g->lam[level - g->lmin];
  return HG_OK;
}

int hg_gmg_set_lambda(hg_gmg* g, int level, double lam) {
  if (int r = smoothed_level(g, level, "hg_gmg_set_lambda")) return r;
  if (!(lam > 0.0) || !std::isfinite(lam)) {
    set_error("hg_gmg_set_lambda: lambda %g must be positive and finite", lam);
    return HG_ERR_INVALID_ARG;
  }
  g->lam[level - g->lmin] = lam;
  return HG_OK;
}

int hg_gmg_potential_lambda(const hg_gmg* g, int level, double* lam) {
  if (int r = smoothed_level(g, level, "hg_gmg_potential_lambda")) return r;
  if (!lam || !g->pot) {
    set_error("hg_gmg_potential_lambda: null output or not a Nedelec multigrid");
    return HG_ERR_INVALID_ARG;
  }
  *lam = g->lam_p[level - g->lmin];
  return HG_OK;
}

int hg_gmg_set_potential_lambda(hg_gmg* g, int level, double lam) {
  if (int r = smoothed_level(g, level, "hg_gmg_set_potential_lambda")) return r;
  if (!g->pot || !(lam > 0.0) || !std::isfinite(lam)) {
    set_error("hg_gmg_set_potential_lambda: not a Nedelec multigrid, or lambda %g not positive "
              "and finite", lam);
    return HG_ERR_INVALID_ARG;
  }
  g->lam_p[level - g->lmin] = lam;
  return HG_OK;
}

int hg_gmg_power_lambda(hg_gmg* g, int level, const double* v0, int iters, double* lam,
                        void* stream) {
  if (int r = smoothed_level(g, level, "hg_gmg_power_lambda")) return r;
  if (!v0 || !lam || iters < 1 || iters > 10000) {
    set_error("hg_gmg_power_lambda: bad argument");
    return HG_ERR_INVALID_ARG;
  }
  return g->power_lambda(level, v0, iters, lam, (cudaStream_t)stream);
}

int hg_fmg(hg_gmg* g, int level, int dtype, void* x, const void* b, int cycles, void* stream) {
  if (!g || !x || !b || x == b || cycles < 0) {
    set_error("hg_fmg: bad argument");
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
  return g->fmg(level, dtype, x, b, cycles, (cudaStream_t)stream);
}

}  // extern "C"

// ======================================================= batched solves
// Many independent problems (each with its own hierarchy/operator/GMG) are
// solved together: every stage of the FP32 V-cycle (a smoothing sweep, the
// residual, a restriction, the coarse solves, a prolongation) and every step
// of the FP64 refinement loop is ONE persistent launch over the work units of
// all problems that take part in it.  V-cycles of problems with different
// depths are aligned by the distance from their finest level.  The stage
// sequence is captured once as two CUDA graphs (residual + norms, correction)
// and replayed; an autotuner picks the plane-window prefetch depth and the
// persistent grid size of the cell stages.
namespace hg {

namespace {

enum StageKind { ST_CELL, ST_RESTRICT, ST_PROLONG, ST_EW, ST_DOT, ST_COARSE };

struct Stage {
  int kind = 0, dtype = 0, op = 0, nprob = 0;
  void* descs = nullptr;
  int* base = nullptr;
  int* base2 = nullptr;
  double* scratch = nullptr;  // per-unit partials of a dot stage
  int units = 0, units2 = 0;
};

struct Batch {
  std::vector<Gmg*> P;
  std::vector<double*> x;
  std::vector<const double*> b;
  std::vector<Stage> init, g1, g2;
  double *rr = nullptr, *rs = nullptr, *nb = nullptr;
  double *rr_host = nullptr, *rs_host = nullptr;
  std::vector<double> nbh;
  double tune_us = 0.0;
  int rows = 1, gfac = 2, sms = 152;
  cudaStream_t cs = nullptr;
  cudaGraphExec_t e1 = nullptr, e2 = nullptr;

  ~Batch() {
    for (auto* L : {&init, &g1, &g2})
      for (Stage& s : *L) {
        cudaFree(s.descs);
        cudaFree(s.base);
        cudaFree(s.base2);
        cudaFree(s.scratch);
      }
    cudaFree(rr);
    cudaFree(rs);
    cudaFree(nb);
    if (rr_host) cudaFreeHost(rr_host);
    if (rs_host) cudaFreeHost(rs_host);
    if (e1) cudaGraphExecDestroy(e1);
    if (e2) cudaGraphExecDestroy(e2);
    if (cs) cudaStreamDestroy(cs);
  }

  int grid() const { return gfac * sms * 4; }

  int finish(Stage& st, const std::vector<char>& host, const std::vector<int>& base,
             const std::vector<int>* base2 = nullptr) {
    st.nprob = (int)base.size() - 1;
    st.units = base.back();
    HG_CUDA(cudaMalloc(&st.descs, std::max<size_t>(host.size(), 16)));
    if (!host.empty()) HG_CUDA(cudaMemcpy(st.descs, host.data(), host.size(), cudaMemcpyHostToDevice));
    HG_CUDA(cudaMalloc(&st.base, base.size() * sizeof(int)));
    HG_CUDA(cudaMemcpy(st.base, base.data(), base.size() * sizeof(int), cudaMemcpyHostToDevice));
    if (base2) {
      st.units2 = base2->back();
      HG_CUDA(cudaMalloc(&st.base2, base2->size() * sizeof(int)));
      HG_CUDA(cudaMemcpy(st.base2, base2->data(), base2->size() * sizeof(int),
                         cudaMemcpyHostToDevice));
    }
    return HG_OK;
  }

  struct CellItem {
    int p, l;
    const void *x, *b;
    void* out;
  };
  int add_cell(std::vector<Stage>& L, int dt, int op, const std::vector<CellItem>& items) {
    if (items.empty()) return HG_OK;
    Stage st;
    st.kind = ST_CELL;
    st.dtype = dt;
    st.op = op;
    const size_t sz = p1_desc_bytes(dt);
    std::vector<char> host(sz * items.size());
    std::vector<int> base(1, 0);
    for (size_t q = 0; q < items.size(); ++q) {
      const Gmg* G = P[items[q].p];
      StencilArgs a{};
      a.x = items[q].x;
      a.b = items[q].b;
      a.out = items[q].out;
      a.op = op;
      a.mode = HG_REPLACE;
      a.mask = HG_MASK_INNER;
      a.omega = G->prm.omega;
      const int li = items[q].l - G->hier->lmin;
      a.sten = dt == HG_F64 ? (const void*)G->op->sten64[li] : (const void*)G->op->sten32[li];
      int u = 0;
      p1_make_desc(G->L(items[q].l), dt, a, host.data() + q * sz, &u);
      base.push_back(base.back() + u);
    }
    if (int r = finish(st, host, base)) return r;
    L.push_back(st);
    return HG_OK;
  }

  struct XferItem {
    int p, lf;
    const void* src;
    void* dst;
  };
  int add_xfer(std::vector<Stage>& L, int kind, int dt, const std::vector<XferItem>& items) {
    if (items.empty()) return HG_OK;
    Stage st;
    st.kind = kind;
    st.dtype = dt;
    const size_t sz = kind == ST_RESTRICT ? restrict_desc_bytes(dt) : prolong_desc_bytes(dt);
    std::vector<char> host(sz * items.size());
    std::vector<int> base(1, 0);
    for (size_t q = 0; q < items.size(); ++q) {
      const Gmg* G = P[items[q].p];
      const LevelDev& F = G->L(items[q].lf);
      const LevelDev& C = G->L(items[q].lf - 1);
      int u = 0;
      if (kind == ST_RESTRICT)
        restrict_make_desc(F, C, dt, items[q].src, items[q].dst, host.data() + q * sz, &u);
      else
        prolong_make_desc(F, C, dt, items[q].src, items[q].dst, host.data() + q * sz, &u);
      base.push_back(base.back() + u);
    }
    if (int r = finish(st, host, base)) return r;
    L.push_back(st);
    return HG_OK;
  }

  int add_ew(std::vector<Stage>& L, int op, const std::vector<EwDesc>& d) {
    if (d.empty()) return HG_OK;
    Stage st;
    st.kind = ST_EW;
    st.op = op;
    std::vector<char> host(sizeof(EwDesc) * d.size());
    memcpy(host.data(), d.data(), host.size());
    std::vector<int> base(1, 0);
    for (const EwDesc& e : d) base.push_back(base.back() + (int)ew_units(e.n));
    if (int r = finish(st, host, base)) return r;
    L.push_back(st);
    return HG_OK;
  }

  int add_dot(std::vector<Stage>& L, int dt, const std::vector<DotDesc>& d) {
    Stage st;
    st.kind = ST_DOT;
    st.dtype = dt;
    std::vector<char> host(sizeof(DotDesc) * d.size());
    memcpy(host.data(), d.data(), host.size());
    std::vector<int> base(1, 0);
    for (const DotDesc& e : d) base.push_back(base.back() + (int)dot_units(e.n_rows));
    if (int r = finish(st, host, base)) return r;
    HG_CUDA(cudaMalloc(&st.scratch, std::max(st.units, 1) * sizeof(double)));
    L.push_back(st);
    return HG_OK;
  }

  int add_coarse(std::vector<Stage>& L, const std::vector<CoarseBDesc>& d) {
    Stage st;
    st.kind = ST_COARSE;
    st.dtype = HG_F32;
    std::vector<char> host(sizeof(CoarseBDesc) * d.size());
    memcpy(host.data(), d.data(), host.size());
    std::vector<int> b1(1, 0), b2(1, 0);
    for (const CoarseBDesc& c : d) {
      b1.push_back(b1.back() + (int)coarse_units_mv(c.nint));
      b2.push_back(b2.back() + (int)coarse_units_sc(c.n_stored));
    }
    if (int r = finish(st, host, b1, &b2)) return r;
    L.push_back(st);
    return HG_OK;
  }

  int run(const Stage& st, cudaStream_t s, double* rr_out) const {
    switch (st.kind) {
      case ST_CELL:
        return launch_p1_batched(st.dtype, st.op, rows, st.descs, st.base, st.nprob,
                                 std::min(grid(), std::max(st.units, 1)), s);
      case ST_RESTRICT:
        return launch_restrict_batched(st.dtype, st.descs, st.base, st.nprob,
                                       std::min(grid(), std::max(st.units, 1)), s);
      case ST_PROLONG:
        return launch_prolong_batched(st.dtype, st.descs, st.base, st.nprob,
                                      std::min(grid(), std::max(st.units, 1)), s);
      case ST_EW:
        return launch_batched_ew(st.op, (const EwDesc*)st.descs, st.base, st.nprob,
                                 std::min(sms * 8, std::max(st.units, 1)), s);
      case ST_DOT:
        return launch_batched_dot(st.dtype, (const DotDesc*)st.descs, st.base, st.nprob,
                                  std::min(sms * 8, std::max(st.units, 1)), st.scratch, rr_out, s);
      case ST_COARSE:
        return launch_batched_coarse(st.dtype, (const CoarseBDesc*)st.descs, st.base, st.base2,
                                     st.nprob,
                                     std::min(sms * 8, std::max(std::max(st.units, st.units2), 1)),
                                     s);
    }
    return HG_OK;
  }

  int run_list(const std::vector<Stage>& L, cudaStream_t s, double* rr_out) const {
    for (const Stage& st : L)
      if (int r = run(st, s, rr_out)) return r;
    return HG_OK;
  }

  int build();
  int capture(const std::vector<Stage>& L, double* rr_out, cudaGraphExec_t* out);
  int autotune(double* best_us);
};

DotDesc dot_desc(const LevelDev& L, const void* x, const void* y) {
  DotDesc d;
  d.n = L.n;
  d.stride = L.cell_stride;
  d.flags = L.cls_flags;
  d.n_rows = L.ncells * ntri32(L.w);
  d.x = x;
  d.y = y;
  return d;
}

int Batch::build() {
  const int np = (int)P.size();
  HG_CUDA(cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, 0));
  HG_CUDA(cudaMalloc(&rr, np * sizeof(double)));
  HG_CUDA(cudaMalloc(&rs, np * sizeof(double)));
  HG_CUDA(cudaMemset(rs, 0, np * sizeof(double)));
  HG_CUDA(cudaMallocHost(&rs_host, np * sizeof(double)));
  HG_CUDA(cudaMalloc(&nb, np * sizeof(double)));
  HG_CUDA(cudaMallocHost(&rr_host, np * sizeof(double)));
  for (Gmg* G : P)
    if (int r = G->alloc_work(HG_F32)) return r;
  // init: x = 0, |b|^2 -> nb
  {
    std::vector<EwDesc> z;
    std::vector<DotDesc> d;
    for (int p = 0; p < np; ++p) {
      const LevelDev& L = P[p]->L(P[p]->lmax);
      z.push_back({L.n_stored, x[p], nullptr, nullptr, HG_F64});
      d.push_back(dot_desc(L, b[p], b[p]));
    }
    if (int r = add_ew(init, EW_ZERO, z)) return r;
    if (int r = add_dot(init, HG_F64, d)) return r;
  }
  // g1: r64 = b - A x (FP64), |r64|^2 -> rr
  {
    std::vector<CellItem> c;
    std::vector<DotDesc> d;
    for (int p = 0; p < np; ++p) {
      c.push_back({p, P[p]->lmax, x[p], b[p], P[p]->r64});
      d.push_back(dot_desc(P[p]->L(P[p]->lmax), P[p]->r64, P[p]->r64));
    }
    if (int r = add_cell(g1, HG_F64, OP_RESID, c)) return r;
    if (int r = add_dot(g1, HG_F64, d)) return r;
  }
  // g2: b32 = r64/|r|, d32 = 0, FP32 V-cycle(s) on (d32, b32), x += |r| d32,
  // with |r|^2 taken from rs (zero for a problem that has converged, which
  // then keeps its iterate unchanged)
  {
    std::vector<EwDesc> dm, zd, pr;
    for (int p = 0; p < np; ++p) {
      const int64_t n = P[p]->L(P[p]->lmax).n_stored;
      dm.push_back({n, P[p]->b32, P[p]->r64, rs + p, HG_F32});
      zd.push_back({n, P[p]->d32, nullptr, nullptr, HG_F32});
      pr.push_back({n, x[p], P[p]->d32, rs + p, HG_F64});
    }
    if (int r = add_ew(g2, EW_DEMOTE, dm)) return r;
    if (int r = add_ew(g2, EW_ZERO, zd)) return r;
    const int nu1 = P[0]->prm.nu1, nu2 = P[0]->prm.nu2;
    int dmax = 0;
    for (Gmg* G : P) dmax = std::max(dmax, G->lmax - G->lmin);
    auto X = [&](int p, int d) -> void* {
      return d == 0 ? (void*)P[p]->d32 : P[p]->W(HG_F32, Gmg::WX, P[p]->lmax - d);
    };
    auto B = [&](int p, int d) -> void* {
      return d == 0 ? (void*)P[p]->b32 : P[p]->W(HG_F32, Gmg::WB, P[p]->lmax - d);
    };
    auto smooth = [&](int d, int nu) -> int {
      for (int q = 0; q < nu; ++q) {
        std::vector<CellItem> c;
        for (int p = 0; p < np; ++p) {
          if (d >= P[p]->lmax - P[p]->lmin) continue;
          const int l = P[p]->lmax - d;
          void* t = P[p]->W(HG_F32, Gmg::WT, l);
          c.push_back({p, l, q % 2 == 0 ? X(p, d) : t, B(p, d), q % 2 == 0 ? t : X(p, d)});
        }
        if (int r = add_cell(g2, HG_F32, OP_JACOBI, c)) return r;
      }
      if (nu % 2) {
        std::vector<EwDesc> cp;
        for (int p = 0; p < np; ++p) {
          if (d >= P[p]->lmax - P[p]->lmin) continue;
          const int l = P[p]->lmax - d;
          cp.push_back({P[p]->L(l).n_stored, X(p, d), P[p]->W(HG_F32, Gmg::WT, l), nullptr, HG_F32});
        }
        if (int r = add_ew(g2, EW_COPY, cp)) return r;
      }
      return HG_OK;
    };
    for (int cyc = 0; cyc < std::max(P[0]->prm.inner_cycles, 1); ++cyc) {
    for (int d = 0; d < dmax; ++d) {
      if (int r = smooth(d, nu1)) return r;
      std::vector<CellItem> res;
      std::vector<XferItem> rs;
      std::vector<EwDesc> zc;
      for (int p = 0; p < np; ++p) {
        if (d >= P[p]->lmax - P[p]->lmin) continue;
        const int l = P[p]->lmax - d;
        void* rv = P[p]->W(HG_F32, Gmg::WR, l);
        res.push_back({p, l, X(p, d), B(p, d), rv});
        rs.push_back({p, l, rv, B(p, d + 1)});
        zc.push_back({P[p]->L(l - 1).n_stored, X(p, d + 1), nullptr, nullptr, HG_F32});
      }
      if (int r = add_cell(g2, HG_F32, OP_RESID, res)) return r;
      if (int r = add_xfer(g2, ST_RESTRICT, HG_F32, rs)) return r;
      if (int r = add_ew(g2, EW_ZERO, zc)) return r;
    }
    std::vector<CoarseBDesc> co;
    for (int p = 0; p < np; ++p) {
      const Gmg* G = P[p];
      const int d = G->lmax - G->lmin;
      const LevelDev& L = G->L(G->lmin);
      co.push_back({G->coarse.n, G->coarse.ainv, G->coarse.stored_rep, B(p, d), G->coarse.xint,
                    L.n_stored, L.canon, G->coarse.int_of_canon, X(p, d)});
    }
    if (int r = add_coarse(g2, co)) return r;
    for (int d = dmax - 1; d >= 0; --d) {
      std::vector<XferItem> pl;
      for (int p = 0; p < np; ++p) {
        if (d >= P[p]->lmax - P[p]->lmin) continue;
        pl.push_back({p, P[p]->lmax - d, X(p, d + 1), X(p, d)});
      }
      if (int r = add_xfer(g2, ST_PROLONG, HG_F32, pl)) return r;
      if (int r = smooth(d, nu2)) return r;
    }
    }
    if (int r = add_ew(g2, EW_PROMOTE, pr)) return r;
  }
  HG_CUDA(cudaStreamCreateWithFlags(&cs, cudaStreamNonBlocking));
  return HG_OK;
}

int Batch::capture(const std::vector<Stage>& L, double* rr_out, cudaGraphExec_t* out) {
  if (*out) {
    cudaGraphExecDestroy(*out);
    *out = nullptr;
  }
  cudaGraph_t g = nullptr;
  HG_CUDA(cudaStreamBeginCapture(cs, cudaStreamCaptureModeThreadLocal));
  const int r = run_list(L, cs, rr_out);
  const cudaError_t e = cudaStreamEndCapture(cs, &g);
  if (r) {
    if (g) cudaGraphDestroy(g);
    return r;
  }
  if (e != cudaSuccess) return cuda_fail(e, "cudaStreamEndCapture");
  const cudaError_t ei = cudaGraphInstantiate(out, g, 0);
  cudaGraphDestroy(g);
  if (ei != cudaSuccess) return cuda_fail(ei, "cudaGraphInstantiate");
  return HG_OK;
}

// Time the first finest-level smoothing stage for each (rows, grid factor).
int Batch::autotune(double* best_us) {
  const Stage* st = nullptr;
  for (const Stage& s : g2)
    if (s.kind == ST_CELL) {
      st = &s;
      break;
    }
  if (!st) return HG_OK;
  cudaEvent_t a, z;
  HG_CUDA(cudaEventCreate(&a));
  HG_CUDA(cudaEventCreate(&z));
  double best = 1e30;
  int br = rows, bg = gfac;
  for (int R : {0, 1, 2})
    for (int gf : {1, 2, 4}) {
      rows = R;
      gfac = gf;
      if (int r = run(*st, cs, rr)) return r;  // warm-up
      HG_CUDA(cudaEventRecord(a, cs));
      for (int q = 0; q < 3; ++q)
        if (int r = run(*st, cs, rr)) return r;
      HG_CUDA(cudaEventRecord(z, cs));
      HG_CUDA(cudaEventSynchronize(z));
      float ms = 0.f;
      HG_CUDA(cudaEventElapsedTime(&ms, a, z));
      if (ms / 3 < best) {
        best = ms / 3;
        br = R;
        bg = gf;
      }
    }
  rows = br;
  gfac = bg;
  cudaEventDestroy(a);
  cudaEventDestroy(z);
  if (best_us) *best_us = best * 1e3;
  return HG_OK;
}

}  // namespace
}  // namespace hg

struct hg_batch : hg::Batch {};

extern "C" {

int hg_gmg_clone(const hg_gmg* src, hg_gmg** out) {
  if (!src || !out) {
    set_error("hg_gmg_clone: null argument");
    return HG_ERR_INVALID_ARG;
  }
  auto g = std::make_unique<hg_gmg>();
  g->op = src->op;
  g->hier = src->hier;
  g->prm = src->prm;
  g->lmin = src->lmin;
  g->lmax = src->lmax;
  g->learned = src->learned;
  g->lam = src->lam;
  if (src->pot) {
    g->pot = new Op();
    if (int r = g->pot->build(g->hier, HG_OP_P1_LAPLACE, nullptr)) return r;
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
  // coarse solver: copies of the source's tables
  g->coarse.n = src->coarse.n;
  const LevelDev& Lc = g->L(g->lmin);
  HG_CUDA(cudaMalloc(&g->coarse.int_of_canon, std::max<int64_t>(Lc.n_unique, 1) * sizeof(int32_t)));
  HG_CUDA(cudaMemcpy(g->coarse.int_of_canon, src->coarse.int_of_canon,
                     Lc.n_unique * sizeof(int32_t), cudaMemcpyDeviceToDevice));
  const int n = src->coarse.n;
  if (n > 0) {
    HG_CUDA(cudaMalloc(&g->coarse.stored_rep, n * sizeof(int64_t)));
    HG_CUDA(cudaMalloc(&g->coarse.xint, n * sizeof(double)));
    HG_CUDA(cudaMalloc(&g->coarse.ainv, (size_t)n * n * sizeof(double)));
    HG_CUDA(cudaMemcpy(g->coarse.stored_rep, src->coarse.stored_rep, n * sizeof(int64_t),
                       cudaMemcpyDeviceToDevice));
    HG_CUDA(cudaMemcpy(g->coarse.ainv, src->coarse.ainv, (size_t)n * n * sizeof(double),
                       cudaMemcpyDeviceToDevice));
  }
  *out = g.release();
  return HG_OK;
}

int hg_batch_create(hg_gmg* const* problems, int count, double* const* x, const double* const* b,
                    int flags, hg_batch** out) {
  if (!problems || !x || !b || count < 1 || !out) {
    set_error("hg_batch_create: bad argument");
    return HG_ERR_INVALID_ARG;
  }
  auto B = std::make_unique<hg_batch>();
  for (int p = 0; p < count; ++p) {
    Gmg* G = problems[p];
    if (!G || !x[p] || !b[p] || (const void*)x[p] == (const void*)b[p]) {
      set_error("hg_batch_create: null problem or vector %d", p);
      return HG_ERR_INVALID_ARG;
    }
    if (G->op->kind != HG_OP_P1_LAPLACE && G->op->kind != HG_OP_P1_MASS) {
      set_error("hg_batch_create: problem %d: batched solves take constant-stencil operators", p);
      return HG_ERR_UNSUPPORTED;
    }
    if (G->prm.smoother != HG_SMOOTH_JACOBI) {
      set_error("hg_batch_create: problem %d: batched solves smooth with weighted Jacobi", p);
      return HG_ERR_UNSUPPORTED;
    }
    if (G->prm.nu1 != problems[0]->prm.nu1 || G->prm.nu2 != problems[0]->prm.nu2 ||
        G->prm.inner_cycles != problems[0]->prm.inner_cycles) {
      set_error("hg_batch_create: all problems need the same nu1/nu2/inner_cycles");
      return HG_ERR_INVALID_ARG;
    }
    B->P.push_back(G);
    B->x.push_back(x[p]);
    B->b.push_back(b[p]);
  }
  {
    std::vector<Gmg*> sorted(B->P);
    std::sort(sorted.begin(), sorted.end());
    if (std::adjacent_find(sorted.begin(), sorted.end()) != sorted.end()) {
      set_error("hg_batch_create: a problem appears twice (each needs its own work vectors)");
      return HG_ERR_INVALID_ARG;
    }
  }
  if (int r = B->build()) return r;
  if (flags & HG_BATCH_AUTOTUNE) {
    if (int r = B->autotune(&B->tune_us)) return r;
  }
  if (flags & HG_BATCH_GRAPH) {
    if (int r = B->capture(B->g1, B->rr, &B->e1)) return r;
    if (int r = B->capture(B->g2, B->rr, &B->e2)) return r;
  }
  HG_CUDA(cudaStreamSynchronize(B->cs));
  *out = B.release();
  return HG_OK;
}

void hg_batch_destroy(hg_batch* B) { delete B; }

int hg_batch_tuning(const hg_batch* B, int* rows, int* grid_factor, double* stage_us) {
  if (!B) {
    set_error("hg_batch_tuning: null handle");
    return HG_ERR_INVALID_ARG;
  }
  if (rows) *rows = B->rows;
  if (grid_factor) *grid_factor = B->gfac;
  if (stage_us) *stage_us = B->tune_us;
  return HG_OK;
}

int hg_batch_solve(hg_batch* B, double rel_tol, int max_iter, int* iters, double* rel_res,
                   void* stream) {
  if (!B || max_iter < 0 || !iters || !rel_res) {
    set_error("hg_batch_solve: bad argument");
    return HG_ERR_INVALID_ARG;
  }
  const int count = (int)B->P.size();
  cudaStream_t us = (cudaStream_t)stream;
  // the work runs on the batch's own stream, ordered after the caller's stream
  cudaEvent_t ev;
  HG_CUDA(cudaEventCreateWithFlags(&ev, cudaEventDisableTiming));
  HG_CUDA(cudaEventRecord(ev, us));
  HG_CUDA(cudaStreamWaitEvent(B->cs, ev, 0));
  const bool graph = B->e1 != nullptr;
  int rc = HG_OK;
  bool all = false;
  B->nbh.assign(count, 0.0);
  if ((rc = B->run_list(B->init, B->cs, B->nb))) goto done;
  if (cudaMemcpyAsync(B->rr_host, B->nb, count * sizeof(double), cudaMemcpyDeviceToHost, B->cs) !=
          cudaSuccess ||
      cudaStreamSynchronize(B->cs) != cudaSuccess) {
    rc = cuda_fail(cudaGetLastError(), "hg_batch_solve: norm of b");
    goto done;
  }
  for (int p = 0; p < count; ++p) {
    B->nbh[p] = std::sqrt(B->rr_host[p]);
    iters[p] = -1;
    rel_res[p] = 1.0;
  }
  for (int it = 0; it <= max_iter; ++it) {
    if (graph) {
      if (cudaGraphLaunch(B->e1, B->cs) != cudaSuccess) {
        rc = cuda_fail(cudaGetLastError(), "cudaGraphLaunch");
        goto done;
      }
    } else if ((rc = B->run_list(B->g1, B->cs, B->rr))) {
      goto done;
    }
    if (cudaMemcpyAsync(B->rr_host, B->rr, count * sizeof(double), cudaMemcpyDeviceToHost,
                        B->cs) != cudaSuccess ||
        cudaStreamSynchronize(B->cs) != cudaSuccess) {
      rc = cuda_fail(cudaGetLastError(), "hg_batch_solve: residual norms");
      goto done;
    }
    all = true;
    for (int p = 0; p < count; ++p) {
      const double rel = B->nbh[p] > 0 ? std::sqrt(B->rr_host[p]) / B->nbh[p] : 0.0;
      if (iters[p] < 0) {
        rel_res[p] = rel;
        if (rel <= rel_tol) iters[p] = it;
      }
      // a converged problem gets a zero correction from here on
      B->rs_host[p] = iters[p] < 0 ? B->rr_host[p] : 0.0;
      if (iters[p] < 0) all = false;
    }
    if (all || it == max_iter) break;
    if (cudaMemcpyAsync(B->rs, B->rs_host, count * sizeof(double), cudaMemcpyHostToDevice,
                        B->cs) != cudaSuccess) {
      rc = cuda_fail(cudaGetLastError(), "hg_batch_solve: scales");
      goto done;
    }
    if (graph) {
      if (cudaGraphLaunch(B->e2, B->cs) != cudaSuccess) {
        rc = cuda_fail(cudaGetLastError(), "cudaGraphLaunch");
        goto done;
      }
    } else if ((rc = B->run_list(B->g2, B->cs, B->rr))) {
      goto done;
    }
  }
  for (int p = 0; p < count; ++p)
    if (iters[p] < 0) iters[p] = max_iter;
done:
  cudaEventRecord(ev, B->cs);
  cudaStreamWaitEvent(us, ev, 0);
  cudaStreamSynchronize(B->cs);
  cudaEventDestroy(ev);
  if (rc) return rc;
  {
    std::vector<const Hier*> hs;
    for (Gmg* G : B->P)
      if (std::find(hs.begin(), hs.end(), G->hier) == hs.end()) hs.push_back(G->hier);
    for (const Hier* h : hs) {
      if (int r = h->fetch_error(B->cs)) return r;
      HG_CUDA(cudaStreamSynchronize(B->cs));
      if (int r = h->check_error()) return r;
    }
  }
  if (!all) {
    set_error("hg_batch_solve: not all problems reached %.1e in %d iterations", rel_tol, max_iter);
    return HG_ERR_NOT_CONVERGED;
  }
  return HG_OK;
}

}  // extern "C"
