// Host set-up of the element-wise P2 operators: per macro cell and P2 level
// the element data of the six micro-cell types (Sec. 3.2) and the quadrature
// rule (Sec. 5.2, element matrices by quadrature), the anchors of the eight
// colour phases, and the inverse assembled diagonal for Jacobi smoothing.
#include <cuda_runtime.h>

#include <cmath>
#include <cstring>
#include <vector>

#include "hg_host.h"

namespace hg {

namespace {

const int kTypeOffP2[6][4][3] = {
    {{0, 0, 0}, {1, 0, 0}, {0, 1, 0}, {0, 0, 1}},
    {{1, 1, 0}, {1, 0, 1}, {0, 1, 1}, {1, 1, 1}},
    {{0, 1, 0}, {1, 0, 1}, {1, 0, 0}, {0, 0, 1}},
    {{0, 1, 0}, {1, 0, 1}, {0, 0, 1}, {0, 1, 1}},
    {{0, 1, 0}, {1, 0, 1}, {0, 1, 1}, {1, 1, 0}},
    {{0, 1, 0}, {1, 0, 1}, {1, 1, 0}, {1, 0, 0}}};
const int kP2Edges[6][2] = {{0, 1}, {0, 2}, {0, 3}, {1, 2}, {1, 3}, {2, 3}};

template <typename T>
int upload_vec(void** dst, const std::vector<T>& src) {
  HG_CUDA(cudaMalloc(dst, std::max<size_t>(src.size(), 1) * sizeof(T)));
  if (!src.empty())
    HG_CUDA(cudaMemcpy(*dst, src.data(), src.size() * sizeof(T), cudaMemcpyHostToDevice));
  return HG_OK;
}

// P2 basis at barycentric point l: vertices l_i (2 l_i - 1), edges 4 l_i l_j.
void p2_basis(const double l[4], double phi[10]) {
  for (int i = 0; i < 4; ++i) phi[i] = l[i] * (2.0 * l[i] - 1.0);
  for (int e = 0; e < 6; ++e) phi[4 + e] = 4.0 * l[kP2Edges[e][0]] * l[kP2Edges[e][1]];
}

}  // namespace

// Anchors of the element-wise phases on a P2/N1 level with n intervals, by
// parity colour (i, j, k mod 2): packed i | j << 10 | k << 20, colour c in
// [off[c], off[c+1]).  Anchors of one colour have disjoint closed cubes
// [p, p+1]^3, so the threads of a phase never touch the same DoF.
std::vector<uint32_t> p2_anchors(int n, int off[9]) {
  std::vector<uint32_t> anch;
  for (int col = 0; col < 8; ++col) {
    off[col] = (int)anch.size();
    for (int k = col >> 2 & 1; k <= n - 1; k += 2)
      for (int j = col >> 1 & 1; j + k <= n - 1; j += 2)
        for (int i = col & 1; i + j + k <= n - 1; i += 2)
          anch.push_back((uint32_t)i | ((uint32_t)j << 10) | ((uint32_t)k << 20));
  }
  off[8] = (int)anch.size();
  return anch;
}

int Op::build_p2(const double* coeff) {
  space = HG_SPACE_P2;
  lmin = std::max(0, hier->lmin - 1);
  lmax = hier->lmax - 1;
  if (lmax < lmin || lmax < 0) {
    set_error("P2 needs a hierarchy with at least two levels above 0 (P2 level l uses lattice l+1)");
    return HG_ERR_LEVEL_RANGE;
  }
  double ka = 1.0, kb = 0.0;
  if (kind == HG_OP_P2_DIVKGRAD) {
    if (!coeff) {
      set_error("HG_OP_P2_DIVKGRAD needs coeff = {a, b}");
      return HG_ERR_INVALID_ARG;
    }
    ka = coeff[0];
    kb = coeff[1];
    // k = a + b sin sin sin lies in [a - |b|, a + |b|]: positive iff a > |b|
    if (!std::isfinite(ka) || !std::isfinite(kb) || !(ka > std::fabs(kb))) {
      set_error("HG_OP_P2_DIVKGRAD: k = a + b sin(2 pi x) sin(2 pi y) sin(2 pi z) must stay "
                "positive, which needs finite a > |b|; got a = %g, b = %g", ka, kb);
      return HG_ERR_INVALID_ARG;
    }
  }
  p2mode = kind == HG_OP_P2_MASS ? P2_MASS : P2_STIFF;
  double qb[14][4], qw[14];
  if (int r = sym14_rule(qb, qw)) return r;
  // reference mass matrix (unit volume): the rule has degree 5 >= 4, so the
  // products of two quadratics integrate exactly
  double M[10][10] = {};
  for (int q = 0; q < 14; ++q) {
    double phi[10];
    p2_basis(qb[q], phi);
    for (int a = 0; a < 10; ++a)
      for (int b = 0; b < 10; ++b) M[a][b] += qw[q] * phi[a] * phi[b];
  }
  if (int r = p2_upload_constants(qb, qw, M)) return r;
  const Mesh& m = *hier->mesh;
  const int nl = lmax - lmin + 1;
  for (int dt = 0; dt < 2; ++dt) {
    p2cells[dt].assign(nl, nullptr);
    p2acc[dt].assign(nl, nullptr);
    p2inv[dt].assign(nl, nullptr);
  }
  p2anchors.assign(nl, nullptr);
  p2off.assign(nl, std::vector<int>(9, 0));
  for (int l = lmin; l <= lmax; ++l) {
    const int li = l - lmin, n = 1 << l;
    if (n > 1023) {
      set_error("P2 level %d too fine for packed anchors", l);
      return HG_ERR_LEVEL_RANGE;
    }
    // anchors (all types admit i+j+k <= n-1 at most) by parity colour
    const std::vector<uint32_t> anch = p2_anchors(n, p2off[li].data());
    if (int r = upload_vec((void**)&p2anchors[li], anch)) return r;
    // element data per cell
    std::vector<P2Cell<double>> c64(m.nc);
    std::vector<P2Cell<float>> c32(m.nc);
    for (int64_t c = 0; c < m.nc; ++c) {
      P2Cell<double>& P = c64[c];
      memset(&P, 0, sizeof P);
      const double* V[4];
      for (int q = 0; q < 4; ++q) V[q] = &m.xyz[3 * m.cells[c][q]];
      double vol0 = 0.0;
      for (int t = 0; t < 6; ++t) {
        double X[4][3], G[4][3], vol;
        for (int a = 0; a < 4; ++a)
          for (int r = 0; r < 3; ++r)
            X[a][r] = V[0][r] + (kTypeOffP2[t][a][0] * (V[1][r] - V[0][r]) +
                                 kTypeOffP2[t][a][1] * (V[2][r] - V[0][r]) +
                                 kTypeOffP2[t][a][2] * (V[3][r] - V[0][r])) / (double)n;
        bary_gradients(X, G, &vol);
        if (t == 0) vol0 = vol;
        int e = 0;
        for (int a = 0; a < 4; ++a)
          for (int b = a; b < 4; ++b, ++e)
            P.H[t][e] = G[a][0] * G[b][0] + G[a][1] * G[b][1] + G[a][2] * G[b][2];
        for (int q = 0; q < 14; ++q)
          for (int r = 0; r < 3; ++r) {
            double d = -V[0][r];
            for (int a = 0; a < 4; ++a) d += qb[q][a] * X[a][r];
            P.sc[t][q][2 * r] = std::sin(2.0 * M_PI * d);
            P.sc[t][q][2 * r + 1] = std::cos(2.0 * M_PI * d);
          }
      }
      P.vol = vol0;
      for (int q = 0; q < 14; ++q) {
        P.kA[q] = qw[q] * vol0 * ka;
        P.kB[q] = qw[q] * vol0 * kb;
      }
      for (int r = 0; r < 3; ++r) {
        P.x0[r] = V[0][r];
        for (int a = 0; a < 3; ++a) P.e[a][r] = (V[a + 1][r] - V[0][r]) / (double)n;
      }
      const double* src = reinterpret_cast<const double*>(&P);
      float* dst = reinterpret_cast<float*>(&c32[c]);
      for (size_t q = 0; q < sizeof(P) / sizeof(double); ++q) dst[q] = (float)src[q];
    }
    if (int r = upload_vec(&p2cells[HG_F64][li], c64)) return r;
    if (int r = upload_vec(&p2cells[HG_F32][li], c32)) return r;
    const LevelDev& L = dev(l);
    for (int dt = 0; dt < 2; ++dt) {
      const size_t bytes = L.n_stored * (dt == HG_F64 ? 8 : 4);
      HG_CUDA(cudaMalloc(&p2acc[dt][li], bytes));
      HG_CUDA(cudaMalloc(&p2inv[dt][li], bytes));
      HG_CUDA(cudaMemset(p2inv[dt][li], 0, bytes));
      P2Args A;
      A.n = n;
      A.ncells = (int)m.nc;
      A.cells = p2cells[dt][li];
      A.anchors = p2anchors[li];
      for (int q = 0; q < 9; ++q) A.anchor_off[q] = p2off[li][q];
      A.mode = p2mode;
      A.acc = p2acc[dt][li];
      A.invdiag = nullptr;
      if (p2mode == P2_STIFF)
        if (int r = launch_p2_diag(L, dt, A, p2inv[dt][li], 0)) return r;
    }
  }
  HG_CUDA(cudaDeviceSynchronize());
  return HG_OK;
}

// Lowest-order Nedelec operator alpha curl curl + beta I on the P2 storage
// (edge DoFs; Sec. 6, Nedelec elements for the curl-curl problem).  Per cell
// and type the 6x6 element matrix of the Whitney basis
//   w_e = l_a grad l_b - l_b grad l_a,  curl w_e = 2 grad l_a x grad l_b,
//   K_ef = |T| curl w_e . curl w_f,  M_ef = int w_e . w_f (int l_i l_j = |T| (1 + d_ij) / 20),
// scaled by the signs that map the local edge a -> b to the global
// orientation (lower canonical key -> higher: the first nonzero of dz, dy, dx
// of the edge vector is positive).
int Op::build_n1(const double* coeff) {
  space = HG_SPACE_P2;
  lmin = std::max(0, hier->lmin - 1);
  lmax = hier->lmax - 1;
  if (lmax < lmin || lmax < 0) {
    set_error("N1 needs a hierarchy with at least two levels above 0 (N1 level l uses lattice l+1)");
    return HG_ERR_LEVEL_RANGE;
  }
  if (!coeff || !(coeff[0] >= 0.0) || !(coeff[1] > 0.0)) {
    set_error("HG_OP_N1_CURLCURL needs coeff = {alpha >= 0, beta > 0}");
    return HG_ERR_INVALID_ARG;
  }
  const double alpha = coeff[0], beta = coeff[1];
  n1alpha = alpha;
  n1beta = beta;
  p2mode = P2_N1;
  const Mesh& m = *hier->mesh;
  // orientation sign of each lattice direction in each cell: +1 when the
  // physical vector has a positive first nonzero of z, y, x
  {
    std::vector<int8_t> sg(8 * m.nc, 0);
    for (int64_t c = 0; c < m.nc; ++c) {
      const double* V[4];
      for (int q = 0; q < 4; ++q) V[q] = &m.xyz[3 * m.cells[c][q]];
      for (int d = 0; d < 7; ++d) {
        double v[3], len = 0.0;
        for (int r = 0; r < 3; ++r) {
          v[r] = kN1Dir[d][0] * (V[1][r] - V[0][r]) + kN1Dir[d][1] * (V[2][r] - V[0][r]) +
                 kN1Dir[d][2] * (V[3][r] - V[0][r]);
          len += v[r] * v[r];
        }
        const double tol = 1e-9 * std::sqrt(len);
        sg[8 * c + d] = std::fabs(v[2]) > tol ? (v[2] > 0 ? 1 : -1)
                        : std::fabs(v[1]) > tol ? (v[1] > 0 ? 1 : -1)
                                                : (v[0] > 0 ? 1 : -1);
      }
    }
    if (int r = upload_vec((void**)&n1sign, sg)) return r;
  }
  const int nl = lmax - lmin + 1;
  for (int dt = 0; dt < 2; ++dt) {
    p2cells[dt].assign(nl, nullptr);
    p2acc[dt].assign(nl, nullptr);
    p2inv[dt].assign(nl, nullptr);
  }
  p2anchors.assign(nl, nullptr);
  p2off.assign(nl, std::vector<int>(9, 0));
  for (int l = lmin; l <= lmax; ++l) {
    const int li = l - lmin, n = 1 << l;
    if (n > 1023) {
      set_error("N1 level %d too fine for packed anchors", l);
      return HG_ERR_LEVEL_RANGE;
    }
    const std::vector<uint32_t> anch = p2_anchors(n, p2off[li].data());
    if (int r = upload_vec((void**)&p2anchors[li], anch)) return r;
    std::vector<N1Cell<double>> c64(m.nc);
    std::vector<N1Cell<float>> c32(m.nc);
    for (int64_t c = 0; c < m.nc; ++c) {
      const double* V[4];
      for (int q = 0; q < 4; ++q) V[q] = &m.xyz[3 * m.cells[c][q]];
      for (int t = 0; t < 6; ++t) {
        double X[4][3], G[4][3], vol;
        for (int a = 0; a < 4; ++a)
          for (int r = 0; r < 3; ++r)
            X[a][r] = V[0][r] + (kTypeOffP2[t][a][0] * (V[1][r] - V[0][r]) +
                                 kTypeOffP2[t][a][1] * (V[2][r] - V[0][r]) +
                                 kTypeOffP2[t][a][2] * (V[3][r] - V[0][r])) / (double)n;
        bary_gradients(X, G, &vol);
        double C[6][3], sg[6];
        for (int e = 0; e < 6; ++e) {
          const int a = kP2Edges[e][0], b = kP2Edges[e][1];
          C[e][0] = 2.0 * (G[a][1] * G[b][2] - G[a][2] * G[b][1]);
          C[e][1] = 2.0 * (G[a][2] * G[b][0] - G[a][0] * G[b][2]);
          C[e][2] = 2.0 * (G[a][0] * G[b][1] - G[a][1] * G[b][0]);
          double d[3], len = 0.0;
          for (int r = 0; r < 3; ++r) {
            d[r] = X[b][r] - X[a][r];
            len += d[r] * d[r];
          }
          const double tol = 1e-9 * std::sqrt(len);
          sg[e] = std::fabs(d[2]) > tol ? (d[2] > 0 ? 1.0 : -1.0)
                  : std::fabs(d[1]) > tol ? (d[1] > 0 ? 1.0 : -1.0)
                                          : (d[0] > 0 ? 1.0 : -1.0);
        }
        double GG[4][4];
        for (int a = 0; a < 4; ++a)
          for (int b = 0; b < 4; ++b)
            GG[a][b] = G[a][0] * G[b][0] + G[a][1] * G[b][1] + G[a][2] * G[b][2];
        auto L = [](int i, int j) { return (i == j ? 2.0 : 1.0) / 20.0; };
        for (int e = 0; e < 6; ++e)
          for (int f = 0; f < 6; ++f) {
            const int a = kP2Edges[e][0], b = kP2Edges[e][1];
            const int cc = kP2Edges[f][0], dd = kP2Edges[f][1];
            const double kc = C[e][0] * C[f][0] + C[e][1] * C[f][1] + C[e][2] * C[f][2];
            const double ms = L(a, cc) * GG[b][dd] - L(a, dd) * GG[b][cc] - L(b, cc) * GG[a][dd] +
                              L(b, dd) * GG[a][cc];
            const double v = sg[e] * sg[f] * vol * (alpha * kc + beta * ms);
            c64[c].K[t][6 * e + f] = v;
            c32[c].K[t][6 * e + f] = (float)v;
          }
      }
    }
    if (int r = upload_vec(&p2cells[HG_F64][li], c64)) return r;
    if (int r = upload_vec(&p2cells[HG_F32][li], c32)) return r;
    const LevelDev& Ld = dev(l);
    for (int dt = 0; dt < 2; ++dt) {
      const size_t bytes = Ld.n_stored * (dt == HG_F64 ? 8 : 4);
      HG_CUDA(cudaMalloc(&p2acc[dt][li], bytes));
      HG_CUDA(cudaMalloc(&p2inv[dt][li], bytes));
      HG_CUDA(cudaMemset(p2inv[dt][li], 0, bytes));
      P2Args A;
      A.n = n;
      A.ncells = (int)m.nc;
      A.cells = p2cells[dt][li];
      A.anchors = p2anchors[li];
      for (int q = 0; q < 9; ++q) A.anchor_off[q] = p2off[li][q];
      A.mode = P2_N1;
      A.acc = p2acc[dt][li];
      A.invdiag = nullptr;
      if (int r = launch_p2_diag(Ld, dt, A, p2inv[dt][li], 0)) return r;
    }
  }
  HG_CUDA(cudaDeviceSynchronize());
  return HG_OK;
}

}  // namespace hg

extern "C" int hg_p2_anchors(int level, uint32_t* out, int* off, int* n_anchors) {
  if (level < 0 || level > 9 || !n_anchors) {
    hg::set_error("hg_p2_anchors: bad argument");
    return HG_ERR_INVALID_ARG;
  }
  int o[9];
  const std::vector<uint32_t> a = hg::p2_anchors(1 << level, o);
  *n_anchors = (int)a.size();
  if (off)
    for (int c = 0; c < 9; ++c) off[c] = o[c];
  if (out)
    for (size_t q = 0; q < a.size(); ++q) out[q] = a[q];
  return HG_OK;
}
