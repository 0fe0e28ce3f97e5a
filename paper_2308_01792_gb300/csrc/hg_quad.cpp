// Quadrature on the tetrahedron for the variable-coefficient P2 element
// matrices (Sec. 5.2: element matrices formed on the fly by quadrature; the
// paper names its forms by quadrature order only).
//
// The rule is the symmetric 14-point, degree-5, positive-weight rule with
// orbits 4 + 4 + 6 (Walkington, "Quadrature on simplices of arbitrary
// dimension", 2000).  It is not copied from a table: its six parameters
// (w1, a1, w2, a2, w3, a3) solve the six moment equations of the symmetric
// invariants of degree 0, 2, 3, 4, 4, 5 and are found here by Newton's
// method from four-digit starting values.  Barycentric monomials integrate to
// 3! prod(alpha_i!) / (|alpha| + 3)! on a tetrahedron of unit volume.
#include <cmath>
#include <cstring>
#include <mutex>

#include "hg_host.h"

namespace hg {

namespace {

double factorial(int k) {
  double f = 1.0;
  for (int q = 2; q <= k; ++q) f *= q;
  return f;
}

double exact_moment(const int al[4]) {
  return 6.0 * factorial(al[0]) * factorial(al[1]) * factorial(al[2]) * factorial(al[3]) /
         factorial(al[0] + al[1] + al[2] + al[3] + 3);
}

// Points of the rule for parameters p = (w1, a1, w2, a2, w3, a3).
void rule_points(const double p[6], double bary[14][4], double w[14]) {
  int q = 0;
  for (int orb = 0; orb < 2; ++orb) {
    const double wt = p[2 * orb], a = p[2 * orb + 1];
    for (int m = 0; m < 4; ++m, ++q) {
      for (int r = 0; r < 4; ++r) bary[q][r] = r == m ? 1.0 - 3.0 * a : a;
      w[q] = wt;
    }
  }
  // the six arrangements of (a, a, b, b), b = 1/2 - a
  const double a = p[5], b = 0.5 - p[5];
  static const int pairs[6][2] = {{0, 1}, {0, 2}, {0, 3}, {1, 2}, {1, 3}, {2, 3}};
  for (int e = 0; e < 6; ++e, ++q) {
    for (int r = 0; r < 4; ++r) bary[q][r] = b;
    bary[q][pairs[e][0]] = a;
    bary[q][pairs[e][1]] = a;
    w[q] = p[4];
  }
}

const int kMoments[6][4] = {{0, 0, 0, 0}, {2, 0, 0, 0}, {3, 0, 0, 0},
                            {4, 0, 0, 0}, {2, 2, 0, 0}, {5, 0, 0, 0}};

void residual(const double p[6], double f[6]) {
  double bary[14][4], w[14];
  rule_points(p, bary, w);
  for (int e = 0; e < 6; ++e) {
    double s = 0.0;
    for (int q = 0; q < 14; ++q) {
      double m = w[q];
      for (int r = 0; r < 4; ++r) m *= std::pow(bary[q][r], kMoments[e][r]);
      s += m;
    }
    f[e] = s - exact_moment(kMoments[e]);
  }
}

// Dense 6x6 solve with partial pivoting; false if singular.
bool solve6(double A[6][6], double b[6]) {
  for (int c = 0; c < 6; ++c) {
    int piv = c;
    for (int r = c + 1; r < 6; ++r)
      if (std::fabs(A[r][c]) > std::fabs(A[piv][c])) piv = r;
    if (std::fabs(A[piv][c]) < 1e-300) return false;
    if (piv != c) {
      for (int k = 0; k < 6; ++k) std::swap(A[c][k], A[piv][k]);
      std::swap(b[c], b[piv]);
    }
    for (int r = c + 1; r < 6; ++r) {
      const double f = A[r][c] / A[c][c];
      for (int k = c; k < 6; ++k) A[r][k] -= f * A[c][k];
      b[r] -= f * b[c];
    }
  }
  for (int c = 5; c >= 0; --c) {
    double v = b[c];
    for (int k = c + 1; k < 6; ++k) v -= A[c][k] * b[k];
    b[c] = v / A[c][c];
  }
  return true;
}

}  // namespace

int derive_sym14(double sb[14][4], double sw[14]);

int sym14_rule(double bary[14][4], double w[14]) {
  static std::once_flag once;
  static int status = HG_OK;
  static double sb[14][4], sw[14];
  std::call_once(once, [] { status = derive_sym14(sb, sw); });
  if (status) {
    set_error("quadrature: the degree-5 rule could not be derived");
    return status;
  }
  memcpy(bary, sb, sizeof sb);
  memcpy(w, sw, sizeof sw);
  return HG_OK;
}

int derive_sym14(double sb[14][4], double sw[14]) {
  {
    double p[6] = {0.0735, 0.0927, 0.1127, 0.3109, 0.0425, 0.4545};
    for (int it = 0; it < 50; ++it) {
      double f[6], J[6][6];
      residual(p, f);
      double nf = 0.0;
      for (double v : f) nf = std::fmax(nf, std::fabs(v));
      if (nf < 1e-16) break;
      for (int c = 0; c < 6; ++c) {
        double pp[6], fp[6];
        memcpy(pp, p, sizeof pp);
        const double h = 1e-7 * std::fmax(1.0, std::fabs(p[c]));
        pp[c] += h;
        residual(pp, fp);
        for (int r = 0; r < 6; ++r) J[r][c] = (fp[r] - f[r]) / h;
      }
      double d[6];
      for (int r = 0; r < 6; ++r) d[r] = -f[r];
      if (!solve6(J, d)) {
        set_error("quadrature: singular Newton system");
        return HG_ERR_INVALID_ARG;
      }
      for (int c = 0; c < 6; ++c) p[c] += d[c];
    }
    double f[6];
    residual(p, f);
    for (double v : f)
      if (!(std::fabs(v) < 1e-14)) {
        set_error("quadrature: moment equations not solved (residual %g)", v);
        return HG_ERR_INVALID_ARG;
      }
    rule_points(p, sb, sw);
    for (int q = 0; q < 14; ++q)
      if (!(sw[q] > 0.0)) {
        set_error("quadrature: non-positive weight");
        return HG_ERR_INVALID_ARG;
      }
  }
  return HG_OK;
}

}  // namespace hg

extern "C" int hg_quadrature_rule(double* bary, double* weights, int* npoints) {
  double b[14][4], w[14];
  if (int r = hg::sym14_rule(b, w)) return r;
  if (npoints) *npoints = 14;
  if (bary) memcpy(bary, b, sizeof b);
  if (weights) memcpy(weights, w, sizeof w);
  return HG_OK;
}
