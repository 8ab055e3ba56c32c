// Univariate B-spline matrices and loads on the host (Sec. 2.1, Sec. 3.3).
//
// For each non-empty knot span the p+1 B-splines that do not vanish there are
// evaluated together by the triangular form of the Cox-de Boor recursion
// (Sec. 2.1), their first derivatives from the degree p-1 values, and the
// products are integrated with a Gauss-Legendre rule whose nodes are found by
// Newton's method on the Legendre three-term recurrence.
#include <cmath>
#include <vector>

#include "stfd.h"
#include "stfd_internal.h"

namespace stfd {

// Open uniform knot vector on [0, L]: p+1 zeros, n_el-1 simple interior
// knots, p+1 copies of L (Sec. 2.1 with maximal smoothness, Sec. 5).
std::vector<double> open_knots(int p, int n_el, double L) {
  std::vector<double> kv;
  kv.reserve(n_el + 2 * p + 1);
  for (int i = 0; i <= p; ++i) kv.push_back(0.0);
  for (int e = 1; e < n_el; ++e) kv.push_back(L * e / n_el);
  for (int i = 0; i <= p; ++i) kv.push_back(L);
  return kv;
}

// nq-point Gauss-Legendre nodes/weights on [-1, 1].
void gauss_legendre(int nq, std::vector<double>& x, std::vector<double>& w) {
  x.assign(nq, 0.0);
  w.assign(nq, 0.0);
  const double pi = 3.14159265358979323846;
  for (int i = 0; i < (nq + 1) / 2; ++i) {
    double z = std::cos(pi * (i + 0.75) / (nq + 0.5));
    double dp = 1.0;
    for (int it = 0; it < 100; ++it) {
      double p0 = 1.0, p1 = z;          // P_0, P_1
      for (int k = 2; k <= nq; ++k) {   // k P_k = (2k-1) z P_{k-1} - (k-1) P_{k-2}
        double pk = ((2.0 * k - 1.0) * z * p1 - (k - 1.0) * p0) / k;
        p0 = p1;
        p1 = pk;
      }
      if (nq == 1) { p1 = z; p0 = 1.0; }
      dp = nq * (z * p1 - p0) / (z * z - 1.0);   // P_n'
      double dz = p1 / dp;
      z -= dz;
      if (std::fabs(dz) < 1e-16) break;
    }
    // recompute derivative at the converged node
    double p0 = 1.0, p1 = z;
    for (int k = 2; k <= nq; ++k) {
      double pk = ((2.0 * k - 1.0) * z * p1 - (k - 1.0) * p0) / k;
      p0 = p1;
      p1 = pk;
    }
    dp = (nq == 1) ? 1.0 : nq * (z * p1 - p0) / (z * z - 1.0);
    x[i] = -z;
    x[nq - 1 - i] = z;
    double wi = 2.0 / ((1.0 - z * z) * dp * dp);
    w[i] = wi;
    w[nq - 1 - i] = wi;
  }
}

// Values N[0..deg] of the B-splines b_{k-deg..k} of degree `deg` at x in span
// k (kv[k] <= x <= kv[k+1]): triangular Cox-de Boor, each stage raising the
// degree by one through the two-term recursion of Sec. 2.1.
static void span_values(const std::vector<double>& kv, int k, int deg, double x, double* N) {
  double left[32], right[32];
  N[0] = 1.0;
  for (int j = 1; j <= deg; ++j) {
    left[j] = x - kv[k + 1 - j];
    right[j] = kv[k + j] - x;
    double carry = 0.0;
    for (int r = 0; r < j; ++r) {
      double den = right[r + 1] + left[j - r];
      double t = (den != 0.0) ? N[r] / den : 0.0;   // 0/0 = 0
      N[r] = carry + right[r + 1] * t;
      carry = left[j - r] * t;
    }
    N[j] = carry;
  }
}

// Values and first derivatives of b_{k-p..k} at x in span k.
void span_values_derivs(const std::vector<double>& kv, int k, int p, double x,
                               double* N, double* dN) {
  span_values(kv, k, p, x, N);
  if (p == 0) { dN[0] = 0.0; return; }
  double Nm[32];
  span_values(kv, k, p - 1, x, Nm);        // b_{k-p+1..k} of degree p-1
  // b'_{i,p} = p b_{i,p-1}/(kv[i+p]-kv[i]) - p b_{i+1,p-1}/(kv[i+p+1]-kv[i+1])
  for (int a = 0; a <= p; ++a) {
    int i = k - p + a;
    double lo = (a >= 1) ? Nm[a - 1] : 0.0;     // b_{i,p-1}
    double hi = (a <= p - 1) ? Nm[a] : 0.0;     // b_{i+1,p-1}
    double d1 = kv[i + p] - kv[i];
    double d2 = kv[i + p + 1] - kv[i + 1];
    dN[a] = (d1 != 0.0 ? p * lo / d1 : 0.0) - (d2 != 0.0 ? p * hi / d2 : 0.0);
  }
}

static int reduced_range(int m, int bc, int* lo) {
  if (bc == STFD_BC_NONE) { *lo = 0; return m; }
  if (bc == STFD_BC_INITIAL) { *lo = 1; return m - 1; }
  if (bc == STFD_BC_DIRICHLET) { *lo = 1; return m - 2; }
  return -1;
}

}  // namespace stfd

using namespace stfd;

extern "C" int stfd_spline_matrices(int p, int n_el, double length, int bc,
                                    double* M, double* K, double* W, int* n_out) {
  if (p < 1 || p > 30 || n_el < 1 || !(length > 0.0)) return STFD_ERR_ARG;
  const int m = n_el + p;
  int lo = 0;
  const int n = reduced_range(m, bc, &lo);
  if (n < 1) return STFD_ERR_ARG;
  if (n_out) *n_out = n;
  if (!M && !K && !W) return STFD_OK;
  std::vector<double> kv = open_knots(p, n_el, length);
  std::vector<double> full_M((size_t)m * m, 0.0), full_K((size_t)m * m, 0.0), full_W((size_t)m * m, 0.0);
  std::vector<double> gx, gw;
  gauss_legendre(p + 1, gx, gw);   // exact for the degree <= 2p integrands
  double N[32], dN[32];
  for (int k = p; k < p + n_el; ++k) {     // non-empty spans kv[k] < kv[k+1]
    const double a = kv[k], b = kv[k + 1];
    const double half = 0.5 * (b - a);
    for (size_t q = 0; q < gx.size(); ++q) {
      const double x = a + half * (gx[q] + 1.0);
      const double wq = half * gw[q];
      span_values_derivs(kv, k, p, x, N, dN);
      for (int r = 0; r <= p; ++r) {
        const int i = k - p + r;
        for (int c = 0; c <= p; ++c) {
          const int j = k - p + c;
          full_M[i + (size_t)m * j] += wq * N[r] * N[c];
          full_K[i + (size_t)m * j] += wq * dN[r] * dN[c];
          full_W[i + (size_t)m * j] += wq * N[r] * dN[c];   // W[i,j] = int b'_j b_i
        }
      }
    }
  }
  for (int j = 0; j < n; ++j)
    for (int i = 0; i < n; ++i) {
      const size_t src = (i + lo) + (size_t)m * (j + lo), dst = i + (size_t)n * j;
      if (M) M[dst] = full_M[src];
      if (K) K[dst] = full_K[src];
      if (W) W[dst] = full_W[src];
    }
  return STFD_OK;
}

extern "C" int stfd_spline_load_trig(int p, int n_el, double length, int bc,
                                     double freq, double c_sin, double c_cos, double* out) {
  if (p < 1 || p > 30 || n_el < 1 || !(length > 0.0) || !out) return STFD_ERR_ARG;
  const int m = n_el + p;
  int lo = 0;
  const int n = reduced_range(m, bc, &lo);
  if (n < 1) return STFD_ERR_ARG;
  std::vector<double> kv = open_knots(p, n_el, length);
  std::vector<double> full(m, 0.0), gx, gw;
  gauss_legendre(12, gx, gw);
  double N[32];
  for (int k = p; k < p + n_el; ++k) {
    const double a = kv[k], b = kv[k + 1];
    const double half = 0.5 * (b - a);
    for (size_t q = 0; q < gx.size(); ++q) {
      const double x = a + half * (gx[q] + 1.0);
      const double fx = c_sin * std::sin(freq * x) + c_cos * std::cos(freq * x);
      span_values(kv, k, p, x, N);
      for (int r = 0; r <= p; ++r) full[k - p + r] += half * gw[q] * fx * N[r];
    }
  }
  for (int i = 0; i < n; ++i) out[i] = full[i + lo];
  return STFD_OK;
}
