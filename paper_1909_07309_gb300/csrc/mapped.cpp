// Spatial matrices of a mapped single-patch domain with variable coefficients
// (Sec. 4.6 and 4.6.1), the element data of the geometry-aware preconditioner
// (eq. separation) and weighted univariate matrices (eq. over_A). Host code.
//
// On every parametric element the local matrices
//     M_e[a,b] = sum_q w_q c(q) |det J(q)| B^_a(q) B^_b(q)
//     K_e[a,b] = sum_q w_q kappa(q) grad^B^_a(q) . G(q) grad^B^_b(q),
//     G = |det J| J^{-1} J^{-T},
// are integrated by sum factorisation over the tensor Gauss points (one
// direction contracted at a time), then scattered into the tensor-product
// stencil layout described in stfd.h. Lines of elements along direction 1 are
// processed in colours of the outer directions (indices mod p+1) so that
// threads never write the same row.
#include <algorithm>
#include <cmath>
#include <thread>
#include <vector>

#include "stfd.h"
#include "stfd_internal.h"

namespace stfd {
namespace {

constexpr double kW1 = 0.70710678118654752440;   // weight of the middle control point, 1/sqrt(2)

// Rational quadratic quarter circle with control points (1,0), (1,1), (0,1)
// and weights 1, 1/sqrt(2), 1: point C(t) and derivative C'(t) (quotient rule).
void quarter_circle(double t, double* C, double* dC) {
  const double s = 1.0 - t;
  const double b0 = s * s, b1 = 2.0 * t * s, b2 = t * t;              // Bernstein basis
  const double d0 = -2.0 * s, d1 = 2.0 - 4.0 * t, d2 = 2.0 * t;
  const double w = b0 + kW1 * b1 + b2, dw = d0 + kW1 * d1 + d2;
  const double nx = b0 + kW1 * b1, ny = kW1 * b1 + b2;                 // weighted control points
  const double dnx = d0 + kW1 * d1, dny = kW1 * d1 + d2;
  C[0] = nx / w;
  C[1] = ny / w;
  dC[0] = (dnx - C[0] * dw) / w;
  dC[1] = (dny - C[1] * dw) / w;
}

// x = F(eta) and J[a * d + b] = d x_a / d eta_b. The quarter annulus is
// (1 + eta_1) C(eta_2), extruded in eta_3 when d = 3.
bool geom_eval(int geom, int d, const double* eta, double* x, double* J) {
  for (int k = 0; k < d * d; ++k) J[k] = 0.0;
  if (geom == STFD_GEOM_BOX) {
    for (int a = 0; a < d; ++a) {
      x[a] = eta[a];
      J[a * d + a] = 1.0;
    }
    return true;
  }
  if (geom == STFD_GEOM_QUARTER_ANNULUS && d >= 2) {
    const double r = 1.0 + eta[0];
    double C[2], dC[2];
    quarter_circle(eta[1], C, dC);
    x[0] = r * C[0];
    x[1] = r * C[1];
    J[0 * d + 0] = C[0];
    J[1 * d + 0] = C[1];
    J[0 * d + 1] = r * dC[0];
    J[1 * d + 1] = r * dC[1];
    if (d == 3) {
      x[2] = eta[2];
      J[2 * d + 2] = 1.0;
    }
    return true;
  }
  if (geom == STFD_GEOM_REVOLVED_QUARTER_ANNULUS && d == 3) {
    // planar annulus (a, b) = (1 + eta_1) C(eta_2), turned about {(x_1, -1, 0)} by the angle of C(eta_3)
    const double r = 1.0 + eta[0];
    double C2[2], dC2[2], C3[2], dC3[2];
    quarter_circle(eta[1], C2, dC2);
    quarter_circle(eta[2], C3, dC3);
    const double a = r * C2[0], b = r * C2[1];
    const double da[3] = {C2[0], r * dC2[0], 0.0}, db[3] = {C2[1], r * dC2[1], 0.0};
    x[0] = a;
    x[1] = -1.0 + (b + 1.0) * C3[0];
    x[2] = (b + 1.0) * C3[1];
    for (int k = 0; k < 3; ++k) {
      J[0 * 3 + k] = da[k];
      J[1 * 3 + k] = db[k] * C3[0];
      J[2 * 3 + k] = db[k] * C3[1];
    }
    J[1 * 3 + 2] += (b + 1.0) * dC3[0];
    J[2 * 3 + 2] += (b + 1.0) * dC3[1];
    return true;
  }
  return false;
}

bool geom_ok(int geom, int d) {
  return geom == STFD_GEOM_BOX || (geom == STFD_GEOM_QUARTER_ANNULUS && d >= 2) ||
         (geom == STFD_GEOM_REVOLVED_QUARTER_ANNULUS && d == 3);
}

// All three geometries have J^T J diagonal (C' is orthogonal to C, and the
// turn is orthogonal to the plane of the annulus), so only the diagonal
// entries of G carry stiffness terms.
bool diagonal_metric(int geom) {
  return geom == STFD_GEOM_BOX || geom == STFD_GEOM_QUARTER_ANNULUS || geom == STFD_GEOM_REVOLVED_QUARTER_ANNULUS;
}

// G = |det J| J^{-1} J^{-T}; returns |det J| (0 if J is singular).
double metric(int d, const double* J, double* G) {
  double inv[9];
  double det;
  if (d == 1) {
    det = J[0];
    if (det == 0.0) return 0.0;
    inv[0] = 1.0 / det;
  } else if (d == 2) {
    det = J[0] * J[3] - J[1] * J[2];
    if (det == 0.0) return 0.0;
    inv[0] = J[3] / det;
    inv[1] = -J[1] / det;
    inv[2] = -J[2] / det;
    inv[3] = J[0] / det;
  } else {
    const double c00 = J[4] * J[8] - J[5] * J[7], c01 = J[5] * J[6] - J[3] * J[8], c02 = J[3] * J[7] - J[4] * J[6];
    det = J[0] * c00 + J[1] * c01 + J[2] * c02;
    if (det == 0.0) return 0.0;
    inv[0] = c00 / det;
    inv[3] = c01 / det;
    inv[6] = c02 / det;
    inv[1] = (J[2] * J[7] - J[1] * J[8]) / det;
    inv[4] = (J[0] * J[8] - J[2] * J[6]) / det;
    inv[7] = (J[1] * J[6] - J[0] * J[7]) / det;
    inv[2] = (J[1] * J[5] - J[2] * J[4]) / det;
    inv[5] = (J[2] * J[3] - J[0] * J[5]) / det;
    inv[8] = (J[0] * J[4] - J[1] * J[3]) / det;
  }
  const double ad = std::fabs(det);
  for (int a = 0; a < d; ++a)
    for (int b = 0; b < d; ++b) {
      double s = 0.0;
      for (int c = 0; c < d; ++c) s += inv[a * d + c] * inv[b * d + c];
      G[a * d + b] = ad * s;
    }
  return ad;
}

// Per 1D element of (0, 1): Gauss points, weights, and the p+1 active
// B-splines (full indices k..k+p) with derivatives at each point.
struct Tab1 {
  int nq = 0, L = 0;
  std::vector<double> x, w;      // [k][q]
  std::vector<double> V, D;      // [k][a][q]
};

Tab1 make_tab(int p, int n_el, int nq) {
  Tab1 t;
  t.nq = nq;
  t.L = p + 1;
  std::vector<double> kv = open_knots(p, n_el, 1.0);
  std::vector<double> gx, gw;
  gauss_legendre(nq, gx, gw);
  t.x.resize((size_t)n_el * nq);
  t.w.resize((size_t)n_el * nq);
  t.V.resize((size_t)n_el * t.L * nq);
  t.D.resize((size_t)n_el * t.L * nq);
  double N[32], dN[32];
  for (int k = 0; k < n_el; ++k) {
    const double a = kv[p + k], b = kv[p + k + 1], half = 0.5 * (b - a);
    for (int q = 0; q < nq; ++q) {
      const double x = a + half * (gx[q] + 1.0);
      t.x[(size_t)k * nq + q] = x;
      t.w[(size_t)k * nq + q] = half * gw[q];
      span_values_derivs(kv, p + k, p, x, N, dN);
      for (int r = 0; r <= p; ++r) {
        t.V[((size_t)k * t.L + r) * nq + q] = N[r];
        t.D[((size_t)k * t.L + r) * nq + q] = dN[r];
      }
    }
  }
  return t;
}

struct Problem {
  int d, p, n_el, geom, nq;
  int L, Ld, Qe;        // local functions per direction, per element, points per element
  long long n_elem;
  int n_s;
  long long Ns;
  Tab1 tab;
};

bool problem_init(Problem& P, int d, int p, int n_el, int geom, int nq) {
  if (d < 1 || d > kMaxDim || p < 1 || p > 10 || n_el < 1 || nq < 1 || nq > 32) return false;
  if (!geom_ok(geom, d)) return false;
  if (n_el + p - 2 < 1) return false;
  P.d = d;
  P.p = p;
  P.n_el = n_el;
  P.geom = geom;
  P.nq = nq;
  P.L = p + 1;
  P.Ld = 1;
  P.Qe = 1;
  P.n_elem = 1;
  for (int l = 0; l < d; ++l) {
    P.Ld *= P.L;
    P.Qe *= nq;
    P.n_elem *= n_el;
  }
  P.n_s = n_el + p - 2;
  P.Ns = 1;
  for (int l = 0; l < d; ++l) P.Ns *= P.n_s;
  P.tab = make_tab(p, n_el, nq);
  return true;
}

// Element multi-index of the colexicographic element number.
void elem_index(const Problem& P, long long e, int* ei) {
  for (int l = 0; l < P.d; ++l) {
    ei[l] = (int)(e % P.n_el);
    e /= P.n_el;
  }
}

// Geometry at the element's points: eta-ordered colexicographically.
// Fills x (d per point), detw = w |det J|, G (d*d per point, scaled by w).
void element_geometry(const Problem& P, const int* ei, std::vector<double>& x, std::vector<double>& detw,
                      std::vector<double>& Gw) {
  const int d = P.d, nq = P.nq;
  x.resize((size_t)P.Qe * d);
  detw.resize(P.Qe);
  Gw.resize((size_t)P.Qe * d * d);
  double eta[3], J[9], G[9];
  for (int q = 0; q < P.Qe; ++q) {
    int rest = q;
    double w = 1.0;
    for (int l = 0; l < d; ++l) {
      const int ql = rest % nq;
      rest /= nq;
      eta[l] = P.tab.x[(size_t)ei[l] * nq + ql];
      w *= P.tab.w[(size_t)ei[l] * nq + ql];
    }
    geom_eval(P.geom, d, eta, &x[(size_t)q * d], J);
    const double ad = metric(d, J, G);
    detw[q] = w * ad;
    for (int k = 0; k < d * d; ++k) Gw[(size_t)q * d * d + k] = w * G[k];
  }
}

// Loc[a][b] += sum_q W[q] prod_l R_l[a_l][q_l] C_l[b_l][q_l] by sum
// factorisation; directions beyond d are padded with a single point of
// weight 1 and a single function of value 1.
struct SumFact {
  std::vector<double> T1, T2;
  void run(const Problem& P, const double* W, const double* const* R, const double* const* C, double* Loc) {
    const int d = P.d, nq = P.nq, L = P.L;
    const int n1 = nq, n2 = d >= 2 ? nq : 1, n3 = d >= 3 ? nq : 1;
    const int L1 = L, L2 = d >= 2 ? L : 1, L3 = d >= 3 ? L : 1;
    static const double one = 1.0;
    const double* R2 = d >= 2 ? R[1] : &one;
    const double* C2 = d >= 2 ? C[1] : &one;
    const double* R3 = d >= 3 ? R[2] : &one;
    const double* C3 = d >= 3 ? C[2] : &one;
    // stage 1: T1[q3][q2][a1][b1]
    T1.assign((size_t)n3 * n2 * L1 * L1, 0.0);
    for (int q3 = 0; q3 < n3; ++q3)
      for (int q2 = 0; q2 < n2; ++q2) {
        const double* Wq = W + ((size_t)q3 * n2 + q2) * n1;
        double* t = &T1[(((size_t)q3 * n2 + q2) * L1) * L1];
        for (int a1 = 0; a1 < L1; ++a1)
          for (int b1 = 0; b1 < L1; ++b1) {
            double s = 0.0;
            for (int q1 = 0; q1 < n1; ++q1) s += Wq[q1] * R[0][a1 * nq + q1] * C[0][b1 * nq + q1];
            t[a1 * L1 + b1] = s;
          }
      }
    // stage 2: T2[q3][(a2, a1)][(b2, b1)] -- rows and columns in the order of a
    // block of Loc, so that stage 3 is a run of contiguous updates
    const int LL1 = L1 * L1, LB = L1 * L2;       // LB: local functions per (a3) slab
    T2.assign((size_t)n3 * LB * LB, 0.0);
    for (int q3 = 0; q3 < n3; ++q3)
      for (int a2 = 0; a2 < L2; ++a2)
        for (int b2 = 0; b2 < L2; ++b2)
          for (int q2 = 0; q2 < n2; ++q2) {
            const double f = R2[a2 * nq + q2] * C2[b2 * nq + q2];
            if (f == 0.0) continue;
            const double* t1 = &T1[((size_t)q3 * n2 + q2) * LL1];
            for (int a1 = 0; a1 < L1; ++a1) {
              double* __restrict__ t2 = &T2[((size_t)q3 * LB + a2 * L1 + a1) * LB + (size_t)b2 * L1];
              const double* __restrict__ t1r = t1 + a1 * L1;
              for (int b1 = 0; b1 < L1; ++b1) t2[b1] += f * t1r[b1];
            }
          }
    // stage 3: block (a3, b3) of Loc (rows a = r + LB a3, columns c + LB b3) gains
    // sum_q3 R3[a3][q3] C3[b3][q3] T2[q3][r][c]
    const int Ld = P.Ld;
    for (int a3 = 0; a3 < L3; ++a3)
      for (int b3 = 0; b3 < L3; ++b3)
        for (int q3 = 0; q3 < n3; ++q3) {
          const double f3 = R3[a3 * nq + q3] * C3[b3 * nq + q3];
          if (f3 == 0.0) continue;
          const double* t2 = &T2[(size_t)q3 * LB * LB];
          for (int r = 0; r < LB; ++r) {
            double* __restrict__ dst = Loc + (size_t)(r + LB * a3) * Ld + (size_t)LB * b3;
            const double* __restrict__ src = t2 + (size_t)r * LB;
            for (int c = 0; c < LB; ++c) dst[c] += f3 * src[c];
          }
        }
  }
};

// Local mass (if Mloc) and stiffness (if Kloc) of element ei with point
// coefficients c, kappa (nullptr = 1) given per point of this element.
void element_matrices(const Problem& P, const int* ei, const double* c, const double* kappa, double* Mloc,
                      double* Kloc, SumFact& sf, std::vector<double>& x, std::vector<double>& detw,
                      std::vector<double>& Gw, std::vector<double>& W) {
  const int d = P.d, nq = P.nq, L = P.L;
  element_geometry(P, ei, x, detw, Gw);
  const double* V[3];
  const double* D[3];
  for (int l = 0; l < d; ++l) {
    V[l] = &P.tab.V[(size_t)ei[l] * L * nq];
    D[l] = &P.tab.D[(size_t)ei[l] * L * nq];
  }
  W.resize(P.Qe);
  if (Mloc) {
    std::fill(Mloc, Mloc + (size_t)P.Ld * P.Ld, 0.0);
    for (int q = 0; q < P.Qe; ++q) W[q] = detw[q] * (c ? c[q] : 1.0);
    sf.run(P, W.data(), V, V, Mloc);
  }
  if (Kloc) {
    std::fill(Kloc, Kloc + (size_t)P.Ld * P.Ld, 0.0);
    const bool diag = diagonal_metric(P.geom);
    for (int al = 0; al < d; ++al)
      for (int be = 0; be < d; ++be) {
        if (diag && al != be) continue;
        for (int q = 0; q < P.Qe; ++q) W[q] = Gw[(size_t)q * d * d + al * d + be] * (kappa ? kappa[q] : 1.0);
        const double* R[3];
        const double* C[3];
        for (int l = 0; l < d; ++l) {
          R[l] = l == al ? D[l] : V[l];
          C[l] = l == be ? D[l] : V[l];
        }
        sf.run(P, W.data(), R, C, Kloc);
      }
  }
}

int n_threads() {
  const unsigned h = std::thread::hardware_concurrency();
  return (int)std::max(1u, std::min(64u, h));
}

}  // namespace
}  // namespace stfd

using namespace stfd;

extern "C" int stfd_spatial_quadrature_points(int d, int p, int n_el, int geom, int nq, double* x) {
  Problem P;
  if (!problem_init(P, d, p, n_el, geom, nq) || !x) return STFD_ERR_ARG;
  const long long Q = P.n_elem * P.Qe;
  const int nt = (int)std::min<long long>(n_threads(), P.n_elem);
  std::vector<std::thread> th;
  for (int t = 0; t < nt; ++t)
    th.emplace_back([&, t]() {
      std::vector<double> xe, detw, Gw;
      int ei[3];
      for (long long e = t; e < P.n_elem; e += nt) {
        elem_index(P, e, ei);
        element_geometry(P, ei, xe, detw, Gw);
        for (int q = 0; q < P.Qe; ++q)
          for (int a = 0; a < d; ++a) x[(size_t)a * Q + e * P.Qe + q] = xe[(size_t)q * d + a];
      }
    });
  for (auto& t : th) t.join();
  return STFD_OK;
}

extern "C" int stfd_spatial_element_midpoints(int d, int n_el, int geom, double* x) {
  if (d < 1 || d > kMaxDim || n_el < 1 || !x) return STFD_ERR_ARG;
  if (!geom_ok(geom, d)) return STFD_ERR_ARG;
  long long n_elem = 1;
  for (int l = 0; l < d; ++l) n_elem *= n_el;
  double eta[3], xe[3], J[9];
  for (long long e = 0; e < n_elem; ++e) {
    long long r = e;
    for (int l = 0; l < d; ++l) {
      eta[l] = ((double)(r % n_el) + 0.5) / n_el;
      r /= n_el;
    }
    geom_eval(geom, d, eta, xe, J);
    for (int a = 0; a < d; ++a) x[(size_t)a * n_elem + e] = xe[a];
  }
  return STFD_OK;
}

extern "C" int stfd_spatial_assemble(int d, int p, int n_el, int geom, int nq, const double* c_q,
                                     const double* kappa_q, double* Ms, double* Ks) {
  Problem P;
  if (!problem_init(P, d, p, n_el, geom, nq)) return STFD_ERR_ARG;
  if (!Ms && !Ks) return STFD_ERR_ARG;
  int S = 1;
  for (int l = 0; l < d; ++l) S *= 2 * p + 1;
  if (Ms) std::fill(Ms, Ms + (size_t)S * P.Ns, 0.0);
  if (Ks) std::fill(Ks, Ks + (size_t)S * P.Ns, 0.0);
  const int L = P.L, Ld = P.Ld;
  // the stencil offset of local pair (a, b) depends on a and b only:
  // o(a, b) = sum_l (b_l - a_l + p) (2p+1)^(l-1)
  std::vector<int> off_ab((size_t)Ld * Ld);
  for (int a = 0; a < Ld; ++a)
    for (int b = 0; b < Ld; ++b) {
      int ra = a, rb = b, o = 0, so = 1;
      for (int l = 0; l < d; ++l) {
        o += (rb % L - ra % L + p) * so;
        ra /= L;
        rb /= L;
        so *= 2 * p + 1;
      }
      off_ab[(size_t)a * Ld + b] = o;
    }
  // reduced global row of each local function of element ei (-1: removed by the reduction)
  auto local_rows = [&](const int* ei, long long* rows) {
    for (int a = 0; a < Ld; ++a) {
      int ra = a;
      long long row = 0, stride = 1;
      bool ok = true;
      for (int l = 0; l < d; ++l) {
        const int il = ei[l] + ra % L - 1;   // full index e + a minus the dropped first function
        ra /= L;
        if (il < 0 || il >= P.n_s) ok = false;
        row += (long long)il * stride;
        stride *= P.n_s;
      }
      rows[a] = ok ? row : -1;
    }
  };
  auto scatter = [&](const long long* rows, const double* Loc, double* out) {
    for (int a = 0; a < Ld; ++a) {
      if (rows[a] < 0) continue;
      const int* oa = &off_ab[(size_t)a * Ld];
      const double* la = Loc + (size_t)a * Ld;
      for (int b = 0; b < Ld; ++b)
        if (rows[b] >= 0) out[(size_t)oa[b] * P.Ns + rows[a]] += la[b];
    }
  };
  // Colours: elements whose outer indices (directions 2 and 3, or direction 1
  // when d = 1) agree modulo p+1 share no row across different work items.
  // A work item is one line of elements along direction 1 (one element when
  // d = 1); lines of one colour run on separate threads.
  const int nouter = d == 1 ? 1 : d - 1;                 // directions that are coloured
  const long long line = d == 1 ? 1 : n_el;              // elements per work item
  int ncol = 1;
  for (int k = 0; k < nouter; ++k) ncol *= p + 1;
  for (int colour = 0; colour < ncol; ++colour) {
    int cc[2] = {colour % (p + 1), colour / (p + 1)};
    std::vector<long long> items;                        // first element of each line
    if (d == 1) {
      for (int k = cc[0]; k < n_el; k += p + 1) items.push_back(k);
    } else if (d == 2) {
      for (int k = cc[0]; k < n_el; k += p + 1) items.push_back((long long)k * n_el);
    } else {
      for (int k3 = cc[1]; k3 < n_el; k3 += p + 1)
        for (int k2 = cc[0]; k2 < n_el; k2 += p + 1) items.push_back(((long long)k3 * n_el + k2) * n_el);
    }
    const int nt = std::min<int>(n_threads(), (int)items.size());
    std::vector<std::thread> th;
    for (int t = 0; t < nt; ++t)
      th.emplace_back([&, t]() {
        SumFact sf;
        std::vector<double> x, detw, Gw, W, Mloc((size_t)Ld * Ld), Kloc((size_t)Ld * Ld);
        std::vector<long long> rows(Ld);
        int ei[3];
        for (size_t it = t; it < items.size(); it += nt) {
          for (long long r = 0; r < line; ++r) {
            const long long e = items[it] + r;
            elem_index(P, e, ei);
            const double* cq = c_q ? c_q + e * P.Qe : nullptr;
            const double* kq = kappa_q ? kappa_q + e * P.Qe : nullptr;
            element_matrices(P, ei, cq, kq, Ms ? Mloc.data() : nullptr, Ks ? Kloc.data() : nullptr, sf, x, detw, Gw,
                             W);
            local_rows(ei, rows.data());
            if (Ms) scatter(rows.data(), Mloc.data(), Ms);
            if (Ks) scatter(rows.data(), Kloc.data(), Ks);
          }
        }
      });
    for (auto& t : th) t.join();
  }
  return STFD_OK;
}

extern "C" int stfd_spatial_element_stiffness(int d, int p, int n_el, int geom, int nq, double* Ke) {
  Problem P;
  if (!problem_init(P, d, p, n_el, geom, nq) || !Ke) return STFD_ERR_ARG;
  const int Ld = P.Ld;
  const int nt = (int)std::min<long long>(n_threads(), P.n_elem);
  std::vector<std::thread> th;
  for (int t = 0; t < nt; ++t)
    th.emplace_back([&, t]() {
      SumFact sf;
      std::vector<double> x, detw, Gw, W;
      int ei[3];
      for (long long e = t; e < P.n_elem; e += nt) {
        elem_index(P, e, ei);
        element_matrices(P, ei, nullptr, nullptr, nullptr, Ke + (size_t)e * Ld * Ld, sf, x, detw, Gw, W);
      }
    });
  for (auto& t : th) t.join();
  return STFD_OK;
}

extern "C" int stfd_geo_separate(int d, int n_el, int geom, const double* c_mid, const double* kappa_mid,
                                 double* phi, double* Phi) {
  if (d < 1 || d > kMaxDim || n_el < 1 || !phi || !Phi) return STFD_ERR_ARG;
  if (!geom_ok(geom, d)) return STFD_ERR_ARG;
  long long n_elem = 1;
  for (int l = 0; l < d; ++l) n_elem *= n_el;
  // log of the diagonal of frak{C} at the element midpoints: rows 0..d-1
  // stiffness (kappa |det J| [J^{-1} J^{-T}]_ll), row d mass (c |det J|)
  std::vector<double> lg((size_t)(d + 1) * n_elem);
  double eta[3], x[3], J[9], G[9];
  for (long long e = 0; e < n_elem; ++e) {
    long long r = e;
    for (int l = 0; l < d; ++l) {
      eta[l] = ((double)(r % n_el) + 0.5) / n_el;
      r /= n_el;
    }
    geom_eval(geom, d, eta, x, J);
    const double ad = metric(d, J, G);
    const double kv = kappa_mid ? kappa_mid[e] : 1.0, cv = c_mid ? c_mid[e] : 1.0;
    if (!(ad > 0.0) || !(kv > 0.0) || !(cv > 0.0)) return STFD_ERR_ARG;
    for (int l = 0; l < d; ++l) lg[(size_t)l * n_elem + e] = std::log(kv * G[l * d + l]);
    lg[(size_t)d * n_elem + e] = std::log(cv * ad);
  }
  auto idx = [&](long long e, int l) {   // index of element e in direction l
    for (int k = 0; k < l; ++k) e /= n_el;
    return (int)(e % n_el);
  };
  // mass: log phi_l(k) = marginal mean over the other directions - (d-1)/d grand mean
  const double* lm = &lg[(size_t)d * n_elem];
  double grand = 0.0;
  for (long long e = 0; e < n_elem; ++e) grand += lm[e];
  grand /= (double)n_elem;
  std::vector<double> lphi((size_t)d * n_el, 0.0);
  const double per = (double)(n_elem / n_el);
  for (int l = 0; l < d; ++l) {
    for (long long e = 0; e < n_elem; ++e) lphi[(size_t)l * n_el + idx(e, l)] += lm[e];
    for (int k = 0; k < n_el; ++k) lphi[(size_t)l * n_el + k] = lphi[(size_t)l * n_el + k] / per - (d - 1.0) / d * grand;
  }
  // stiffness l: log Phi_l(k) = mean over the others of [log C_l - sum_{m != l} log phi_m]
  for (int l = 0; l < d; ++l) {
    std::vector<double> acc(n_el, 0.0);
    for (long long e = 0; e < n_elem; ++e) {
      double v = lg[(size_t)l * n_elem + e];
      for (int m = 0; m < d; ++m)
        if (m != l) v -= lphi[(size_t)m * n_el + idx(e, m)];
      acc[idx(e, l)] += v;
    }
    for (int k = 0; k < n_el; ++k) {
      Phi[(size_t)l * n_el + k] = std::exp(acc[k] / per);
      phi[(size_t)l * n_el + k] = std::exp(lphi[(size_t)l * n_el + k]);
    }
  }
  return STFD_OK;
}

extern "C" int stfd_spline_matrices_weighted(int p, int n_el, double length, int bc, const double* w_mass,
                                             const double* w_stiff, double* M, double* K, int* n_out) {
  if (p < 1 || p > 30 || n_el < 1 || !(length > 0.0)) return STFD_ERR_ARG;
  const int m = n_el + p;
  int lo = 0, n = -1;
  if (bc == STFD_BC_NONE) n = m;
  if (bc == STFD_BC_INITIAL) { lo = 1; n = m - 1; }
  if (bc == STFD_BC_DIRICHLET) { lo = 1; n = m - 2; }
  if (n < 1) return STFD_ERR_ARG;
  if (n_out) *n_out = n;
  if (!M && !K) return STFD_OK;
  std::vector<double> kv = open_knots(p, n_el, length);
  std::vector<double> fM((size_t)m * m, 0.0), fK((size_t)m * m, 0.0), gx, gw;
  gauss_legendre(p + 1, gx, gw);
  double N[32], dN[32];
  for (int e = 0; e < n_el; ++e) {
    const int k = p + e;
    const double a = kv[k], b = kv[k + 1], half = 0.5 * (b - a);
    const double wm = w_mass ? w_mass[e] : 1.0, ws = w_stiff ? w_stiff[e] : 1.0;
    for (size_t q = 0; q < gx.size(); ++q) {
      const double x = a + half * (gx[q] + 1.0), wq = half * gw[q];
      span_values_derivs(kv, k, p, x, N, dN);
      for (int r = 0; r <= p; ++r)
        for (int c = 0; c <= p; ++c) {
          const size_t ij = (size_t)(k - p + r) + (size_t)m * (k - p + c);
          fM[ij] += wm * wq * N[r] * N[c];
          fK[ij] += ws * wq * dN[r] * dN[c];
        }
    }
  }
  for (int j = 0; j < n; ++j)
    for (int i = 0; i < n; ++i) {
      const size_t src = (size_t)(i + lo) + (size_t)m * (j + lo), dst = (size_t)i + (size_t)n * j;
      if (M) M[dst] = fM[src];
      if (K) K[dst] = fK[src];
    }
  return STFD_OK;
}
