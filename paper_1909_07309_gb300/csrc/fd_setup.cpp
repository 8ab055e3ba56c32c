// Step 1 of Algorithm 1 on the host: the spatial generalised eigenproblems
// (eq. space_eig) and the arrowhead factorisation of the time pencil
// (Sec. 4.2.2) in the real form of the Remark in Sec. 4.5.
//
// Dense kernels written for this library (no LAPACK on the target image):
// Cholesky, cyclic Jacobi for real symmetric matrices, and cyclic Jacobi for
// complex Hermitian matrices. Sizes are at most 256, so O(n^3) sweeps cost
// milliseconds and run once per handle.
#include <algorithm>
#include <cmath>
#include <complex>
#include <numeric>
#include <vector>

#include "stfd.h"
#include "stfd_internal.h"

namespace stfd {
namespace {

using cplx = std::complex<double>;
constexpr double kEps = 2.220446049250313e-16;

// A = L L^T, A column-major n x n, L lower (column-major). false if not SPD.
bool cholesky(int n, const double* A, std::vector<double>& L) {
  L.assign((size_t)n * n, 0.0);
  for (int j = 0; j < n; ++j) {
    double s = A[j + (size_t)n * j];
    for (int k = 0; k < j; ++k) s -= L[j + (size_t)n * k] * L[j + (size_t)n * k];
    if (!(s > 0.0)) return false;
    const double ljj = std::sqrt(s);
    L[j + (size_t)n * j] = ljj;
    for (int i = j + 1; i < n; ++i) {
      double t = A[i + (size_t)n * j];
      for (int k = 0; k < j; ++k) t -= L[i + (size_t)n * k] * L[j + (size_t)n * k];
      L[i + (size_t)n * j] = t / ljj;
    }
  }
  return true;
}

// Inverse of a lower-triangular L (column-major) by forward substitution.
std::vector<double> lower_inverse(int n, const std::vector<double>& L) {
  std::vector<double> X((size_t)n * n, 0.0);
  for (int c = 0; c < n; ++c) {
    for (int i = c; i < n; ++i) {
      double t = (i == c) ? 1.0 : 0.0;
      for (int k = c; k < i; ++k) t -= L[i + (size_t)n * k] * X[k + (size_t)n * c];
      X[i + (size_t)n * c] = t / L[i + (size_t)n * i];
    }
  }
  return X;
}

// C = A * B for column-major n x n; tA / tB transpose the operand.
std::vector<double> matmul(int n, const double* A, bool tA, const double* B, bool tB) {
  std::vector<double> C((size_t)n * n, 0.0);
  for (int j = 0; j < n; ++j)
    for (int k = 0; k < n; ++k) {
      const double b = tB ? B[j + (size_t)n * k] : B[k + (size_t)n * j];
      if (b == 0.0) continue;
      for (int i = 0; i < n; ++i) C[i + (size_t)n * j] += (tA ? A[k + (size_t)n * i] : A[i + (size_t)n * k]) * b;
    }
  return C;
}

// Cyclic Jacobi for a real symmetric A (overwritten): A = V diag(w) V^T.
bool jacobi_symmetric(int n, std::vector<double>& A, std::vector<double>& V, std::vector<double>& w) {
  V.assign((size_t)n * n, 0.0);
  for (int i = 0; i < n; ++i) V[i + (size_t)n * i] = 1.0;
  double fro = 0.0;
  for (double x : A) fro += x * x;
  const double floor_abs = 1e-19 * std::sqrt(fro);
  bool ok = false;
  for (int sweep = 0; sweep < 100 && !ok; ++sweep) {
    int rotations = 0;
    for (int p = 0; p < n - 1; ++p)
      for (int q = p + 1; q < n; ++q) {
        const double apq = A[p + (size_t)n * q];
        // rotate only while the coupling exceeds the relative-accuracy threshold
        const double thr = std::max(kEps * std::sqrt(std::fabs(A[p + (size_t)n * p] * A[q + (size_t)n * q])), floor_abs);
        if (!(std::fabs(apq) > thr)) continue;
        ++rotations;
        const double app = A[p + (size_t)n * p], aqq = A[q + (size_t)n * q];
        const double theta = (aqq - app) / (2.0 * apq);
        const double t = (theta >= 0 ? 1.0 : -1.0) / (std::fabs(theta) + std::sqrt(theta * theta + 1.0));
        const double c = 1.0 / std::sqrt(1.0 + t * t), s = t * c;
        for (int k = 0; k < n; ++k) {   // columns p, q of A P
          const double akp = A[k + (size_t)n * p], akq = A[k + (size_t)n * q];
          A[k + (size_t)n * p] = c * akp - s * akq;
          A[k + (size_t)n * q] = s * akp + c * akq;
        }
        for (int k = 0; k < n; ++k) {   // rows p, q of P^T (A P)
          const double apk = A[p + (size_t)n * k], aqk = A[q + (size_t)n * k];
          A[p + (size_t)n * k] = c * apk - s * aqk;
          A[q + (size_t)n * k] = s * apk + c * aqk;
        }
        for (int k = 0; k < n; ++k) {
          const double vkp = V[k + (size_t)n * p], vkq = V[k + (size_t)n * q];
          V[k + (size_t)n * p] = c * vkp - s * vkq;
          V[k + (size_t)n * q] = s * vkp + c * vkq;
        }
      }
    ok = (rotations == 0);
  }
  w.resize(n);
  for (int i = 0; i < n; ++i) w[i] = A[i + (size_t)n * i];
  return ok;
}

// Cyclic Jacobi for a complex Hermitian H (overwritten): H = Z diag(w) Z^*.
// Each pivot first removes the phase of h_pq with diag(1, e^{-i phi}), then a
// real rotation annihilates the now real symmetric 2 x 2 block.
bool jacobi_hermitian(int n, std::vector<cplx>& H, std::vector<cplx>& Z, std::vector<double>& w) {
  Z.assign((size_t)n * n, cplx(0.0, 0.0));
  for (int i = 0; i < n; ++i) Z[i + (size_t)n * i] = 1.0;
  double fro = 0.0;
  for (const cplx& x : H) fro += std::norm(x);
  const double floor_abs = 1e-19 * std::sqrt(fro);
  bool ok = false;
  for (int sweep = 0; sweep < 100 && !ok; ++sweep) {
    int rotations = 0;
    for (int p = 0; p < n - 1; ++p)
      for (int q = p + 1; q < n; ++q) {
        const cplx hpq = H[p + (size_t)n * q];
        const double e = std::abs(hpq);
        const double thr = std::max(kEps * std::sqrt(std::fabs(H[p + (size_t)n * p].real() * H[q + (size_t)n * q].real())),
                                    floor_abs);
        if (!(e > thr)) continue;
        ++rotations;
        const cplx ph = hpq / e;                    // e^{i phi}
        const cplx phc = std::conj(ph);             // e^{-i phi}
        const double a = H[p + (size_t)n * p].real(), b = H[q + (size_t)n * q].real();
        const double theta = (b - a) / (2.0 * e);
        const double t = (theta >= 0 ? 1.0 : -1.0) / (std::fabs(theta) + std::sqrt(theta * theta + 1.0));
        const double cs = 1.0 / std::sqrt(1.0 + t * t), sn = t * cs;
        // G = diag(1, e^{-i phi}) [[cs, sn], [-sn, cs]]
        const cplx g11 = cs, g12 = sn, g21 = -sn * phc, g22 = cs * phc;
        for (int k = 0; k < n; ++k) {
          const cplx hp = H[k + (size_t)n * p], hq = H[k + (size_t)n * q];
          H[k + (size_t)n * p] = hp * g11 + hq * g21;
          H[k + (size_t)n * q] = hp * g12 + hq * g22;
        }
        for (int k = 0; k < n; ++k) {
          const cplx hp = H[p + (size_t)n * k], hq = H[q + (size_t)n * k];
          H[p + (size_t)n * k] = std::conj(g11) * hp + std::conj(g21) * hq;
          H[q + (size_t)n * k] = std::conj(g12) * hp + std::conj(g22) * hq;
        }
        for (int k = 0; k < n; ++k) {
          const cplx zp = Z[k + (size_t)n * p], zq = Z[k + (size_t)n * q];
          Z[k + (size_t)n * p] = zp * g11 + zq * g21;
          Z[k + (size_t)n * q] = zp * g12 + zq * g22;
        }
      }
    ok = (rotations == 0);
  }
  w.resize(n);
  for (int i = 0; i < n; ++i) w[i] = H[i + (size_t)n * i].real();
  return ok;
}

// K U = M U Lambda, U^T M U = I: with M = L L^T and L^{-1} K L^{-T} = Q diag Q^T,
// U = L^{-T} Q (eigenvalues ascending).
int spatial_factor(int n, const double* K, const double* M, std::vector<double>& U, std::vector<double>& lam) {
  std::vector<double> L;
  if (!cholesky(n, M, L)) return STFD_ERR_NOT_SPD;
  std::vector<double> Li = lower_inverse(n, L);
  std::vector<double> T = matmul(n, Li.data(), false, K, false);
  std::vector<double> C = matmul(n, T.data(), false, Li.data(), true);
  for (int j = 0; j < n; ++j)
    for (int i = 0; i < j; ++i) {
      const double s = 0.5 * (C[i + (size_t)n * j] + C[j + (size_t)n * i]);
      C[i + (size_t)n * j] = C[j + (size_t)n * i] = s;
    }
  std::vector<double> Q, w;
  if (!jacobi_symmetric(n, C, Q, w)) return STFD_ERR_EIG;
  std::vector<int> order(n);
  std::iota(order.begin(), order.end(), 0);
  std::sort(order.begin(), order.end(), [&](int x, int y) { return w[x] < w[y]; });
  std::vector<double> Qs((size_t)n * n);
  lam.resize(n);
  for (int c = 0; c < n; ++c) {
    lam[c] = w[order[c]];
    for (int i = 0; i < n; ++i) Qs[i + (size_t)n * c] = Q[i + (size_t)n * order[c]];
  }
  U = matmul(n, Li.data(), true, Qs.data(), false);
  return STFD_OK;
}

// Arrowhead factorisation of (W_t, M_t), real form (Sec. 4.2.2 and the Remark
// of Sec. 4.5). Column order of U_t: the q pairs (2 columns each), then the
// zero block if n_t - 1 is odd, then the arrow column [r; rho].
int time_factor(int nt, const double* Wt, const double* Mt, HostFactors& f) {
  const int n0 = nt - 1;
  std::vector<double> W0((size_t)n0 * n0), M0((size_t)n0 * n0), w(n0), m(n0);
  for (int j = 0; j < n0; ++j) {
    for (int i = 0; i < n0; ++i) {
      W0[i + (size_t)n0 * j] = Wt[i + (size_t)nt * j];
      M0[i + (size_t)n0 * j] = Mt[i + (size_t)nt * j];
    }
    w[j] = Wt[j + (size_t)nt * n0];     // eq. split: last column of W_t
    m[j] = Mt[j + (size_t)nt * n0];
  }
  std::vector<double> L;
  if (!cholesky(n0, M0.data(), L)) return STFD_ERR_NOT_SPD;
  std::vector<double> Li = lower_inverse(n0, L);
  std::vector<double> T = matmul(n0, Li.data(), false, W0.data(), false);
  std::vector<double> S = matmul(n0, T.data(), false, Li.data(), true);
  // W0 is skew-symmetric (eq. integral_W); keep S exactly skew.
  for (int j = 0; j < n0; ++j)
    for (int i = 0; i <= j; ++i) {
      const double s = (i == j) ? 0.0 : 0.5 * (S[i + (size_t)n0 * j] - S[j + (size_t)n0 * i]);
      S[i + (size_t)n0 * j] = s;
      S[j + (size_t)n0 * i] = -s;
    }
  // i S is Hermitian: i S z = theta z  <=>  S z = -i theta z. With z = a + i b
  // and theta > 0: S a = theta b, S b = -theta a, so the real pair
  // (sqrt2 b, sqrt2 a) spans an invariant plane where S acts as
  // [[0, theta], [-theta, 0]] -- the 2 x 2 block of the Remark (lam_j = theta).
  std::vector<cplx> H((size_t)n0 * n0), Z;
  for (size_t k = 0; k < H.size(); ++k) H[k] = cplx(0.0, S[k]);
  std::vector<double> theta;
  if (!jacobi_hermitian(n0, H, Z, theta)) return STFD_ERR_EIG;
  double tmax = 0.0;
  for (double t : theta) tmax = std::max(tmax, std::fabs(t));
  const double tol = 1e-8 * std::max(tmax, 1e-300);
  std::vector<int> pos, zer;
  int nneg = 0;
  for (int k = 0; k < n0; ++k) {
    if (theta[k] > tol) pos.push_back(k);
    else if (theta[k] < -tol) ++nneg;
    else zer.push_back(k);
  }
  if ((int)pos.size() != nneg || (int)zer.size() != (n0 % 2)) return STFD_ERR_EIG;
  std::sort(pos.begin(), pos.end(), [&](int x, int y) { return theta[x] < theta[y]; });
  std::vector<double> Q((size_t)n0 * n0, 0.0);
  int col = 0;
  const double r2 = std::sqrt(2.0);
  for (int k : pos) {
    for (int i = 0; i < n0; ++i) {
      Q[i + (size_t)n0 * col] = r2 * Z[i + (size_t)n0 * k].imag();
      Q[i + (size_t)n0 * (col + 1)] = r2 * Z[i + (size_t)n0 * k].real();
    }
    col += 2;
  }
  if (!zer.empty()) {   // null vector of S: rotate the phase so it is real
    const int k = zer[0];
    int imax = 0;
    for (int i = 1; i < n0; ++i)
      if (std::abs(Z[i + (size_t)n0 * k]) > std::abs(Z[imax + (size_t)n0 * k])) imax = i;
    const cplx ph = std::conj(Z[imax + (size_t)n0 * k]) / std::abs(Z[imax + (size_t)n0 * k]);
    double nrm = 0.0;
    for (int i = 0; i < n0; ++i) {
      const double v = (Z[i + (size_t)n0 * k] * ph).real();
      Q[i + (size_t)n0 * col] = v;
      nrm += v * v;
    }
    nrm = std::sqrt(nrm);
    for (int i = 0; i < n0; ++i) Q[i + (size_t)n0 * col] /= nrm;
    ++col;
  }
  // U0 = L^{-T} Q: M0-orthonormal, U0^T W0 U0 = blockdiag (eq. factorization_first_block)
  std::vector<double> U0 = matmul(n0, Li.data(), true, Q.data(), false);
  std::vector<double> D0 = matmul(n0, U0.data(), true, matmul(n0, W0.data(), false, U0.data(), false).data(), false);
  f.n_pairs = (int)pos.size();
  f.has_zero = (int)zer.size();
  f.lamt.resize(f.n_pairs);
  // scale of U0^T W0 U0: max |W_t| * max |U0|^2 * n0 bounds every entry
  double wmax = 0.0, umax = 0.0;
  for (size_t k = 0; k < (size_t)nt * nt; ++k) wmax = std::max(wmax, std::fabs(Wt[k]));
  for (double x : U0) umax = std::max(umax, std::fabs(x));
  const double dmax = std::max(wmax * umax * umax * n0, 1e-300);
  for (int j = 0; j < f.n_pairs; ++j)
    f.lamt[j] = 0.5 * (D0[2 * j + (size_t)n0 * (2 * j + 1)] - D0[2 * j + 1 + (size_t)n0 * (2 * j)]);
  // structure check: everything outside the 2 x 2 blocks must vanish
  for (int j = 0; j < n0; ++j)
    for (int i = 0; i < n0; ++i) {
      const bool in_block = (i / 2 == j / 2) && (i < 2 * f.n_pairs) && (j < 2 * f.n_pairs);
      const bool diag_pair = in_block && i != j;
      if (!diag_pair && std::fabs(D0[i + (size_t)n0 * j]) > 1e-9 * dmax) return STFD_ERR_EIG;
    }
  // eq. syst_v: M0 v = -m, then normalise [v; 1] in the M_t norm
  std::vector<double> v(n0), y(n0);
  for (int i = 0; i < n0; ++i) {        // L y = -m
    double t = -m[i];
    for (int k = 0; k < i; ++k) t -= L[i + (size_t)n0 * k] * y[k];
    y[i] = t / L[i + (size_t)n0 * i];
  }
  for (int i = n0 - 1; i >= 0; --i) {   // L^T v = y
    double t = y[i];
    for (int k = i + 1; k < n0; ++k) t -= L[k + (size_t)n0 * i] * v[k];
    v[i] = t / L[i + (size_t)n0 * i];
  }
  std::vector<double> vv(nt);
  for (int i = 0; i < n0; ++i) vv[i] = v[i];
  vv[n0] = 1.0;
  double q = 0.0;
  for (int j = 0; j < nt; ++j)
    for (int i = 0; i < nt; ++i) q += vv[i] * Mt[i + (size_t)nt * j] * vv[j];
  if (!(q > 0.0)) return STFD_ERR_NOT_SPD;
  const double nrm = std::sqrt(q);
  std::vector<double> rr(nt);
  for (int i = 0; i < nt; ++i) rr[i] = vv[i] / nrm;   // [r; rho]
  // U_t = [[U0, r], [0, rho]]   (eq. U_t)
  f.Ut.assign((size_t)nt * nt, 0.0);
  for (int j = 0; j < n0; ++j)
    for (int i = 0; i < n0; ++i) f.Ut[i + (size_t)nt * j] = U0[i + (size_t)n0 * j];
  for (int i = 0; i < nt; ++i) f.Ut[i + (size_t)nt * n0] = rr[i];
  // eq. time_eig_2: g = U0^T [W0 w] [r; rho],  sigma = [r; rho]^T W_t [r; rho]
  std::vector<double> Wr(n0, 0.0);
  for (int i = 0; i < n0; ++i) {
    double t = w[i] * rr[n0];
    for (int k = 0; k < n0; ++k) t += W0[i + (size_t)n0 * k] * rr[k];
    Wr[i] = t;
  }
  f.g.assign(n0, 0.0);
  for (int j = 0; j < n0; ++j) {
    double t = 0.0;
    for (int i = 0; i < n0; ++i) t += U0[i + (size_t)n0 * j] * Wr[i];
    f.g[j] = t;
  }
  double s = 0.0;
  for (int j = 0; j < nt; ++j)
    for (int i = 0; i < nt; ++i) s += rr[i] * Wt[i + (size_t)nt * j] * rr[j];
  f.sigma = s;
  return STFD_OK;
}

}  // namespace

int factorize_host(int d, const int* n, const double* const* K, const double* const* M,
                   const double* Wt, const double* Mt, HostFactors& f) {
  if (d < 1 || d > kMaxDim || !n || !K || !M || !Wt || !Mt) return STFD_ERR_ARG;
  for (int l = 0; l < d; ++l)
    if (n[l] < 1 || n[l] > kMaxN || !K[l] || !M[l]) return STFD_ERR_ARG;
  if (n[d] < 2 || n[d] > kMaxN) return STFD_ERR_ARG;
  f.d = d;
  for (int l = 0; l <= d; ++l) f.n[l] = n[l];
  for (int l = 0; l < d; ++l) {
    const int rc = spatial_factor(n[l], K[l], M[l], f.U[l], f.lam[l]);
    if (rc != STFD_OK) return rc;
  }
  return time_factor(n[d], Wt, Mt, f);
}

}  // namespace stfd

extern "C" int stfd_fd_factors(int d, const int* n, const double* const* K, const double* const* M,
                               const double* Wt, const double* Mt,
                               double* const* U, double* const* lam, double* Ut, double* lamt,
                               double* g, double* sigma, int* n_pairs, int* has_zero) {
  stfd::HostFactors f;
  const int rc = stfd::factorize_host(d, n, K, M, Wt, Mt, f);
  if (rc != STFD_OK) return rc;
  for (int l = 0; l < d; ++l) {
    if (U && U[l]) std::copy(f.U[l].begin(), f.U[l].end(), U[l]);
    if (lam && lam[l]) std::copy(f.lam[l].begin(), f.lam[l].end(), lam[l]);
  }
  if (Ut) std::copy(f.Ut.begin(), f.Ut.end(), Ut);
  if (lamt) std::copy(f.lamt.begin(), f.lamt.end(), lamt);
  if (g) std::copy(f.g.begin(), f.g.end(), g);
  if (sigma) *sigma = f.sigma;
  if (n_pairs) *n_pairs = f.n_pairs;
  if (has_zero) *has_zero = f.has_zero;
  return STFD_OK;
}

namespace stfd {

// Reciprocals of the Schur complement of the arrowhead per spatial index
// (eq. block_LU): with a = nu mu_k,
// S_k = gamma sigma + a + sum_j gamma^2 a |g_j|^2 / (a^2 + gamma^2 lam_j^2) [+ gamma^2 g_z^2 / a].
std::vector<double> schur_reciprocals(const HostFactors& f, double gamma, double nu) {
  long long Ns = 1;
  for (int l = 0; l < f.d; ++l) Ns *= f.n[l];
  std::vector<double> Sinv((size_t)Ns);
  for (long long k = 0; k < Ns; ++k) {
    long long rest = k;
    double mu = 0.0;
    for (int l = 0; l < f.d; ++l) {
      mu += f.lam[l][rest % f.n[l]];
      rest /= f.n[l];
    }
    const double a = nu * mu;
    double S = gamma * f.sigma + a;
    for (int j = 0; j < f.n_pairs; ++j) {
      const double b = gamma * f.lamt[j];
      const double g2 = f.g[2 * j] * f.g[2 * j] + f.g[2 * j + 1] * f.g[2 * j + 1];
      S += gamma * gamma * a * g2 / (a * a + b * b);
    }
    if (f.has_zero) S += gamma * gamma * f.g[2 * f.n_pairs] * f.g[2 * f.n_pairs] / a;
    Sinv[k] = 1.0 / S;
  }
  return Sinv;
}

}  // namespace stfd
