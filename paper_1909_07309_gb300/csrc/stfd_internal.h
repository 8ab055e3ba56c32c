// Internal declarations shared by the host and device translation units.
#pragma once
#include <cstdint>
#include <vector>

namespace stfd {

constexpr int kMaxDim = 3;       // spatial dimensions d in {1, 2, 3}
constexpr int kMaxN = 256;       // largest univariate size n_l / n_t

std::vector<double> open_knots(int p, int n_el, double L);
void gauss_legendre(int nq, std::vector<double>& x, std::vector<double>& w);
// Values N[0..p] and derivatives dN[0..p] of b_{k-p..k} at x in knot span k.
void span_values_derivs(const std::vector<double>& kv, int k, int p, double x, double* N, double* dN);

// Host factorisation of Step 1 of Algorithm 1 (real form). Column-major.
struct HostFactors {
  int d = 0;
  int n[kMaxDim + 1] = {0, 0, 0, 0};
  std::vector<double> U[kMaxDim];     // n_l x n_l
  std::vector<double> lam[kMaxDim];   // n_l
  std::vector<double> Ut;             // n_t x n_t
  std::vector<double> lamt;           // n_pairs
  std::vector<double> g;              // n_t - 1
  double sigma = 0.0;
  int n_pairs = 0;
  int has_zero = 0;
};

int factorize_host(int d, const int* n, const double* const* K, const double* const* M,
                   const double* Wt, const double* Mt, HostFactors& f);

// S_k^{-1} of eq. block_LU for every spatial index k.
std::vector<double> schur_reciprocals(const HostFactors& f, double gamma, double nu);

}  // namespace stfd
