// Step 3 of Algorithm 1 in double-float arithmetic for one spatial index k:
// the real 2 x 2-block arrowhead solve of the Remark in Sec. 4.5 with
// a = nu mu_k, H_j = [[a, b_j], [-b_j, a]], b_j = gamma lam_j, coupling gamma g
// (signs flipped for the transposed system), Schur reciprocal S_k^{-1}.
// Shared by the per-problem kernel (fd_df.cu) and the batched one (batch.cu).
#pragma once
#include "df.cuh"

namespace stfd {

struct ArrowDF {
  int d, n1, n2, nt, n_pairs, has_zero;
  long long Ns;
  const float2* lam[3];   // spatial eigenvalues
  const float2* B;        // gamma lam_j per pair
  const float2* BB;       // (gamma lam_j)^2 per pair
  const float2* G;        // gamma g, nt - 1 entries
  const float2* Sinv;     // Ns
  float2 nu;
  float sgn;              // +1: Delta_t, -1: Delta_t^T
};

__device__ __forceinline__ dfa::df sgnd(float2 v, float sgn) { return dfa::df{v.x * sgn, v.y * sgn}; }

__device__ __forceinline__ void arrowhead_df_point(float2* __restrict__ X, const ArrowDF& p, long long k) {
  using dfa::df;
  const long long Ns = p.Ns;
  long long rest = k;
  const int i1 = (int)(rest % p.n1);
  rest /= p.n1;
  df mu = dfa::from_float2(p.lam[0][i1]);
  if (p.d >= 2) {
    const int i2 = (int)(rest % p.n2);
    rest /= p.n2;
    mu = dfa::add(mu, dfa::from_float2(p.lam[1][i2]));
  }
  if (p.d >= 3) mu = dfa::add(mu, dfa::from_float2(p.lam[2][rest]));
  const df a = dfa::mul(dfa::from_float2(p.nu), mu);
  const df a2 = dfa::mul(a, a);
  df y = dfa::from_float2(X[(long long)(p.nt - 1) * Ns + k]);
  for (int j = 0; j < p.n_pairs; ++j) {
    const df x1 = dfa::from_float2(X[(long long)(2 * j) * Ns + k]);
    const df x2 = dfa::from_float2(X[(long long)(2 * j + 1) * Ns + k]);
    const df b = sgnd(p.B[j], p.sgn);
    const df inv = dfa::recip(dfa::add(a2, dfa::from_float2(p.BB[j])));
    const df h1 = dfa::mul(dfa::sub(dfa::mul(a, x1), dfa::mul(b, x2)), inv);
    const df h2 = dfa::mul(dfa::add(dfa::mul(b, x1), dfa::mul(a, x2)), inv);
    y = dfa::add(y, dfa::add(dfa::mul(sgnd(p.G[2 * j], p.sgn), h1), dfa::mul(sgnd(p.G[2 * j + 1], p.sgn), h2)));
  }
  const int z = 2 * p.n_pairs;
  df x0{0.f, 0.f}, inva{0.f, 0.f};
  if (p.has_zero) {
    x0 = dfa::from_float2(X[(long long)z * Ns + k]);
    inva = dfa::recip(a);
    y = dfa::add(y, dfa::mul(sgnd(p.G[z], p.sgn), dfa::mul(x0, inva)));
  }
  const df qn = dfa::mul(y, dfa::from_float2(p.Sinv[k]));
  X[(long long)(p.nt - 1) * Ns + k] = make_float2(qn.h, qn.l);
  for (int j = 0; j < p.n_pairs; ++j) {
    const long long o1 = (long long)(2 * j) * Ns + k, o2 = (long long)(2 * j + 1) * Ns + k;
    const df b = sgnd(p.B[j], p.sgn);
    const df inv = dfa::recip(dfa::add(a2, dfa::from_float2(p.BB[j])));
    const df r1 = dfa::sub(dfa::from_float2(X[o1]), dfa::mul(sgnd(p.G[2 * j], p.sgn), qn));
    const df r2 = dfa::sub(dfa::from_float2(X[o2]), dfa::mul(sgnd(p.G[2 * j + 1], p.sgn), qn));
    const df q1 = dfa::mul(dfa::sub(dfa::mul(a, r1), dfa::mul(b, r2)), inv);
    const df q2 = dfa::mul(dfa::add(dfa::mul(b, r1), dfa::mul(a, r2)), inv);
    X[o1] = make_float2(q1.h, q1.l);
    X[o2] = make_float2(q2.h, q2.l);
  }
  if (p.has_zero) {
    const df q0 = dfa::mul(dfa::sub(x0, dfa::mul(sgnd(p.G[z], p.sgn), qn)), inva);
    X[(long long)z * Ns + k] = make_float2(q0.h, q0.l);
  }
}

}  // namespace stfd
