// C ABI: handles, Algorithm 1 (fd_apply), the Kronecker system matvec and the
// flexible GMRES driver. Every step of the numerical path runs in the device
// kernels of kernels.cu; the host only factorises once (fd_setup.cpp), drives
// the launches and does the (restart+1) x restart Hessenberg/Givens work.
#include <cuda_runtime.h>

#include <algorithm>
#include <cmath>
#include <cstring>
#include <new>
#include <vector>

#include "device_state.h"
#include "kernels.h"
#include "stfd.h"
#include "stfd_internal.h"

using namespace stfd;

namespace {

#define STFD_CU(x)                                   \
  do {                                               \
    if ((x) != cudaSuccess) return STFD_ERR_CUDA;    \
  } while (0)

template <class T>
int dev_upload(T** dst, const T* src, size_t count, cudaStream_t st) {
  *dst = nullptr;
  if (count == 0) return STFD_OK;
  if (cudaMalloc((void**)dst, count * sizeof(T)) != cudaSuccess) {
    *dst = nullptr;
    return STFD_ERR_ALLOC;
  }
  if (src && cudaMemcpyAsync(*dst, src, count * sizeof(T), cudaMemcpyHostToDevice, st) != cudaSuccess)
    return STFD_ERR_CUDA;
  return STFD_OK;
}

void dev_free(void* p) {
  if (p) cudaFree(p);
}

// Row-major J[i*n + a] = A[i, a] from a column-major host matrix A.
std::vector<double> row_major(int n, const double* A) {
  std::vector<double> J((size_t)n * n);
  for (int i = 0; i < n; ++i)
    for (int a = 0; a < n; ++a) J[(size_t)i * n + a] = A[i + (size_t)n * a];
  return J;
}

int bandwidth(int n, const double* A) {
  int bw = 0;
  for (int j = 0; j < n; ++j)
    for (int i = 0; i < n; ++i)
      if (A[i + (size_t)n * j] != 0.0) bw = std::max(bw, std::abs(i - j));
  return bw;
}

bool sizes_ok(int d, const int* n) {
  if (d < 1 || d > kMaxDim || !n) return false;
  for (int l = 0; l < d; ++l)
    if (n[l] < 1 || n[l] > kMaxN) return false;
  return n[d] >= 2 && n[d] <= kMaxN;
}

}  // namespace

struct stfd_fd {
  int d = 0;
  int n[kMaxDim + 1] = {0, 0, 0, 0};
  long long Ns = 0, N = 0;
  double gamma = 1.0, nu = 1.0;
  int precision = STFD_FP64;
  double* Jf[kMaxDim + 1] = {nullptr, nullptr, nullptr, nullptr};  // U_l^T, U_t^T (row-major J)
  double* Jb[kMaxDim + 1] = {nullptr, nullptr, nullptr, nullptr};  // U_l,   U_t
  double* lam[kMaxDim] = {nullptr, nullptr, nullptr};
  double* lamt = nullptr;
  double* g = nullptr;
  double* Sinv = nullptr;
  double* work = nullptr;
  // FP64 Step 3 (STFD_FP64, STFD_FP64TC7): complex reciprocals w_jk, about one
  // N-vector (n_pairs x N_s double2), and G = gamma g
  double2* wtab = nullptr;
  double* Gg = nullptr;
  int n_pairs = 0, has_zero = 0;
  double sigma = 0.0;
  // low-precision path (STFD_TF32 / STFD_BF16): operand images of U^T / U and FP32 copies
  unsigned char* Bf[kMaxDim + 1] = {nullptr, nullptr, nullptr, nullptr};
  unsigned char* Bb[kMaxDim + 1] = {nullptr, nullptr, nullptr, nullptr};
  float* lam_f[kMaxDim] = {nullptr, nullptr, nullptr};
  float* lamt_f = nullptr;
  float* g_f = nullptr;
  float* Sinv_f = nullptr;
  // double-float path (STFD_DF32): (hi, lo) factors and arrowhead data
  float2* Jf2[kMaxDim + 1] = {nullptr, nullptr, nullptr, nullptr};
  float2* Jb2[kMaxDim + 1] = {nullptr, nullptr, nullptr, nullptr};
  float2* lam2[kMaxDim] = {nullptr, nullptr, nullptr};
  float2* B2 = nullptr;
  float2* BB2 = nullptr;
  float2* G2 = nullptr;
  float2* Sinv2 = nullptr;
  // tensor-core FP64-accurate path (STFD_FP64TC): digit planes and row scales of U^T / U
  // (STFD_FP64TC7: seven-digit planes and row exponents, same fields)
  unsigned char* Zf[kMaxDim + 1] = {nullptr, nullptr, nullptr, nullptr};
  unsigned char* Zb[kMaxDim + 1] = {nullptr, nullptr, nullptr, nullptr};
  int* zvf[kMaxDim + 1] = {nullptr, nullptr, nullptr, nullptr};
  int* zvb[kMaxDim + 1] = {nullptr, nullptr, nullptr, nullptr};
  // diagonals of the univariate factors (host), for the scaling of eq. prec_geo
  std::vector<double> diagM[kMaxDim], diagK[kMaxDim], diagWt, diagMt;
  double* dscale = nullptr;   // D^{-1/2} per dof (device), or nullptr
  double* work2 = nullptr;    // scaled right-hand side
  // double-float paths (STFD_DF32, STFD_FP64TC): exact power-of-two range scaling
  double* work3 = nullptr;    // the range-scaled input
  int* bexp = nullptr;        // its exponent (device)
};

struct GmresWork {
  std::vector<double*> V, Z;     // device N-vectors
  double** dV = nullptr;         // device copy of the V pointers (capacity cap_v)
  double** dZ = nullptr;
  int cap_v = 0, cap_z = 0;
  double* partial = nullptr;     // dot_blocks() * (restart + 1)
  int partial_cap = 0;
  double* h = nullptr;           // 2 restart + 6: h, h2, ||w||^2
  double* hostbuf = nullptr;     // pinned, device-mapped mirror of h
  double* hostbuf_dev = nullptr; // its device address
  int hcap = 0;
};

struct stfd_op {
  int d = 0;
  int n[kMaxDim + 1] = {0, 0, 0, 0};
  long long N = 0;
  double gamma = 1.0, nu = 1.0;
  double* JM[kMaxDim] = {nullptr, nullptr, nullptr};
  double* JK[kMaxDim] = {nullptr, nullptr, nullptr};
  int bwM[kMaxDim] = {0, 0, 0}, bwK[kMaxDim] = {0, 0, 0};
  double* JW = nullptr;
  double* JWT = nullptr;   // W_t^T, for A^T
  double* JMt = nullptr;
  int bwW = 0, bwMt = 0;
  double* tmp[4] = {nullptr, nullptr, nullptr, nullptr};
  double* tmp5 = nullptr;   // range-scaled input of the double-float matvec
  int* bexp = nullptr;
  GmresWork* gw = nullptr;
  int arith = STFD_OP_FP64;
  // double-float factors (hi, lo) for STFD_OP_DF32
  float2* JM2[kMaxDim] = {nullptr, nullptr, nullptr};
  float2* JK2[kMaxDim] = {nullptr, nullptr, nullptr};
  float2* JW2 = nullptr;
  float2* JWT2 = nullptr;
  float2* JMt2 = nullptr;
  // band-compressed double-float factors Ab[i][t] = A[i][i-p+t] (when every p <= 4):
  // K_l as (hi, lo) for the scalar chain of the middle directions
  int pb[kMaxDim + 1] = {0, 0, 0, 0};
  bool banded = false;
  float2* Kb[kMaxDim] = {nullptr, nullptr, nullptr};
  // the same bands as coefficient pairs (hi_1, hi_2, lo_1, lo_2) for the paired kernels:
  // (M_l, K_l), (M_l, M_l), (W_t, M_t), (W_t^T, M_t)
  float4* MK4[kMaxDim] = {nullptr, nullptr, nullptr};
  float4* MM4[kMaxDim] = {nullptr, nullptr, nullptr};
  float4* WMt4 = nullptr;
  float4* WTMt4 = nullptr;
  // STFD_OP_FX64: integer-limb band tables per direction (M, K) and for the time
  // pass (gamma W, nu M_t) and (gamma W^T, nu M_t), with the row exponents
  bool fx = false;
  int2* FXC[kMaxDim + 2] = {nullptr, nullptr, nullptr, nullptr, nullptr};
  int* FXE[kMaxDim + 2] = {nullptr, nullptr, nullptr, nullptr, nullptr};
  // general spatial matrices (stfd_op_create_stencil)
  int kind = 0;                                   // 0: Kronecker factors, 1: stencil
  StencilOpDev sop;
  void* sbuf[7] = {nullptr, nullptr, nullptr, nullptr, nullptr, nullptr, nullptr};
  double* MtbU = nullptr;                         // band rows of M_t (unscaled, FP64) for gradients
  int pt = 0;
};

extern "C" const char* stfd_strerror(int code) {
  switch (code) {
    case STFD_OK: return "ok";
    case STFD_ERR_ARG: return "invalid argument";
    case STFD_ERR_NOT_SPD: return "mass matrix is not symmetric positive definite";
    case STFD_ERR_EIG: return "eigen-solver failed or factor structure check failed";
    case STFD_ERR_CUDA: return "CUDA runtime error";
    case STFD_ERR_NAN: return "non-finite value";
    case STFD_ERR_BREAKDOWN: return "Krylov breakdown";
    case STFD_ERR_TIMEOUT: return "bounded device wait timed out";
    case STFD_ERR_ALLOC: return "allocation failed";
    case STFD_NOT_CONVERGED: return "not converged";
    default: return "unknown status";
  }
}

extern "C" int stfd_version(void) { return 1; }

extern "C" int stfd_device_status(void) {
  if (cudaDeviceSynchronize() != cudaSuccess) return STFD_ERR_CUDA;
  return (status_read_and_clear() & kStatusTimeout) ? STFD_ERR_TIMEOUT : STFD_OK;
}

// ---------------------------------------------------------------------------
// Preconditioner
// ---------------------------------------------------------------------------

extern "C" void stfd_fd_destroy(stfd_fd* h) {
  if (!h) return;
  for (int l = 0; l <= kMaxDim; ++l) {
    dev_free(h->Jf[l]);
    dev_free(h->Jb[l]);
  }
  for (int l = 0; l < kMaxDim; ++l) dev_free(h->lam[l]);
  dev_free(h->lamt);
  dev_free(h->g);
  dev_free(h->Sinv);
  dev_free(h->work);
  dev_free(h->wtab);
  dev_free(h->Gg);
  for (int l = 0; l <= kMaxDim; ++l) {
    dev_free(h->Bf[l]);
    dev_free(h->Bb[l]);
  }
  for (int l = 0; l < kMaxDim; ++l) dev_free(h->lam_f[l]);
  dev_free(h->lamt_f);
  dev_free(h->g_f);
  dev_free(h->Sinv_f);
  for (int l = 0; l <= kMaxDim; ++l) {
    dev_free(h->Jf2[l]);
    dev_free(h->Jb2[l]);
  }
  for (int l = 0; l < kMaxDim; ++l) dev_free(h->lam2[l]);
  dev_free(h->B2);
  dev_free(h->BB2);
  dev_free(h->G2);
  dev_free(h->Sinv2);
  for (int l = 0; l <= kMaxDim; ++l) {
    dev_free(h->Zf[l]);
    dev_free(h->Zb[l]);
    dev_free(h->zvf[l]);
    dev_free(h->zvb[l]);
  }
  dev_free(h->dscale);
  dev_free(h->work2);
  dev_free(h->work3);
  dev_free(h->bexp);
  delete h;
}

extern "C" int stfd_fd_setup(stfd_fd** out, int d, const int* n, const double* const* K,
                             const double* const* M, const double* Wt, const double* Mt,
                             double gamma, double nu, int precision, void* stream) {
  if (!out) return STFD_ERR_ARG;
  *out = nullptr;
  if (!sizes_ok(d, n) || !K || !M || !Wt || !Mt) return STFD_ERR_ARG;
  if (!(gamma > 0.0) || !(nu > 0.0) || !std::isfinite(gamma) || !std::isfinite(nu)) return STFD_ERR_ARG;
  if (precision != STFD_FP64 && precision != STFD_TF32 && precision != STFD_BF16 && precision != STFD_DF32 &&
      precision != STFD_FP64TC && precision != STFD_FP64TC7)
    return STFD_ERR_ARG;
  if (precision == STFD_FP64TC)
    for (int l = 0; l <= d; ++l)
      if (n[l] > ozaki_max_n()) return STFD_ERR_ARG;
  if (precision == STFD_FP64TC7)
    for (int l = 0; l <= d; ++l)
      if (n[l] > oz7_max_n()) return STFD_ERR_ARG;
  if (precision == STFD_TF32 || precision == STFD_BF16)
    for (int l = 0; l <= d; ++l)
      if (n[l] > 128) return STFD_ERR_ARG;   // factor + tile + staging must fit in shared memory
  HostFactors f;
  int rc = factorize_host(d, n, K, M, Wt, Mt, f);
  if (rc != STFD_OK) return rc;
  cudaStream_t st = (cudaStream_t)stream;
  stfd_fd* h = new (std::nothrow) stfd_fd;
  if (!h) return STFD_ERR_ALLOC;
  h->d = d;
  h->Ns = 1;
  for (int l = 0; l <= d; ++l) h->n[l] = n[l];
  for (int l = 0; l < d; ++l) h->Ns *= n[l];
  h->N = h->Ns * n[d];
  h->gamma = gamma;
  h->nu = nu;
  h->precision = precision;
  h->n_pairs = f.n_pairs;
  h->has_zero = f.has_zero;
  h->sigma = f.sigma;
  for (int l = 0; l < d; ++l)
    for (int i = 0; i < n[l]; ++i) {
      h->diagM[l].push_back(M[l][i + (size_t)n[l] * i]);
      h->diagK[l].push_back(K[l][i + (size_t)n[l] * i]);
    }
  for (int i = 0; i < n[d]; ++i) {
    h->diagWt.push_back(Wt[i + (size_t)n[d] * i]);
    h->diagMt.push_back(Mt[i + (size_t)n[d] * i]);
  }
  // Step 2 uses J = U^T (row-major J[i][a] = U[a][i] = column-major U as is),
  // Step 4 uses J = U.
  std::vector<std::vector<double>> keep;
  for (int l = 0; l <= d; ++l) {
    const int nl = n[l];
    const std::vector<double>& U = (l < d) ? f.U[l] : f.Ut;
    keep.push_back(U);
    keep.push_back(row_major(nl, U.data()));
    if ((rc = dev_upload(&h->Jf[l], keep[keep.size() - 2].data(), (size_t)nl * nl, st)) != STFD_OK) break;
    if ((rc = dev_upload(&h->Jb[l], keep.back().data(), (size_t)nl * nl, st)) != STFD_OK) break;
    if (l < d && (rc = dev_upload(&h->lam[l], f.lam[l].data(), (size_t)nl, st)) != STFD_OK) break;
  }
  // Schur complement of the arrowhead per spatial index (eq. block_LU):
  // S_k = gamma sigma + a + sum_j gamma^2 a |g_j|^2 / (a^2 + gamma^2 lam_j^2) [+ gamma^2 g_z^2 / a]
  std::vector<double> Sinv;
  if (rc == STFD_OK) {
    Sinv = schur_reciprocals(f, gamma, nu);
    rc = dev_upload(&h->Sinv, Sinv.data(), Sinv.size(), st);
  }
  if (rc == STFD_OK && f.n_pairs > 0) rc = dev_upload(&h->lamt, f.lamt.data(), f.lamt.size(), st);
  if (rc == STFD_OK) rc = dev_upload(&h->g, f.g.data(), f.g.size(), st);
  // N doubles, or two FP32 N-vectors each starting on a 16-byte boundary (+4)
  if (rc == STFD_OK) rc = dev_upload<double>(&h->work, nullptr, (size_t)h->N + 4, st);
  if (rc == STFD_OK && (precision == STFD_DF32 || precision == STFD_FP64TC)) {
    rc = dev_upload<double>(&h->work3, nullptr, (size_t)h->N, st);
    if (rc == STFD_OK) rc = dev_upload<int>(&h->bexp, nullptr, 1, st);
  }
  std::vector<double> G(f.g.size());   // alive until the stream is synchronised below
  if (rc == STFD_OK && (precision == STFD_FP64 || precision == STFD_FP64TC7)) {
    for (size_t j = 0; j < f.g.size(); ++j) G[j] = gamma * f.g[j];
    rc = dev_upload(&h->Gg, G.data(), G.size(), st);
    if (rc == STFD_OK && f.n_pairs > 0) {
      rc = dev_upload<double2>(&h->wtab, nullptr, (size_t)f.n_pairs * (size_t)h->Ns, st);
      if (rc == STFD_OK) {
        ArrowParams ap;
        ap.d = d;
        ap.n1 = n[0];
        ap.n2 = d >= 2 ? n[1] : 1;
        ap.nt = n[d];
        ap.n_pairs = f.n_pairs;
        ap.has_zero = f.has_zero;
        ap.Ns = h->Ns;
        for (int l = 0; l < 3; ++l) ap.lam[l] = l < d ? h->lam[l] : nullptr;
        ap.lamt = h->lamt;
        ap.g = h->g;
        ap.Sinv = h->Sinv;
        ap.gamma = gamma;
        ap.nu = nu;
        ap.sgn = 1.0;
        if (launch_arrow_wtab(h->wtab, ap, st) != cudaSuccess) rc = STFD_ERR_CUDA;
      }
    }
  }
  // low precision: operand images and FP32 copies (kept alive in `keep` until the sync)
  std::vector<std::vector<float>> keepf;
  std::vector<std::vector<unsigned char>> keepb;
  std::vector<std::vector<float2>> keep2;
  auto up2 = [&](const double* v, size_t cnt, float2** dst) {
    keep2.emplace_back(cnt);
    for (size_t k = 0; k < cnt; ++k) {
      const float hh = (float)v[k];
      keep2.back()[k] = make_float2(hh, (float)(v[k] - (double)hh));
    }
    return dev_upload(dst, keep2.back().data(), cnt, st);
  };
  std::vector<std::vector<unsigned char>> keepz;
  std::vector<std::vector<int>> keepv;
  if (rc == STFD_OK && (precision == STFD_FP64TC || precision == STFD_FP64TC7)) {
    for (int l = 0; l <= d && rc == STFD_OK; ++l) {
      for (int dir = 0; dir < 2 && rc == STFD_OK; ++dir) {
        keepv.emplace_back();
        const double* J = keep[2 * l + dir].data();
        for (size_t k = 0; k < (size_t)n[l] * n[l]; ++k)
          if (!std::isfinite(J[k])) rc = STFD_ERR_EIG;
        if (rc != STFD_OK) break;
        keepz.push_back(precision == STFD_FP64TC ? ozaki_planes(J, n[l], keepv.back())
                                                 : oz7_planes(J, n[l], keepv.back()));
        rc = dev_upload(dir == 0 ? &h->Zf[l] : &h->Zb[l], keepz.back().data(), keepz.back().size(), st);
        if (rc == STFD_OK) rc = dev_upload(dir == 0 ? &h->zvf[l] : &h->zvb[l], keepv.back().data(), keepv.back().size(), st);
      }
    }
  }
  if (rc == STFD_OK && (precision == STFD_DF32 || precision == STFD_FP64TC)) {
    for (int l = 0; l <= d && rc == STFD_OK; ++l) {
      if (precision == STFD_DF32) {
        rc = up2(keep[2 * l].data(), keep[2 * l].size(), &h->Jf2[l]);
        if (rc == STFD_OK) rc = up2(keep[2 * l + 1].data(), keep[2 * l + 1].size(), &h->Jb2[l]);
      }
      if (rc == STFD_OK && l < d) rc = up2(f.lam[l].data(), f.lam[l].size(), &h->lam2[l]);
    }
    std::vector<double> B(std::max(1, f.n_pairs)), BB(std::max(1, f.n_pairs)), G(f.g.size());
    for (int j = 0; j < f.n_pairs; ++j) {
      B[j] = gamma * f.lamt[j];
      BB[j] = B[j] * B[j];
    }
    for (size_t j = 0; j < f.g.size(); ++j) G[j] = gamma * f.g[j];
    if (rc == STFD_OK) rc = up2(B.data(), B.size(), &h->B2);
    if (rc == STFD_OK) rc = up2(BB.data(), BB.size(), &h->BB2);
    if (rc == STFD_OK) rc = up2(G.data(), G.size(), &h->G2);
    if (rc == STFD_OK) rc = up2(Sinv.data(), Sinv.size(), &h->Sinv2);
  }
  if (rc == STFD_OK && (precision == STFD_TF32 || precision == STFD_BF16)) {
    const int kind = precision == STFD_BF16 ? 0 : 1;
    for (int l = 0; l <= d && rc == STFD_OK; ++l) {
      // keep[2l] is row-major U^T (= column-major U), keep[2l+1] row-major U
      keepb.push_back(tc_operand_image(keep[2 * l].data(), n[l], kind));
      rc = dev_upload(&h->Bf[l], keepb.back().data(), keepb.back().size(), st);
      if (rc != STFD_OK) break;
      keepb.push_back(tc_operand_image(keep[2 * l + 1].data(), n[l], kind));
      rc = dev_upload(&h->Bb[l], keepb.back().data(), keepb.back().size(), st);
      if (rc == STFD_OK && l < d) {
        keepf.emplace_back(f.lam[l].begin(), f.lam[l].end());
        rc = dev_upload(&h->lam_f[l], keepf.back().data(), keepf.back().size(), st);
      }
    }
    if (rc == STFD_OK && f.n_pairs > 0) {
      keepf.emplace_back(f.lamt.begin(), f.lamt.end());
      rc = dev_upload(&h->lamt_f, keepf.back().data(), keepf.back().size(), st);
    }
    if (rc == STFD_OK) {
      keepf.emplace_back(f.g.begin(), f.g.end());
      rc = dev_upload(&h->g_f, keepf.back().data(), keepf.back().size(), st);
    }
    if (rc == STFD_OK) {
      keepf.emplace_back(Sinv.begin(), Sinv.end());
      rc = dev_upload(&h->Sinv_f, keepf.back().data(), keepf.back().size(), st);
    }
  }
  if (rc == STFD_OK && cudaStreamSynchronize(st) != cudaSuccess) rc = STFD_ERR_CUDA;
  if (rc != STFD_OK) {
    stfd_fd_destroy(h);
    return rc;
  }
  *out = h;
  return STFD_OK;
}

extern "C" int stfd_fd_shape(const stfd_fd* h, int* d_out, int* n, long long* N_out) {
  if (!h) return STFD_ERR_ARG;
  if (d_out) *d_out = h->d;
  if (n)
    for (int l = 0; l <= h->d; ++l) n[l] = h->n[l];
  if (N_out) *N_out = h->N;
  return STFD_OK;
}

namespace {

// Low-precision Algorithm 1: tensor-core mode products with FP32 intermediates
// held in the handle's scratch (two FP32 N-vectors in the FP64 work buffer).
int fd_apply_one_lowp(const stfd_fd* h, const double* r, double* s, double* work, int trans, cudaStream_t st) {
  const int d = h->d;
  const int kind = h->precision == STFD_BF16 ? 0 : 1;
  float* buf[2] = {reinterpret_cast<float*>(work), reinterpret_cast<float*>(work) + ((h->N + 3) & ~3LL)};
  int cur = -1;   // -1: the FP64 input r
  long long inner = 1;
  for (int l = 0; l <= d; ++l) {
    const long long outer = h->N / (inner * h->n[l]);
    const int dst = (cur == 0) ? 1 : 0;
    const void* X = cur < 0 ? static_cast<const void*>(r) : static_cast<const void*>(buf[cur]);
    STFD_CU(launch_tc_mode(kind, X, cur < 0 ? 1 : 0, buf[dst], 0, h->Bf[l], h->n[l], inner, outer, st));
    cur = dst;
    inner *= h->n[l];
  }
  ArrowParamsT<float> ap;
  ap.d = d;
  ap.n1 = h->n[0];
  ap.n2 = d >= 2 ? h->n[1] : 1;
  ap.nt = h->n[d];
  ap.n_pairs = h->n_pairs;
  ap.has_zero = h->has_zero;
  ap.Ns = h->Ns;
  for (int l = 0; l < 3; ++l) ap.lam[l] = l < d ? h->lam_f[l] : nullptr;
  ap.lamt = h->lamt_f;
  ap.g = h->g_f;
  ap.Sinv = h->Sinv_f;
  ap.gamma = (float)h->gamma;
  ap.nu = (float)h->nu;
  ap.sgn = trans ? -1.0f : 1.0f;
  STFD_CU(launch_arrowhead_fp32(buf[cur], ap, st));
  for (int l = d; l >= 0; --l) {
    inner /= h->n[l];
    const long long outer = h->N / (inner * h->n[l]);
    const int dst = (cur == 0) ? 1 : 0;
    void* Y = (l == 0) ? static_cast<void*>(s) : static_cast<void*>(buf[dst]);
    STFD_CU(launch_tc_mode(kind, buf[cur], 0, Y, l == 0 ? 1 : 0, h->Bb[l], h->n[l], inner, outer, st));
    cur = dst;
  }
  return STFD_OK;
}

// Double-float Algorithm 1 (mode products in double-float on the FP32 pipes,
// or on the tensor cores by exact digit slices): same pass structure as the
// FP64 path, intermediates stored as float2 in the scratch and output buffers.
int fd_apply_one_df(const stfd_fd* h, const double* r, double* s, double* work, int trans, cudaStream_t st) {
  const bool tc = h->precision == STFD_FP64TC;
  auto mode = [&](const void* X, int xd, int l, bool fwd, void* Y, int yd, long long inner, long long outer) {
    if (tc)
      return launch_fd_mode_ozaki(X, xd, fwd ? h->Zf[l] : h->Zb[l], fwd ? h->zvf[l] : h->zvb[l], Y, yd, h->n[l],
                                  inner, outer, st);
    return launch_fd_mode_df(X, xd, fwd ? h->Jf2[l] : h->Jb2[l], Y, yd, h->n[l], inner, outer, st);
  };
  const int d = h->d;
  const int P = 2 * (d + 1);
  auto buf = [&](int k) { return ((P - k) % 2 == 0) ? static_cast<void*>(s) : static_cast<void*>(work); };
  // The mode products of Steps 2 and 4 commute. The FP64 input is read by the
  // time mode and the FP64 output written by it (a strided mode: its entries
  // travel straight to and from registers), so that mode 1, whose rows are
  // contiguous and go through a shared-memory stage, carries float2 only.
  // Forward order t, 1, .., d; backward order 1, .., d, t.
  long long inner_of[kMaxDim + 1];
  inner_of[0] = 1;
  for (int l = 1; l <= d; ++l) inner_of[l] = inner_of[l - 1] * h->n[l - 1];
  const void* src = r;
  int pass = 0;
  for (int k = 0; k <= d; ++k) {
    const int l = k == 0 ? d : k - 1;
    const long long outer = h->N / (inner_of[l] * h->n[l]);
    void* dst = buf(++pass);
    STFD_CU(mode(src, pass == 1 ? 1 : 0, l, true, dst, 0, inner_of[l], outer));
    src = dst;
  }
  const float2* lam[3] = {h->lam2[0], h->lam2[1], h->lam2[2]};
  STFD_CU(launch_arrowhead_df(static_cast<float2*>(const_cast<void*>(src)), d, h->n[0], d >= 2 ? h->n[1] : 1,
                              h->n[d], h->n_pairs, h->has_zero, h->Ns, lam, h->B2, h->BB2, h->G2, h->Sinv2, h->nu,
                              trans ? -1 : 1, st));
  for (int k = 0; k <= d; ++k) {
    const int l = k;
    const long long outer = h->N / (inner_of[l] * h->n[l]);
    void* dst = buf(++pass);
    STFD_CU(mode(src, 0, l, false, dst, pass == P ? 1 : 0, inner_of[l], outer));
    src = dst;
  }
  return STFD_OK;
}

// One right-hand side: s = P^{-1} r (trans = 0) or s = P^{-T} r (trans = 1)
// through 2(d+1) mode products and Step 3. P^{-T} = (U_t x U_s) Delta^{-T}
// (U_t x U_s)^T uses the same factors; only the arrowhead core is transposed,
// which in the real 2 x 2-block form flips the signs of lambda_j and g.
int fd_apply_core(const stfd_fd* h, const double* r, double* s, double* work, int trans, cudaStream_t st) {
  if (h->precision == STFD_DF32 || h->precision == STFD_FP64TC) {
    // the double-float intermediates have FP32's exponent range: run on r 2^{1023 - E}
    // (E the largest biased exponent of r) and scale the result back; both exact
    STFD_CU(launch_range_scale(r, h->work3, h->N, h->bexp, -1, st));
    const int rc = fd_apply_one_df(h, h->work3, s, work, trans, st);
    if (rc != STFD_OK) return rc;
    STFD_CU(launch_range_scale(s, s, h->N, h->bexp, 1, st));
    return STFD_OK;
  }
  if (h->precision != STFD_FP64 && h->precision != STFD_FP64TC7) return fd_apply_one_lowp(h, r, s, work, trans, st);
  const int d = h->d;
  const int P = 2 * (d + 1);
  auto buf = [&](int k) { return ((P - k) % 2 == 0) ? s : work; };   // pass k writes buf(k), buf(P) = s
  const double* src = r;
  int pass = 0;
  // FP64 mode products: on the FP64 pipe, or on the tensor cores by seven exact
  // digit slices per entry (STFD_FP64TC7); both FP64 in and out
  const bool tc7 = h->precision == STFD_FP64TC7;
  auto mode = [&](const double* X, int l, bool fwd, double* Y, long long inner, long long outer) {
    if (tc7)
      return launch_fd_mode_tc7(X, fwd ? h->Zf[l] : h->Zb[l], fwd ? h->zvf[l] : h->zvb[l], Y, h->n[l], inner, outer,
                                st);
    return launch_fd_mode_fp64(X, fwd ? h->Jf[l] : h->Jb[l], Y, h->n[l], inner, outer, st);
  };
  // Step 2: X x_1 U_1^T ... x_d U_d^T x_{d+1} U_t^T
  long long inner = 1;
  for (int l = 0; l <= d; ++l) {
    const long long outer = h->N / (inner * h->n[l]);
    double* dst = buf(++pass);
    STFD_CU(mode(src, l, true, dst, inner, outer));
    src = dst;
    inner *= h->n[l];
  }
  // Step 3 in place
  ArrowParams ap;
  ap.d = d;
  ap.n1 = h->n[0];
  ap.n2 = d >= 2 ? h->n[1] : 1;
  ap.nt = h->n[d];
  ap.n_pairs = h->n_pairs;
  ap.has_zero = h->has_zero;
  ap.Ns = h->Ns;
  for (int l = 0; l < 3; ++l) ap.lam[l] = l < d ? h->lam[l] : nullptr;
  ap.lamt = h->lamt;
  ap.g = h->g;
  ap.Sinv = h->Sinv;
  ap.gamma = h->gamma;
  ap.nu = h->nu;
  ap.sgn = trans ? -1.0 : 1.0;
  if (h->Gg && (h->wtab || h->n_pairs == 0)) {
    STFD_CU(launch_arrowhead_fp64_tab(const_cast<double*>(src), ap, h->wtab, h->Gg, st));
  } else {
    STFD_CU(launch_arrowhead_fp64(const_cast<double*>(src), ap, st));
  }
  // Step 4: x_{d+1} U_t, then x_d U_d ... x_1 U_1
  for (int l = d; l >= 0; --l) {
    inner /= h->n[l];
    const long long outer = h->N / (inner * h->n[l]);
    double* dst = buf(++pass);
    STFD_CU(mode(src, l, false, dst, inner, outer));
    src = dst;
  }
  return STFD_OK;
}

// With the diagonal scaling of eq. prec_geo, P = D^{1/2} A~ D^{1/2}, so
// P^{-1} r = D^{-1/2} A~^{-1} (D^{-1/2} r) (and the same with A~^{-T}).
int fd_apply_one(const stfd_fd* h, const double* r, double* s, double* work, int trans, cudaStream_t st) {
  if (!h->dscale) return fd_apply_core(h, r, s, work, trans, st);
  STFD_CU(launch_scale(r, h->dscale, h->work2, h->N, st));
  const int rc = fd_apply_core(h, h->work2, s, work, trans, st);
  if (rc != STFD_OK) return rc;
  STFD_CU(launch_scale(s, h->dscale, s, h->N, st));
  return STFD_OK;
}

}  // namespace

extern "C" int stfd_fd_set_scaling(stfd_fd* h, const double* Ms_diag, const double* Ks_diag, void* stream) {
  if (!h) return STFD_ERR_ARG;
  cudaStream_t st = (cudaStream_t)stream;
  if (!Ms_diag && !Ks_diag) {
    if (cudaStreamSynchronize(st) != cudaSuccess) return STFD_ERR_CUDA;
    dev_free(h->dscale);
    dev_free(h->work2);
    h->dscale = h->work2 = nullptr;
    return STFD_OK;
  }
  if (!Ms_diag || !Ks_diag) return STFD_ERR_ARG;
  // D_(k,t) = (gamma w_t a_k + nu m_t b_k) / (gamma w_t a~_k + nu m_t b~_k) with a, b the
  // diagonals of M_s, K_s and a~, b~ those of the Kronecker factors of the handle.
  const int d = h->d;
  std::vector<double> at((size_t)h->Ns), bt((size_t)h->Ns);
  for (long long k = 0; k < h->Ns; ++k) {
    long long rest = k;
    int idx[kMaxDim];
    for (int l = 0; l < d; ++l) {
      idx[l] = (int)(rest % h->n[l]);
      rest /= h->n[l];
    }
    double m = 1.0, kk = 0.0;
    for (int l = 0; l < d; ++l) m *= h->diagM[l][idx[l]];
    for (int l = 0; l < d; ++l) {
      double t = h->diagK[l][idx[l]];
      for (int q = 0; q < d; ++q)
        if (q != l) t *= h->diagM[q][idx[q]];
      kk += t;
    }
    at[k] = m;
    bt[k] = kk;
  }
  std::vector<double> ds((size_t)h->N);
  const int nt = h->n[d];
  for (int t = 0; t < nt; ++t) {
    const double w = h->gamma * h->diagWt[t], mt = h->nu * h->diagMt[t];
    for (long long k = 0; k < h->Ns; ++k) {
      const double num = w * Ms_diag[k] + mt * Ks_diag[k];
      const double den = w * at[k] + mt * bt[k];
      const double D = num / den;
      if (!(D > 0.0) || !std::isfinite(D)) return STFD_ERR_ARG;
      ds[(size_t)t * h->Ns + k] = 1.0 / std::sqrt(D);
    }
  }
  if (!h->work2 && dev_upload<double>(&h->work2, nullptr, (size_t)h->N, st) != STFD_OK) return STFD_ERR_ALLOC;
  if (!h->dscale && dev_upload<double>(&h->dscale, nullptr, (size_t)h->N, st) != STFD_OK) return STFD_ERR_ALLOC;
  STFD_CU(cudaMemcpyAsync(h->dscale, ds.data(), ds.size() * sizeof(double), cudaMemcpyHostToDevice, st));
  if (cudaStreamSynchronize(st) != cudaSuccess) return STFD_ERR_CUDA;
  return STFD_OK;
}

namespace {
int fd_apply_batch(const stfd_fd* h, const double* r, double* s, int nrhs, int trans, void* stream) {
  if (!h || nrhs < 0 || (nrhs > 0 && (!r || !s))) return STFD_ERR_ARG;
  if (nrhs > 0 && r == s) return STFD_ERR_ARG;
  // a bounded device wait of an earlier, completed launch ran out
  if (status_read_and_clear() & kStatusTimeout) return STFD_ERR_TIMEOUT;
  cudaStream_t st = (cudaStream_t)stream;
  for (int k = 0; k < nrhs; ++k) {
    const int rc = fd_apply_one(h, r + (size_t)k * h->N, s + (size_t)k * h->N, h->work, trans, st);
    if (rc != STFD_OK) return rc;
  }
  return STFD_OK;
}
}  // namespace

extern "C" int stfd_fd_apply(const stfd_fd* h, const double* r, double* s, int nrhs, void* stream) {
  return fd_apply_batch(h, r, s, nrhs, 0, stream);
}

extern "C" int stfd_fd_apply_transpose(const stfd_fd* h, const double* r, double* s, int nrhs, void* stream) {
  return fd_apply_batch(h, r, s, nrhs, 1, stream);
}

// ---------------------------------------------------------------------------
// System operator
// ---------------------------------------------------------------------------

static void gmres_free(GmresWork* w) {
  if (!w) return;
  for (double* p : w->V) dev_free(p);
  for (double* p : w->Z) dev_free(p);
  dev_free(w->dV);
  dev_free(w->dZ);
  dev_free(w->partial);
  dev_free(w->h);
  if (w->hostbuf) cudaFreeHost(w->hostbuf);
  delete w;
}

extern "C" void stfd_op_destroy(stfd_op* A) {
  if (!A) return;
  for (int l = 0; l < kMaxDim; ++l) {
    dev_free(A->JM[l]);
    dev_free(A->JK[l]);
  }
  dev_free(A->JW);
  dev_free(A->JWT);
  dev_free(A->JMt);
  for (int l = 0; l < kMaxDim; ++l) {
    dev_free(A->JM2[l]);
    dev_free(A->JK2[l]);
  }
  dev_free(A->JW2);
  dev_free(A->JWT2);
  dev_free(A->JMt2);
  for (int l = 0; l < kMaxDim; ++l) {
    dev_free(A->Kb[l]);
  }
  for (int l = 0; l < kMaxDim; ++l) {
    dev_free(A->MK4[l]);
    dev_free(A->MM4[l]);
  }
  dev_free(A->WMt4);
  dev_free(A->WTMt4);
  for (int k = 0; k < kMaxDim + 2; ++k) {
    dev_free(A->FXC[k]);
    dev_free(A->FXE[k]);
  }
  for (int k = 0; k < 4; ++k) dev_free(A->tmp[k]);
  dev_free(A->tmp5);
  dev_free(A->bexp);
  for (int k = 0; k < 7; ++k) dev_free(A->sbuf[k]);
  dev_free(A->MtbU);
  gmres_free(A->gw);
  delete A;
}

extern "C" int stfd_op_create_kron(stfd_op** out, int d, const int* n, const double* const* K,
                                   const double* const* M, const double* Wt, const double* Mt,
                                   double gamma, double nu, int arith, void* stream) {
  if (!out) return STFD_ERR_ARG;
  *out = nullptr;
  if (!sizes_ok(d, n) || !K || !M || !Wt || !Mt) return STFD_ERR_ARG;
  for (int l = 0; l < d; ++l)
    if (!K[l] || !M[l]) return STFD_ERR_ARG;
  if (!std::isfinite(gamma) || !std::isfinite(nu)) return STFD_ERR_ARG;
  if (arith != STFD_OP_FP64 && arith != STFD_OP_DF32 && arith != STFD_OP_FX64) return STFD_ERR_ARG;
  cudaStream_t st = (cudaStream_t)stream;
  stfd_op* A = new (std::nothrow) stfd_op;
  if (!A) return STFD_ERR_ALLOC;
  A->d = d;
  A->N = 1;
  for (int l = 0; l <= d; ++l) {
    A->n[l] = n[l];
    A->N *= n[l];
  }
  A->gamma = gamma;
  A->nu = nu;
  A->arith = arith;
  int rc = STFD_OK;
  std::vector<std::vector<double>> keep;
  for (int l = 0; l < d && rc == STFD_OK; ++l) {
    keep.push_back(row_major(n[l], M[l]));
    rc = dev_upload(&A->JM[l], keep.back().data(), keep.back().size(), st);
    A->bwM[l] = bandwidth(n[l], M[l]);
    if (rc != STFD_OK) break;
    keep.push_back(row_major(n[l], K[l]));
    rc = dev_upload(&A->JK[l], keep.back().data(), keep.back().size(), st);
    A->bwK[l] = bandwidth(n[l], K[l]);
  }
  if (rc == STFD_OK) {
    keep.push_back(row_major(n[d], Wt));
    rc = dev_upload(&A->JW, keep.back().data(), keep.back().size(), st);
    A->bwW = bandwidth(n[d], Wt);
  }
  if (rc == STFD_OK) {
    keep.push_back(row_major(n[d], Mt));
    rc = dev_upload(&A->JMt, keep.back().data(), keep.back().size(), st);
    A->bwMt = bandwidth(n[d], Mt);
  }
  // W_t^T row-major is W_t column-major read as rows: keep[2d + 2]
  if (rc == STFD_OK) {
    keep.emplace_back(Wt, Wt + (size_t)n[d] * n[d]);
    rc = dev_upload(&A->JWT, keep.back().data(), keep.back().size(), st);
  }
  for (int k = 0; k < 4 && rc == STFD_OK; ++k) rc = dev_upload<double>(&A->tmp[k], nullptr, (size_t)A->N, st);
  if (rc == STFD_OK && arith == STFD_OP_DF32) {
    rc = dev_upload<double>(&A->tmp5, nullptr, (size_t)A->N, st);
    if (rc == STFD_OK) rc = dev_upload<int>(&A->bexp, nullptr, 1, st);
  }
  if (rc == STFD_OK) {
    A->pt = A->bwMt;
    std::vector<double> MbU((size_t)n[d] * (2 * A->pt + 1), 0.0);
    for (int t = 0; t < n[d]; ++t)
      for (int k = 0; k <= 2 * A->pt; ++k) {
        const int a = t - A->pt + k;
        if (a >= 0 && a < n[d]) MbU[(size_t)t * (2 * A->pt + 1) + k] = Mt[t + (size_t)n[d] * a];
      }
    rc = dev_upload(&A->MtbU, MbU.data(), MbU.size(), st);
  }
  // integer-limb band tables (STFD_OP_FX64) when every half-bandwidth is 1..4;
  // otherwise the op keeps the FP64 passes (the same arithmetic class)
  std::vector<std::vector<int2>> keepc;
  std::vector<std::vector<int>> keepe;
  if (rc == STFD_OK && arith == STFD_OP_FX64) {
    int pb[kMaxDim + 1];
    bool ok = true;
    for (int l = 0; l <= d; ++l) {
      pb[l] = l < d ? std::max(A->bwM[l], A->bwK[l]) : std::max(A->bwW, A->bwMt);
      if (pb[l] < 1 || pb[l] > 4) ok = false;
    }
    A->fx = ok;
    if (ok) {
      for (int l = 0; l <= d; ++l) A->pb[l] = pb[l];
      const size_t nt2 = (size_t)n[d] * n[d];
      std::vector<double> gW(nt2), gWT(nt2), nMt(nt2);
      for (size_t k = 0; k < nt2; ++k) {
        gW[k] = gamma * keep[2 * d][k];
        gWT[k] = gamma * keep[2 * d + 2][k];
        nMt[k] = nu * keep[2 * d + 1][k];
      }
      for (int k = 0; k <= d + 1 && rc == STFD_OK; ++k) {
        keepc.emplace_back();
        keepe.emplace_back();
        if (k < d) fx_tables(keep[2 * k].data(), keep[2 * k + 1].data(), n[k], pb[k], keepc.back(), keepe.back());
        else fx_tables(k == d ? gW.data() : gWT.data(), nMt.data(), n[d], pb[d], keepc.back(), keepe.back());
        rc = dev_upload(&A->FXC[k], keepc.back().data(), keepc.back().size(), st);
        if (rc == STFD_OK) rc = dev_upload(&A->FXE[k], keepe.back().data(), keepe.back().size(), st);
      }
      if (rc == STFD_OK && cudaStreamSynchronize(st) != cudaSuccess) rc = STFD_ERR_CUDA;   // gW, gWT, nMt die here
    }
  }
  // double-float copies (hi, lo) of the row-major factors: keep = [M_0, K_0, M_1, K_1, ..., W_t, M_t]
  std::vector<std::vector<float2>> keep2;
  std::vector<std::vector<float4>> keep4;
  if (rc == STFD_OK && arith == STFD_OP_DF32) {
    auto split = [&](const std::vector<double>& J, float2** dst) {
      keep2.emplace_back(J.size());
      for (size_t k = 0; k < J.size(); ++k) {
        const float h = (float)J[k];
        keep2.back()[k] = make_float2(h, (float)(J[k] - (double)h));
      }
      return dev_upload(dst, keep2.back().data(), keep2.back().size(), st);
    };
    for (int l = 0; l < d && rc == STFD_OK; ++l) {
      rc = split(keep[2 * l], &A->JM2[l]);
      if (rc == STFD_OK) rc = split(keep[2 * l + 1], &A->JK2[l]);
    }
    if (rc == STFD_OK) rc = split(keep[2 * d], &A->JW2);
    if (rc == STFD_OK) rc = split(keep[2 * d + 1], &A->JMt2);
    if (rc == STFD_OK) rc = split(keep[2 * d + 2], &A->JWT2);
    // band-compressed copies for the unrolled kernels (half-bandwidth 1..4 in every direction)
    A->banded = true;
    for (int l = 0; l <= d; ++l) {
      A->pb[l] = l < d ? std::max(A->bwM[l], A->bwK[l]) : std::max(A->bwW, A->bwMt);
      if (A->pb[l] < 1 || A->pb[l] > 4) A->banded = false;
    }
    auto compress = [&](const std::vector<double>& J, int nl, int p, float2** dst) {
      const int W = 2 * p + 1;
      std::vector<double> band((size_t)nl * W, 0.0);
      for (int i = 0; i < nl; ++i)
        for (int t = 0; t < W; ++t) {
          const int a = i - p + t;
          if (a >= 0 && a < nl) band[(size_t)i * W + t] = J[(size_t)i * nl + a];
        }
      return split(band, dst);
    };
    // two band matrices as coefficient pairs (hi_1, hi_2, lo_1, lo_2) per tap
    auto compress_pair = [&](const std::vector<double>& J1, const std::vector<double>& J2, int nl, int p,
                             float4** dst) {
      const int W = 2 * p + 1;
      keep4.emplace_back((size_t)nl * W, make_float4(0.f, 0.f, 0.f, 0.f));
      for (int i = 0; i < nl; ++i)
        for (int t = 0; t < W; ++t) {
          const int a = i - p + t;
          if (a < 0 || a >= nl) continue;
          const double v1 = J1[(size_t)i * nl + a], v2 = J2[(size_t)i * nl + a];
          const float h1 = (float)v1, h2 = (float)v2;
          keep4.back()[(size_t)i * W + t] = make_float4(h1, h2, (float)(v1 - (double)h1), (float)(v2 - (double)h2));
        }
      return dev_upload(dst, keep4.back().data(), keep4.back().size(), st);
    };
    if (A->banded) {
      for (int l = 0; l < d && rc == STFD_OK; ++l) {
        rc = compress(keep[2 * l + 1], n[l], A->pb[l], &A->Kb[l]);
        if (rc == STFD_OK) rc = compress_pair(keep[2 * l], keep[2 * l + 1], n[l], A->pb[l], &A->MK4[l]);
        if (rc == STFD_OK) rc = compress_pair(keep[2 * l], keep[2 * l], n[l], A->pb[l], &A->MM4[l]);
      }
      if (rc == STFD_OK) rc = compress_pair(keep[2 * d], keep[2 * d + 1], n[d], A->pb[d], &A->WMt4);
      if (rc == STFD_OK) rc = compress_pair(keep[2 * d + 2], keep[2 * d + 1], n[d], A->pb[d], &A->WTMt4);
    }
  }
  if (rc == STFD_OK && cudaStreamSynchronize(st) != cudaSuccess) rc = STFD_ERR_CUDA;
  if (rc != STFD_OK) {
    stfd_op_destroy(A);
    return rc;
  }
  *out = A;
  return STFD_OK;
}

namespace {

// Band rows B[t][k] = s * A[t][t - pb + k] of a column-major n x n matrix
// (transposed if `trans`).
std::vector<double> band_rows(int n, const double* A, int pb, double s, bool trans) {
  const int W = 2 * pb + 1;
  std::vector<double> B((size_t)n * W, 0.0);
  for (int t = 0; t < n; ++t)
    for (int k = 0; k < W; ++k) {
      const int a = t - pb + k;
      if (a < 0 || a >= n) continue;
      B[(size_t)t * W + k] = s * (trans ? A[a + (size_t)n * t] : A[t + (size_t)n * a]);
    }
  return B;
}

}  // namespace

extern "C" int stfd_op_create_stencil(stfd_op** out, int d, const int* n, int p_s, const double* Ms,
                                      const double* Ks, const double* Wt, const double* Mt, double gamma, double nu,
                                      int arith, void* stream) {
  if (!out) return STFD_ERR_ARG;
  *out = nullptr;
  if (!sizes_ok(d, n) || !Ms || !Ks || !Wt || !Mt || p_s < 0 || p_s > 10) return STFD_ERR_ARG;
  if (!std::isfinite(gamma) || !std::isfinite(nu)) return STFD_ERR_ARG;
  if (arith != STFD_OP_FP64 && arith != STFD_OP_DF32 && arith != STFD_OP_FX64) return STFD_ERR_ARG;
  cudaStream_t st = (cudaStream_t)stream;
  stfd_op* A = new (std::nothrow) stfd_op;
  if (!A) return STFD_ERR_ALLOC;
  A->kind = 1;
  A->d = d;
  A->arith = arith;
  A->gamma = gamma;
  A->nu = nu;
  long long Ns = 1;
  for (int l = 0; l < d; ++l) Ns *= n[l];
  for (int l = 0; l <= d; ++l) A->n[l] = n[l];
  const int nt = n[d];
  A->N = Ns * nt;
  int S = 1;
  for (int l = 0; l < d; ++l) S *= 2 * p_s + 1;
  const int pt = std::max(bandwidth(nt, Wt), bandwidth(nt, Mt));
  A->pt = pt;
  StencilOpDev& o = A->sop;
  o.d = d;
  o.p = p_s;
  o.pt = pt;
  o.nt = nt;
  for (int l = 0; l < d; ++l) o.n[l] = n[l];
  o.Ns = Ns;
  o.df = arith == STFD_OP_DF32;
  // integer limbs when the row sums stay exact (at most stencil_fx_max_taps() offsets), else FP64
  o.fx = arith == STFD_OP_FX64 && S <= stencil_fx_max_taps();
  std::vector<double> Wb = band_rows(nt, Wt, pt, gamma, false), WbT = band_rows(nt, Wt, pt, gamma, true),
                      Mb = band_rows(nt, Mt, pt, nu, false), MbU = band_rows(nt, Mt, pt, 1.0, false);
  int rc = dev_upload(&A->MtbU, MbU.data(), MbU.size(), st);
  const double* srcs[5] = {Ms, Ks, Wb.data(), WbT.data(), Mb.data()};
  const size_t cnt[5] = {(size_t)S * Ns, (size_t)S * Ns, Wb.size(), WbT.size(), Mb.size()};
  std::vector<std::vector<float2>> keep2;
  for (int k = 0; k < 5 && rc == STFD_OK; ++k) {
    if (o.df) {
      keep2.emplace_back(cnt[k]);
      for (size_t i = 0; i < cnt[k]; ++i) {
        const float h = (float)srcs[k][i];
        keep2.back()[i] = make_float2(h, (float)(srcs[k][i] - (double)h));
      }
      float2* dst = nullptr;
      rc = dev_upload(&dst, keep2.back().data(), cnt[k], st);
      A->sbuf[k] = dst;
    } else {
      double* dst = nullptr;
      rc = dev_upload(&dst, srcs[k], cnt[k], st);
      A->sbuf[k] = dst;
    }
  }
  for (int k = 5; k < 7 && rc == STFD_OK; ++k) {
    double* dst = nullptr;   // float2 and double have the same size
    rc = dev_upload<double>(&dst, nullptr, (size_t)A->N, st);
    A->sbuf[k] = dst;
  }
  if (rc == STFD_OK && o.df) {
    rc = dev_upload<double>(&A->tmp5, nullptr, (size_t)A->N, st);
    if (rc == STFD_OK) rc = dev_upload<int>(&A->bexp, nullptr, 1, st);
  }
  if (rc == STFD_OK && o.fx) {   // row frames, and the coefficients as limbs in place
    for (int k = 0; k < 2 && rc == STFD_OK; ++k) {
      rc = dev_upload<int>(&A->FXE[k], nullptr, (size_t)Ns, st);
      if (rc == STFD_OK && launch_stencil_fx_table(static_cast<double*>(A->sbuf[k]), A->FXE[k], S, Ns, st) !=
                               cudaSuccess)
        rc = STFD_ERR_CUDA;
    }
    o.Em = A->FXE[0];
    o.Ek = A->FXE[1];
  }
  if (rc == STFD_OK) {
    o.Ms = A->sbuf[0];
    o.Ks = A->sbuf[1];
    o.Wb = A->sbuf[2];
    o.WbT = A->sbuf[3];
    o.Mtb = A->sbuf[4];
    o.Z1 = A->sbuf[5];
    o.Z2 = A->sbuf[6];
  }
  if (rc == STFD_OK && cudaStreamSynchronize(st) != cudaSuccess) rc = STFD_ERR_CUDA;
  if (rc != STFD_OK) {
    stfd_op_destroy(A);
    return rc;
  }
  *out = A;
  return STFD_OK;
}

extern "C" int stfd_grad_kappa_elements(const stfd_op* A, int p, int n_el, const double* Ke_dev,
                                        const double* lam_dev, const double* u_dev, double* g_dev, void* stream) {
  if (!A || !Ke_dev || !lam_dev || !u_dev || !g_dev || p < 1 || n_el < 1) return STFD_ERR_ARG;
  const int d = A->d;
  for (int l = 0; l < d; ++l)
    if (A->n[l] != n_el + p - 2) return STFD_ERR_ARG;
  if (grad_elements_smem(d, p) > 200 * 1024) return STFD_ERR_ARG;
  if (!A->MtbU) return STFD_ERR_ARG;
  cudaStream_t st = (cudaStream_t)stream;
  long long Ns = A->N / A->n[d];
  // ubar = (M_t (x) I) u in the op's scratch (two N-vectors of 8-byte entries)
  double* ubar = A->kind == 1 ? static_cast<double*>(A->sbuf[5]) : A->tmp[0];
  double* dup = A->kind == 1 ? static_cast<double*>(A->sbuf[6]) : A->tmp[1];
  STFD_CU(launch_time_mass_fp64(u_dev, A->MtbU, ubar, dup, Ns, A->n[d], A->pt, st));
  STFD_CU(launch_grad_elements(Ke_dev, lam_dev, ubar, g_dev, d, p, n_el, n_el + p - 2, Ns, A->n[d], A->nu, st));
  return STFD_OK;
}

namespace {

// y = gamma (W_t x M_d x..x M_1) x + nu (M_t x sum_l M_d..K_l..M_1) x, sum-factorised:
// direction 1: (u, v) = (x x_1 M_1, x x_1 K_1); direction l > 1:
// (u, v) <- (u x_l M_l, u x_l K_l + v x_l M_l); time: y = gamma u x W_t + nu v x M_t.
// Same sum-factorisation in double-float arithmetic, one pass per direction;
// intermediates are float2 (hi, lo) pairs.
int matvec_one_df(const stfd_op* A, const double* x, double* y, int trans, cudaStream_t st) {
  const int d = A->d;
  float2* T[4];
  for (int k = 0; k < 4; ++k) T[k] = reinterpret_cast<float2*>(A->tmp[k]);
  long long inner = 1;
  const float2* u = nullptr;
  const float2* v = nullptr;
  for (int l = 0; l < d; ++l) {
    const int nl = A->n[l];
    const long long outer = A->N / (inner * nl);
    float2* uo = (l % 2 == 0) ? T[0] : T[2];
    float2* vo = (l % 2 == 0) ? T[1] : T[3];
    const int bw = std::max(A->bwM[l], A->bwK[l]);
    if (A->banded) {
      // rotated layouts: every pass reads its fibres contiguous and writes transposed
      if (l == 0) {
        STFD_CU(launch_band_first_pk(x, A->MK4[l], uo, vo, nl, 1, A->N / nl, A->pb[l], 1, st));
      } else {
        STFD_CU(launch_band_mid_pk(u, v, A->MM4[l], A->Kb[l], uo, vo, nl, 1, A->N / nl, A->pb[l], 1, st));
      }
    } else if (l == 0) {
      STFD_CU(launch_band_first_df(x, A->JM2[l], A->JK2[l], uo, vo, nl, inner, outer, bw, st));
    } else {
      STFD_CU(launch_band_mid_df(u, v, A->JM2[l], A->JK2[l], uo, vo, nl, inner, outer, bw, st));
    }
    u = uo;
    v = vo;
    inner *= nl;
  }
  const int nt = A->n[d];
  if (A->banded) {
    STFD_CU(launch_band_last_pk(u, v, trans ? A->WTMt4 : A->WMt4, A->gamma, A->nu, y, nt, 1, A->N / nt, A->pb[d], 1,
                                st));
  } else {
    STFD_CU(launch_band_last_df(u, v, trans ? A->JWT2 : A->JW2, A->gamma, A->JMt2, A->nu, y, nt, inner, 1, std::max(A->bwW, A->bwMt), st));
  }
  return STFD_OK;
}

// The same sum-factorisation with FP64 intermediates, every band product formed
// exactly in 64-bit integer limbs and rounded once (band_fx.cu); rotated layouts
// as in the double-float passes.
int matvec_one_fx(const stfd_op* A, const double* x, double* y, int trans, cudaStream_t st) {
  const int d = A->d;
  double* const* T = A->tmp;
  const double* u = nullptr;
  const double* v = nullptr;
  for (int l = 0; l < d; ++l) {
    const int nl = A->n[l];
    double* uo = (l % 2 == 0) ? T[0] : T[2];
    double* vo = (l % 2 == 0) ? T[1] : T[3];
    if (l == 0) {
      STFD_CU(launch_band_first_fx(x, A->FXC[0], A->FXE[0], uo, vo, nl, 1, A->N / nl, A->pb[0], 1, st));
    } else {
      STFD_CU(launch_band_mid_fx(u, v, A->FXC[l], A->FXE[l], uo, vo, nl, 1, A->N / nl, A->pb[l], 1, st));
    }
    u = uo;
    v = vo;
  }
  const int nt = A->n[d];
  const int k = trans ? d + 1 : d;
  STFD_CU(launch_band_last_fx(u, v, A->FXC[k], A->FXE[k], y, nt, 1, A->N / nt, A->pb[d], 1, st));
  return STFD_OK;
}

int matvec_one_fp(const stfd_op* A, const double* x, double* y, int trans, cudaStream_t st);

// y = A x (trans = 0) or y = A^T x (trans = 1); A^T = gamma W_t^T x M_s + nu M_t x K_s
// since every factor but W_t is symmetric.
int matvec_one(const stfd_op* A, const double* x, double* y, int trans, cudaStream_t st) {
  const bool df = A->kind == 1 ? A->sop.df : A->arith == STFD_OP_DF32;
  if (df) {
    // double-float passes (FP32 exponent range): run on x 2^{1023 - E}, scale y back; exact
    STFD_CU(launch_range_scale(x, A->tmp5, A->N, A->bexp, -1, st));
    x = A->tmp5;
  }
  int rc = STFD_OK;
  if (A->kind == 1) {
    if (launch_stencil_matvec(A->sop, x, y, trans, st) != cudaSuccess) rc = STFD_ERR_CUDA;
  } else if (df) {
    rc = matvec_one_df(A, x, y, trans, st);
  } else {
    rc = matvec_one_fp(A, x, y, trans, st);
  }
  if (rc != STFD_OK) return rc;
  if (df) STFD_CU(launch_range_scale(y, y, A->N, A->bexp, 1, st));
  return STFD_OK;
}

// FP64 results: the integer-limb passes (STFD_OP_FX64) or the FP64 passes.
int matvec_one_fp(const stfd_op* A, const double* x, double* y, int trans, cudaStream_t st) {
  if (A->fx) return matvec_one_fx(A, x, y, trans, st);
  const int d = A->d;
  double* const* T = A->tmp;
  long long inner = 1;
  const double* u = x;
  const double* v = nullptr;
  for (int l = 0; l < d; ++l) {
    const int nl = A->n[l];
    const long long outer = A->N / (inner * nl);
    double* uo = (l % 2 == 0) ? T[0] : T[2];
    double* vo = (l % 2 == 0) ? T[1] : T[3];
    const int bwM = A->bwM[l], bwK = A->bwK[l];
    STFD_CU(launch_band_mode_fp64(u, A->JM[l], 1.0, nullptr, nullptr, 0.0, uo, nl, inner, outer, bwM, st));
    if (l == 0) {
      STFD_CU(launch_band_mode_fp64(u, A->JK[l], 1.0, nullptr, nullptr, 0.0, vo, nl, inner, outer, bwK, st));
    } else {
      STFD_CU(launch_band_mode_fp64(u, A->JK[l], 1.0, v, A->JM[l], 1.0, vo, nl, inner, outer,
                               std::max(bwM, bwK), st));
    }
    u = uo;
    v = vo;
    inner *= nl;
  }
  const int nt = A->n[d];
  STFD_CU(launch_band_mode_fp64(u, trans ? A->JWT : A->JW, A->gamma, v, A->JMt, A->nu, y, nt, inner, 1,
                           std::max(A->bwW, A->bwMt), st));
  return STFD_OK;
}

}  // namespace

namespace {
int matvec_batch(const stfd_op* A, const double* x, double* y, int nrhs, int trans, void* stream) {
  if (!A || nrhs < 0 || (nrhs > 0 && (!x || !y))) return STFD_ERR_ARG;
  if (nrhs > 0 && x == y) return STFD_ERR_ARG;
  cudaStream_t st = (cudaStream_t)stream;
  for (int k = 0; k < nrhs; ++k) {
    const int rc = matvec_one(A, x + (size_t)k * A->N, y + (size_t)k * A->N, trans, st);
    if (rc != STFD_OK) return rc;
  }
  return STFD_OK;
}
}  // namespace

extern "C" int stfd_st_matvec(const stfd_op* A, const double* x, double* y, int nrhs, void* stream) {
  return matvec_batch(A, x, y, nrhs, 0, stream);
}

extern "C" int stfd_st_matvec_transpose(const stfd_op* A, const double* x, double* y, int nrhs, void* stream) {
  return matvec_batch(A, x, y, nrhs, 1, stream);
}

// ---------------------------------------------------------------------------
// Flexible GMRES
// ---------------------------------------------------------------------------

extern "C" void stfd_gmres_default_opts(stfd_gmres_opts* o) {
  if (!o) return;
  o->tol = 1e-8;
  o->restart = 100;
  o->max_it = 1000;
  o->transpose = 0;
}

namespace {

// Pointer arrays (device) sized for `cap` vectors; vectors themselves are
// allocated lazily by ensure_vec when an iteration first needs them.
int ensure_ptr_array(std::vector<double*>& vec, double**& dptr, int& cap, int want) {
  if (want <= cap) return STFD_OK;
  dev_free(dptr);
  dptr = nullptr;
  if (cudaMalloc((void**)&dptr, (size_t)want * sizeof(double*)) != cudaSuccess) return STFD_ERR_ALLOC;
  cap = want;
  if (!vec.empty())
    STFD_CU(cudaMemcpy(dptr, vec.data(), vec.size() * sizeof(double*), cudaMemcpyHostToDevice));
  return STFD_OK;
}

int ensure_vec(std::vector<double*>& vec, double** dptr, int idx, long long N) {
  while ((int)vec.size() <= idx) {
    double* p = nullptr;
    if (cudaMalloc((void**)&p, (size_t)N * sizeof(double)) != cudaSuccess) return STFD_ERR_ALLOC;
    vec.push_back(p);
    STFD_CU(cudaMemcpy(dptr + (vec.size() - 1), &p, sizeof(double*), cudaMemcpyHostToDevice));
  }
  return STFD_OK;
}

int ensure_work(GmresWork* w, int restart) {
  int rc = ensure_ptr_array(w->V, w->dV, w->cap_v, restart + 1);
  if (rc != STFD_OK) return rc;
  rc = ensure_ptr_array(w->Z, w->dZ, w->cap_z, restart);
  if (rc != STFD_OK) return rc;
  const int need_partial = dot_blocks() * (restart + 1);
  if (need_partial > w->partial_cap) {
    dev_free(w->partial);
    w->partial = nullptr;
    if (cudaMalloc((void**)&w->partial, (size_t)need_partial * sizeof(double)) != cudaSuccess) return STFD_ERR_ALLOC;
    w->partial_cap = need_partial;
  }
  if (restart + 3 > w->hcap) {
    dev_free(w->h);
    w->h = nullptr;
    if (w->hostbuf) cudaFreeHost(w->hostbuf);
    w->hostbuf = nullptr;
    w->hostbuf_dev = nullptr;
    if (cudaMalloc((void**)&w->h, (size_t)(2 * restart + 6) * sizeof(double)) != cudaSuccess) return STFD_ERR_ALLOC;
    if (cudaHostAlloc((void**)&w->hostbuf, (size_t)(2 * restart + 6) * sizeof(double), cudaHostAllocMapped) !=
            cudaSuccess ||
        cudaHostGetDevicePointer((void**)&w->hostbuf_dev, w->hostbuf, 0) != cudaSuccess)
      return STFD_ERR_ALLOC;
    w->hcap = restart + 3;
  }
  return STFD_OK;
}


}  // namespace

extern "C" int stfd_gmres_solve(const stfd_op* Ac, const stfd_fd* P, const double* f, double* u,
                                const stfd_gmres_opts* opts, stfd_gmres_info* info, void* stream) {
  if (!Ac || !P || !f || !u || f == u) return STFD_ERR_ARG;
  if (Ac->N != P->N || Ac->d != P->d) return STFD_ERR_ARG;
  stfd_gmres_opts o;
  stfd_gmres_default_opts(&o);
  if (opts) o = *opts;
  if (o.restart < 1 || o.restart > 1000 || o.max_it < 1 || !(o.tol > 0.0)) return STFD_ERR_ARG;
  if (o.transpose != 0 && o.transpose != 1) return STFD_ERR_ARG;
  if (status_read_and_clear() & kStatusTimeout) return STFD_ERR_TIMEOUT;
  const int tr = o.transpose;
  stfd_op* A = const_cast<stfd_op*>(Ac);   // the Krylov workspace is cached in the op
  cudaStream_t st = (cudaStream_t)stream;
  if (!A->gw) {
    A->gw = new (std::nothrow) GmresWork;
    if (!A->gw) return STFD_ERR_ALLOC;
  }
  GmresWork* w = A->gw;
  int rc = ensure_work(w, o.restart);
  if (rc != STFD_OK) return rc;
  if ((rc = ensure_vec(w->V, w->dV, 1, A->N)) != STFD_OK) return rc;
  const long long N = A->N;
  const int m = o.restart;
  const int nb = dot_blocks();
  double* hb = w->hostbuf;        // pinned host mirror of dh
  double* dh = w->h;              // [0..m] h, [m+1 .. 2m+1] h2, [2m+2] ||w||^2
  double* dh2 = w->h + (m + 1);
  double* dnrm = w->h + (2 * m + 2);
  if (info) {
    info->iters = 0;
    info->converged = 0;
    info->rel_res_est = 1.0;
    info->rel_res_true = 1.0;
    info->hist_len = 0;
  }
  // Residual r = f - A u (r = f while u is zero) and ||r||^2 to the host in one
  // fused pass; r is stored in V[0] only when a new cycle starts from it.
  auto residual = [&](bool u_is_zero, bool write_v0, double* nrm2) -> int {
    const double* Au = nullptr;
    if (!u_is_zero) {
      int r2 = matvec_one(A, u, w->V[1], tr, st);
      if (r2 != STFD_OK) return r2;
      Au = w->V[1];
    }
    STFD_CU(launch_sub_norm(write_v0 ? w->V[0] : nullptr, f, Au, N, w->partial, nb, st));
    STFD_CU(launch_reduce_partial(w->partial, 1, nb, dnrm, 0, st));
    STFD_CU(launch_copy_doubles(w->hostbuf_dev + 2 * m + 2, dnrm, 1, st));
    STFD_CU(cudaStreamSynchronize(st));
    if (status_read_and_clear() & kStatusTimeout) return STFD_ERR_TIMEOUT;
    *nrm2 = hb[2 * m + 2];
    return STFD_OK;
  };
  double nrm2 = 0.0;
  if ((rc = residual(true, false, &nrm2)) != STFD_OK) return rc;
  const double fnorm = std::sqrt(nrm2);
  if (!std::isfinite(fnorm)) return STFD_ERR_NAN;
  if (fnorm == 0.0) {
    STFD_CU(cudaMemsetAsync(u, 0, (size_t)N * sizeof(double), st));
    if (info) {
      info->converged = 1;
      info->rel_res_est = info->rel_res_true = 0.0;
    }
    return STFD_OK;
  }
  const double* v0_src = f;   // the first cycle starts from r = f (u = 0)
  bool first_cycle = true;    // u is written (not accumulated) by the first update
  std::vector<double> H((size_t)(m + 1) * m), cs(m), sn(m), g(m + 1), y(m);
  int total = 0;
  bool converged = false;
  double est = 1.0, beta = fnorm;
  while (true) {
    // v_0 = r / beta  (dnrm still holds ||r||^2 on the device)
    STFD_CU(launch_scale_by_inverse(w->V[0], v0_src, dnrm, N, 1, st));
    std::fill(g.begin(), g.end(), 0.0);
    g[0] = beta;
    int j_done = 0;
    bool lucky = false;
    for (int j = 0; j < m && total < o.max_it; ++j) {
      if ((rc = ensure_vec(w->V, w->dV, j + 1, N)) != STFD_OK) return rc;
      if ((rc = ensure_vec(w->Z, w->dZ, j, N)) != STFD_OK) return rc;
      // v_j = w_j / ||w_j||: the normalisation deferred from the previous
      // iteration (dnrm still holds ||w_j||^2), skipped when the cycle stops there
      if (j > 0) STFD_CU(launch_scale_by_inverse(w->V[j], w->V[j], dnrm, N, 1, st));
      // z_j = P^{-1} v_j ;  w = A z_j  (built in V[j+1]); P^{-T}, A^T when transposed
      if ((rc = fd_apply_one(P, w->V[j], w->Z[j], P->work, tr, st)) != STFD_OK) return rc;
      if ((rc = matvec_one(A, w->Z[j], w->V[j + 1], tr, st)) != STFD_OK) return rc;
      // classical Gram-Schmidt twice: h = V^T w, w -= V h, h2 = V^T w, w -= V h2
      STFD_CU(launch_dot_multi(w->dV, j + 1, w->V[j + 1], N, w->partial, nb, st));
      STFD_CU(launch_reduce_partial(w->partial, j + 1, nb, dh, 0, st));
      if (j + 1 <= 4) {   // the first update fused with the second dot products
        STFD_CU(launch_axpy_dot(w->V[j + 1], w->dV, dh, j + 1, N, w->partial, nb, st));
      } else {
        STFD_CU(launch_multi_axpy(w->V[j + 1], w->dV, dh, j + 1, N, -1.0, st));
        STFD_CU(launch_dot_multi(w->dV, j + 1, w->V[j + 1], N, w->partial, nb, st));
      }
      STFD_CU(launch_reduce_partial(w->partial, j + 1, nb, dh2, 0, st));
      // second update fused with ||w||^2 (the normalisation of w happens next iteration)
      STFD_CU(launch_axpy_norm(w->V[j + 1], w->dV, dh2, j + 1, N, -1.0, 0, w->partial, nb, st));
      STFD_CU(launch_reduce_partial(w->partial, 1, nb, dnrm, 0, st));
      STFD_CU(launch_copy_doubles(w->hostbuf_dev, dh, 2 * m + 3, st));
      STFD_CU(cudaStreamSynchronize(st));
      // the preconditioner's tensor-core kernels raise the status word when a
      // bounded wait runs out (they then skip work): the iterate is not valid
      if (status_read_and_clear() & kStatusTimeout) return STFD_ERR_TIMEOUT;
      double* c = &H[(size_t)(m + 1) * j];
      for (int i = 0; i <= j; ++i) c[i] = hb[i] + hb[m + 1 + i];
      const double hn = std::sqrt(hb[2 * m + 2]);
      c[j + 1] = hn;
      for (int i = 0; i <= j + 1; ++i)
        if (!std::isfinite(c[i])) return STFD_ERR_NAN;
      for (int i = 0; i < j; ++i) {   // previous Givens rotations
        const double t = cs[i] * c[i] + sn[i] * c[i + 1];
        c[i + 1] = -sn[i] * c[i] + cs[i] * c[i + 1];
        c[i] = t;
      }
      const double den = std::hypot(c[j], c[j + 1]);
      if (den == 0.0) return STFD_ERR_BREAKDOWN;
      cs[j] = c[j] / den;
      sn[j] = c[j + 1] / den;
      c[j] = den;
      c[j + 1] = 0.0;
      g[j + 1] = -sn[j] * g[j];
      g[j] = cs[j] * g[j];
      ++total;
      j_done = j + 1;
      est = std::fabs(g[j + 1]) / fnorm;
      if (info && info->history && info->hist_len < info->hist_cap) info->history[info->hist_len++] = est;
      if (est <= o.tol) {
        converged = true;
        break;
      }
      if (hn == 0.0) {   // invariant subspace reached: the update below is exact
        lucky = true;
        break;
      }
    }
    // y = R^{-1} g (back substitution), u += Z y
    for (int i = j_done - 1; i >= 0; --i) {
      double t = g[i];
      for (int k = i + 1; k < j_done; ++k) t -= H[i + (size_t)(m + 1) * k] * y[k];
      y[i] = t / H[i + (size_t)(m + 1) * i];
    }
    std::copy(y.begin(), y.begin() + j_done, hb);
    STFD_CU(launch_copy_doubles(dh, w->hostbuf_dev, j_done, st));
    STFD_CU(launch_axpy_norm(u, w->dZ, dh, j_done, N, 1.0, first_cycle ? 1 : 0, nullptr, nb, st));
    first_cycle = false;
    if (converged || lucky || total >= o.max_it) break;
    // restart from the true residual
    if ((rc = residual(false, true, &nrm2)) != STFD_OK) return rc;
    v0_src = w->V[0];
    beta = std::sqrt(nrm2);
    if (!std::isfinite(beta)) return STFD_ERR_NAN;
    if (beta <= o.tol * fnorm) {
      converged = true;
      est = beta / fnorm;
      break;
    }
  }
  // true residual ||f - A u|| / ||f|| (explicit matvec, no vector stored)
  if ((rc = residual(false, false, &nrm2)) != STFD_OK) return rc;
  const double true_res = std::sqrt(nrm2) / fnorm;
  if (info) {
    info->iters = total;
    info->converged = converged ? 1 : 0;
    info->rel_res_est = est;
    info->rel_res_true = true_res;
  }
  if (!std::isfinite(true_res)) return STFD_ERR_NAN;
  return converged ? STFD_OK : STFD_NOT_CONVERGED;
}
