// Launchers of the device kernels (FP64 path). All are stream-ordered and
// return the cudaError_t of the launch.
#pragma once
#include <cuda_runtime.h>

#include <vector>

namespace stfd {

// Mode product of Algorithm 1 (dense n x n factor):
// Y[o, i, c] = sum_a J[i*n + a] X[o, a, c] for o < outer, i < n, c < inner,
// with X[o, a, c] at o*n*inner + a*inner + c. Y must not alias X.
cudaError_t launch_fd_mode_fp64(const double* X, const double* J, double* Y, int n, long long inner,
                                long long outer, cudaStream_t st);

// Banded mode products of the system matvec:
// Y[o, i, c] = s1 sum_a J1[i,a] X1[o,a,c] (+ s2 sum_a J2[i,a] X2[o,a,c]), |a - i| <= bw.
// X2/J2 may be NULL. Y must not alias X1 or X2.
cudaError_t launch_band_mode_fp64(const double* X1, const double* J1, double s1,
                                  const double* X2, const double* J2, double s2,
                                  double* Y, int n, long long inner, long long outer, int bw,
                                  cudaStream_t st);

// In-place Step 3 of Algorithm 1 on the spectral tensor X[t][k] (time index
// slowest): block LU of the real arrowhead system per spatial index k.
template <typename T>
struct ArrowParamsT {
  int d, n1, n2, nt, n_pairs, has_zero;
  long long Ns;
  const T* lam[3];   // spatial eigenvalues per direction
  const T* lamt;     // n_pairs
  const T* g;        // nt - 1
  const T* Sinv;     // Ns reciprocals of the Schur complement
  T gamma, nu;
  T sgn;             // +1: Delta_t;  -1: Delta_t^T (lam_j and g change sign)
};
using ArrowParams = ArrowParamsT<double>;
cudaError_t launch_arrowhead_fp64(double* X, const ArrowParams& p, cudaStream_t st);
// FP64 Step 3 with the per-(pair, index) complex reciprocals W[j][k] of
// launch_arrow_wtab (n_pairs x Ns double2, set-up) and G = gamma g (nt - 1).
cudaError_t launch_arrow_wtab(double2* W, const ArrowParams& p, cudaStream_t st);
cudaError_t launch_arrowhead_fp64_tab(double* X, const ArrowParams& p, const double2* W, const double* G,
                                      cudaStream_t st);
// FP32 variant for the mixed-precision preconditioner
cudaError_t launch_arrowhead_fp32(float* X, const ArrowParamsT<float>& p, cudaStream_t st);

// tcgen05 mode product with BF16 (kind 0) or TF32 (kind 1) operands and FP32
// accumulation: Y[o, i, c] = sum_a J[i, a] X[o, a, c]. X is FP64 or FP32, Y FP32 or
// FP64 (not both FP64). B is the factor image from tc_operand_image (device).
cudaError_t launch_tc_mode(int kind, const void* X, int x_is_double, void* Y, int y_is_double,
                           const unsigned char* B, int n, long long inner, long long outer, cudaStream_t st);
// Host: factor J (row-major n x n, J[i*n + a]) as a K-major canonical operand image.
std::vector<unsigned char> tc_operand_image(const double* J, int n, int kind);
// Self-test of the bounded mbarrier wait (never satisfied): sets the status flag.
cudaError_t launch_probe_bounded_wait(int max_iters, cudaStream_t st);

// Exact power-of-two range scaling: dir = -1 takes E = the largest biased
// exponent of x into *bexp (device int) and writes y = x 2^{1023 - E}; dir = +1
// writes y = x 2^{E - 1023} with the E stored before (y may alias x).
cudaError_t launch_range_scale(const double* x, double* y, long long N, int* bexp, int dir, cudaStream_t st);

// GMRES BLAS: partial[b*m + i] = sum over block b's range of V_i[k] * w[k].
cudaError_t launch_dot_multi(const double* const* V, int m, const double* w, long long N,
                             double* partial, int nblocks, cudaStream_t st);
// out[i] = sum_b partial[b*m + i]  (+ out[i] if accumulate)
cudaError_t launch_reduce_partial(const double* partial, int m, int nblocks, double* out,
                                  int accumulate, cudaStream_t st);
// w[k] += sign * sum_i h[i] V_i[k]
cudaError_t launch_multi_axpy(double* w, const double* const* V, const double* h, int m,
                              long long N, double sign, cudaStream_t st);
// w -= sum_{i<m} h[i] V_i and partial[b*m + i] = block b's share of V_i . w (the
// updated w), for 1 <= m <= 4 (cudaErrorInvalidValue otherwise).
cudaError_t launch_axpy_dot(double* w, const double* const* V, const double* h, int m, long long N,
                            double* partial, int nblocks, cudaStream_t st);
// y[k] = x[k] / *den, or x[k] / sqrt(*den) if sqrt_den (den on the device;
// a non-positive divisor leaves x unscaled)
cudaError_t launch_scale_by_inverse(double* y, const double* x, const double* den, long long N,
                                    int sqrt_den, cudaStream_t st);
// y[k] = a[k] - b[k]
cudaError_t launch_sub(double* y, const double* a, const double* b, long long N, cudaStream_t st);
// dst[i] = src[i], i < n, by a one-block kernel (either side may be host-mapped memory).
cudaError_t launch_copy_doubles(double* dst, const double* src, int n, cudaStream_t st);
// w = (set ? 0 : w) + sign sum_i h[i] V_i; partial[b] (nblocks entries, if not NULL)
// receives block b's share of ||w||^2 of the result.
cudaError_t launch_axpy_norm(double* w, const double* const* V, const double* h, int m, long long N, double sign,
                             int set, double* partial, int nblocks, cudaStream_t st);
// r = f - y (y NULL: r = f), written to out if out is not NULL; partial[b] = block b's share of ||r||^2.
cudaError_t launch_sub_norm(double* out, const double* f, const double* y, long long N, double* partial,
                            int nblocks, cudaStream_t st);

// Double-float banded passes of the matvec (band_df.cu); factors row-major (hi, lo):
//   first direction:  (Uo, Vo) = (x x M, x x K), x FP64
//   other directions: (Uo, Vo) = (u x M, u x K + v x M)
//   time:             y = gamma u x W + nu v x M_t, y FP64
cudaError_t launch_band_first_df(const double* x, const float2* M, const float2* K, float2* Uo, float2* Vo, int n,
                                 long long inner, long long outer, int bw, cudaStream_t st);
cudaError_t launch_band_mid_df(const float2* u, const float2* v, const float2* M, const float2* K, float2* Uo,
                               float2* Vo, int n, long long inner, long long outer, int bw, cudaStream_t st);
cudaError_t launch_band_last_df(const float2* u, const float2* v, const float2* W, double gamma, const float2* Mt,
                                double nu, double* y, int n, long long inner, long long outer, int bw,
                                cudaStream_t st);
// The same three passes with a compile-time half-bandwidth p in 1..4
// (cudaErrorInvalidValue otherwise) over band-compressed factors
// Ab[i][t] = A[i][i-p+t], t < 2p+1, two accumulation chains issued together on
// the paired FP32 instructions; tables of (hi_1, hi_2, lo_1, lo_2) per band tap:
// first direction (M, K), middle directions (M, M) with K from the (hi, lo) band
// table Kb, time (W_t or W_t^T, M_t). With
// rot = 1 the inputs hold the direction fastest (fibres contiguous, inner = 1)
// and entry i of fibre q is written to i Q + q (Q = inner * outer fibres): each
// pass leaves the next direction fastest, and after the time pass the layout
// is the original one again.
cudaError_t launch_band_first_pk(const double* x, const float4* MK, float2* Uo, float2* Vo, int n, long long inner,
                                 long long outer, int p, int rot, cudaStream_t st);
cudaError_t launch_band_mid_pk(const float2* u, const float2* v, const float4* MM, const float2* Kb, float2* Uo,
                               float2* Vo, int n, long long inner, long long outer, int p, int rot, cudaStream_t st);
cudaError_t launch_band_last_pk(const float2* u, const float2* v, const float4* WMt, double gamma, double nu,
                                double* y, int n, long long inner, long long outer, int p, int rot, cudaStream_t st);

// FP64 banded passes in exact 64-bit integer arithmetic (band_fx.cu), same pass
// structure and rotated layouts as the paired double-float passes; C / Ce from
// fx_tables (first and middle passes: (M, K); time pass: (gamma W or gamma W^T,
// nu M_t)); p in 1..4 (cudaErrorInvalidValue otherwise).
cudaError_t launch_band_first_fx(const double* x, const int2* C, const int* Ce, double* Uo, double* Vo, int n,
                                 long long inner, long long outer, int p, int rot, cudaStream_t st);
cudaError_t launch_band_mid_fx(const double* u, const double* v, const int2* C, const int* Ce, double* Uo, double* Vo,
                               int n, long long inner, long long outer, int p, int rot, cudaStream_t st);
cudaError_t launch_band_last_fx(const double* u, const double* v, const int2* C, const int* Ce, double* y, int n,
                                long long inner, long long outer, int p, int rot, cudaStream_t st);
void fx_tables(const double* A, const double* B, int n, int p, std::vector<int2>& C, std::vector<int>& Ce);

// Double-float Algorithm 1 (fd_df.cu): dense mode product with (hi, lo) row-major
// factor J, X FP64 or float2, Y float2 or FP64 (not both FP64); Step 3 in place on
// a float2 spectral tensor with per-pair B = gamma lam_j, BB = B^2, G = gamma g.
cudaError_t launch_fd_mode_df(const void* X, int x_is_double, const float2* J, void* Y, int y_is_double, int n,
                              long long inner, long long outer, cudaStream_t st);
cudaError_t launch_arrowhead_df(float2* X, int d, int n1, int n2, int nt, int n_pairs, int has_zero, long long Ns,
                                const float2* const* lam, const float2* B, const float2* BB, const float2* G,
                                const float2* Sinv, double nu, int sgn, cudaStream_t st);

// FP64-accurate mode product on tcgen05 by exact BF16 digit slices (tc_ozaki.cu):
// X FP64 or float2, Y float2 or FP64 (not both FP64); B / v from ozaki_planes.
cudaError_t launch_fd_mode_ozaki(const void* X, int x_is_double, const unsigned char* B, const int* v, void* Y,
                                 int y_is_double, int n, long long inner, long long outer, cudaStream_t st);
std::vector<unsigned char> ozaki_planes(const double* J, int n, std::vector<int>& v);
int ozaki_max_n();

// FP64 mode product on tcgen05 by seven exact BF16 digit slices per entry
// (tc_oz7.cu): X and Y FP64 (Y must not alias X); B / ej from oz7_planes.
cudaError_t launch_fd_mode_tc7(const double* X, const unsigned char* B, const int* ej, double* Y, int n,
                               long long inner, long long outer, cudaStream_t st);
std::vector<unsigned char> oz7_planes(const double* J, int n, std::vector<int>& ej);
int oz7_max_n();

int dot_blocks();

// General spatial matrices in the tensor-product stencil layout (stencil.cu).
struct StencilOpDev {
  int d = 0, p = 0, pt = 0, nt = 0;
  int n[3] = {1, 1, 1};
  long long Ns = 0;
  bool df = false;                    // coefficients and intermediates as (hi, lo) float pairs
  const void* Ms = nullptr;           // [(2p+1)^d][Ns] double or float2
  const void* Ks = nullptr;
  const void* Wb = nullptr;           // gamma W_t, band rows [nt][2pt+1]
  const void* WbT = nullptr;          // gamma W_t^T
  const void* Mtb = nullptr;          // nu M_t
  void* Z1 = nullptr;                 // scratch nt * Ns
  void* Z2 = nullptr;
  // STFD_OP_FX64: Ms, Ks hold balanced 27-bit limbs (int2) of each row's
  // 53-bit integers under the row frames Em, Ek (largest biased exponent)
  bool fx = false;
  const int* Em = nullptr;
  const int* Ek = nullptr;
};
struct StencilDims {
  int d, p;
  int n1, n2;          // n_s per direction (n2 = 1 when d = 1; n3 implied)
  long long Ns;
  int nt;
};
cudaError_t launch_stencil_matvec(const StencilOpDev& op, const double* x, double* y, int trans, cudaStream_t st);
// STFD_OP_FX64 stencil (stencil_fx.cu): the coefficient rows of one matrix
// ([S][Ns] FP64, S <= stencil_fx_max_taps()) converted in place to limbs, with
// their frames E[Ns]; the spatial pass y_t = M_s Z1_t + K_s Z2_t.
int stencil_fx_max_taps();
cudaError_t launch_stencil_fx_table(double* C, int* E, int S, long long Ns, cudaStream_t st);
cudaError_t launch_stencil_space_fx(const StencilOpDev& op, const double* Z1, const double* Z2, double* y,
                                    const StencilDims& g, cudaStream_t st);
size_t grad_elements_smem(int d, int p);
cudaError_t launch_grad_elements(const double* Ke, const double* lam, const double* ubar, double* g, int d, int p,
                                 int n_el, int n_s, long long Ns, int nt, double nu, cudaStream_t st);
cudaError_t launch_scale(const double* x, const double* s, double* y, long long N, cudaStream_t st);
// y = (M_t (x) I) x with the band rows Mb [nt][2pt+1] (FP64); `scratch` receives a copy.
cudaError_t launch_time_mass_fp64(const double* x, const double* Mb, double* y, double* scratch, long long Ns, int nt,
                                  int pt, cudaStream_t st);

}  // namespace stfd
