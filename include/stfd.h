/*
 * stfd.h -- C ABI of the GB300 space-time Fast Diagonalization library.
 *
 * Problem (Loli, Montardini, Sangalli, Tani, "An efficient solver for
 * space-time isogeometric Galerkin methods for parabolic problems"):
 * the Galerkin discretisation of  gamma d_t u - nu Lap u = f  with
 * maximal-smoothness B-splines in space and time gives (Sec. 3.3, eq. syst_mat)
 *
 *     A = gamma W_t (x) M_s + nu M_t (x) K_s,
 *
 * M_s = M_d (x) .. (x) M_1 and K_s = sum_l M_d (x) .. K_l .. (x) M_1 on the
 * parametric box (Sec. 4, eqs. prec_definition and space_univ_par_mat). The
 * preconditioner P has the same form; it is applied exactly by the extended
 * Fast Diagonalization of Algorithm 1 (Sec. 4.3).
 *
 * Conventions common to every entry point
 *  - Vectors of length N = n_1 * ... * n_d * n_t are stored in the paper's
 *    vec order (Sec. 2.3, eq. kron_vec_multi): i_1 fastest, time slowest.
 *    Several right-hand sides are stored one after another (nrhs * N).
 *  - Pointers named "dev" are CUDA device pointers owned by the caller; all
 *    others are host pointers owned by the caller. The library never frees
 *    caller memory and copies what it keeps.
 *  - Dense matrices on the host are column-major n x n.
 *  - `stream` is a cudaStream_t passed as void* (NULL = legacy default
 *    stream). Device work is stream-ordered and asynchronous unless stated.
 *  - Every int-returning call returns STFD_OK (0) or a negative STFD_ERR_*
 *    code (STFD_NOT_CONVERGED = 1 is a warning); nothing is thrown across
 *    the ABI. stfd_strerror() names a code.
 *  - Handles are immutable after creation, except their device scratch (the
 *    intermediate tensors of an apply or matvec, and the Krylov workspace that
 *    stfd_gmres_solve caches inside an stfd_op): calls on one handle must not
 *    overlap in time, whether from several streams or several host threads.
 */
#ifndef STFD_H
#define STFD_H

#ifdef __cplusplus
extern "C" {
#endif

enum {
  STFD_OK = 0,
  STFD_ERR_ARG = -1,        /* bad size, NULL pointer, unsupported option */
  STFD_ERR_NOT_SPD = -2,    /* Cholesky of a mass matrix failed */
  STFD_ERR_EIG = -3,        /* eigen-solver did not converge or structure check failed */
  STFD_ERR_CUDA = -4,       /* a CUDA runtime call or kernel launch failed */
  STFD_ERR_NAN = -5,        /* non-finite value met (e.g. in the right-hand side) */
  STFD_ERR_BREAKDOWN = -6,  /* Krylov breakdown other than a lucky one */
  STFD_ERR_TIMEOUT = -7,    /* a bounded device-side wait gave up */
  STFD_ERR_ALLOC = -8,      /* device or host allocation failed */
  STFD_NOT_CONVERGED = 1    /* solver stopped at max_it above the tolerance */
};

/* Arithmetic of the preconditioner's mode products (Steps 2 and 4 of
 * Algorithm 1). STFD_FP64: FP64 throughout. STFD_TF32 / STFD_BF16: operands
 * rounded to TF32 / BF16 on the tcgen05 tensor cores with FP32 accumulation,
 * FP32 intermediates and an FP32 Step 3; input and output vectors stay FP64.
 * The low-precision preconditioner is meant for flexible GMRES, which keeps
 * the outer iteration, the system matvec and the residual in FP64. */
enum { STFD_FP64 = 0, STFD_TF32 = 1, STFD_BF16 = 2, STFD_DF32 = 3, STFD_FP64TC = 4, STFD_FP64TC7 = 5 };
/* STFD_FP64TC7: FP64 Algorithm 1 with the mode products on the tcgen05 tensor
 * cores, no narrower than IEEE FP64. Each row of the tensor and of the factor
 * is written under its own power of two as a 55-bit integer (exact for entries
 * within a factor 4 of the row maximum, rounded at 2^-55 of the row scale for
 * the others) and cut exactly into seven signed 8-bit digits; the 28 digit
 * pairs that reach 2^-48 of the row scales run as BF16 MMAs whose FP32
 * accumulators are exact, the partial sums are combined in 64-bit integers and
 * rounded once to FP64. Intermediates between the mode products are FP64, and
 * Step 3 is IEEE FP64. The dropped digit pairs are below 2^-44 of
 * n max|row of X| max|row of U|, under the worst-case rounding error of an FP64
 * dot product of length n. Requires every n[l] <= 80.
 * STFD_FP64TC: the same on six digits (21 pairs, about 48 significant bits),
 * partial sums recombined in double-float, double-float intermediates and
 * Step 3. Requires every n[l] <= 80. Agrees with STFD_FP64 to about 1e-13. */
/* STFD_DF32: FP64-accurate Algorithm 1 in double-float arithmetic on the FP32
 * pipes (every value an unevaluated pair hi + lo of floats, about 48
 * significant bits; products split exactly by FMA, sums by error-free
 * two-sum); FP64 input and output, agrees with STFD_FP64 to about 1e-13. */

/* Boundary treatment of a univariate basis (Sec. 2.2). */
enum {
  STFD_BC_NONE = 0,         /* all m = n_el + p B-splines */
  STFD_BC_INITIAL = 1,      /* drop b_1: time direction, zero initial condition (n = m - 1) */
  STFD_BC_DIRICHLET = 2     /* drop b_1 and b_m: space direction, Dirichlet (n = m - 2) */
};

const char* stfd_strerror(int code);
int stfd_version(void);

/* Device-side failure detection. The tensor-core kernels wait on their own
 * asynchronous tensor-core operations and bulk copies with bounded mbarrier
 * waits. A wait that runs out raises a status word (pinned host memory that
 * every device writes through its mapping); the kernel then lets its own
 * operations in flight finish (bounded), skips its remaining tiles, releases
 * tensor memory and returns, so the CUDA context stays usable but the result
 * of that launch is not valid. The word is read and cleared by:
 *  - stfd_device_status(): synchronises the device first, returns
 *    STFD_ERR_TIMEOUT if the word was raised, else STFD_OK (STFD_ERR_CUDA if
 *    the synchronisation fails);
 *  - stfd_gmres_solve(): after each of its per-iteration synchronisations, so
 *    a solve whose preconditioner timed out returns STFD_ERR_TIMEOUT;
 *  - stfd_fd_apply() and stfd_fd_apply_transpose() on entry (they are
 *    asynchronous, so they report a timeout of an earlier launch that has
 *    completed by then). */
int stfd_device_status(void);

/* Iteration limit of every bounded device wait (default 1 << 22, about a
 * second of polling). Process-wide, read at each launch. 0 makes every wait
 * give up at once (used to test the reporting path). Returns STFD_ERR_ARG
 * outside [0, 2^40]. */
int stfd_set_wait_limit(long long iters);
long long stfd_get_wait_limit(void);

/* ------------------------------------------------------------------------
 * Univariate spline matrices (host, CPU only).
 * Sec. 2.1 (open uniform knot vector on [0, length], Cox-de Boor B-splines of
 * degree p, n_el elements), eq. time_mat and the univariate factors of eq.
 * space_univ_par_mat:
 *     M[i,j] = int b_i b_j,   K[i,j] = int b'_i b'_j,   W[i,j] = int b'_j b_i,
 * with the basis reduced by `bc`. Output: dense column-major n x n where
 * n = n_el + p - {0,1,2} by bc. *n_out receives n. Any of M, K, W may be NULL
 * (skipped); call with all three NULL to query n. Requires p >= 1, n_el >= 1,
 * length > 0, and n >= 1 after the reduction.
 * ------------------------------------------------------------------------ */
int stfd_spline_matrices(int p, int n_el, double length, int bc,
                         double* M, double* K, double* W, int* n_out);

/* Load vector of a trigonometric source (host): out[i] = int_0^length
 * (c_sin sin(freq x) + c_cos cos(freq x)) b_i(x) dx over the reduced basis,
 * i.e. one factor of the linear form F of Sec. 3.1 for a separable f.
 * `out` has n entries (as returned by stfd_spline_matrices). */
int stfd_spline_load_trig(int p, int n_el, double length, int bc,
                          double freq, double c_sin, double c_cos, double* out);

/* ------------------------------------------------------------------------
 * Fast Diagonalization factors (host, CPU only) -- Step 1 of Algorithm 1.
 * Spatial pencils (eq. space_eig): K_l U_l = M_l U_l Lambda_l, U_l^T M_l U_l = I.
 * Time pencil (Sec. 4.2.2, eqs. arrow..time_eig_2, real form of the Remark in
 * Sec. 4.5): W_t U_t = M_t U_t Delta_t, U_t^T M_t U_t = I, with
 *     Delta_t = [ blockdiag(B_1..B_q, [0]) | g ; -g^T | sigma ],
 * B_j = [[0, lam_j], [-lam_j, 0]] for the q pairs of purely imaginary
 * eigenvalues +-i lam_j of the skew leading block, then one 1 x 1 zero block
 * when n_t - 1 is odd, then the last (arrow) index.
 * Inputs: n[0..d-1] spatial sizes (K[l], M[l] are n[l] x n[l]), n[d] = n_t
 * (Wt, Mt are n_t x n_t). Outputs (caller-allocated host arrays):
 *     U[l]  n[l] x n[l] column-major,  lam[l]  n[l],
 *     Ut    n_t x n_t column-major,    lamt  q entries,  g  n_t - 1,
 *     sigma 1 value, *n_pairs = q, *has_zero = 1 if the zero block exists.
 * Any output pointer may be NULL. Returns STFD_ERR_NOT_SPD if a mass matrix
 * is not SPD and STFD_ERR_EIG if an eigen-solver fails its checks.
 * ------------------------------------------------------------------------ */
int stfd_fd_factors(int d, const int* n, const double* const* K, const double* const* M,
                    const double* Wt, const double* Mt,
                    double* const* U, double* const* lam, double* Ut, double* lamt,
                    double* g, double* sigma, int* n_pairs, int* has_zero);

/* ------------------------------------------------------------------------
 * Preconditioner handle (Algorithm 1). d in {1, 2, 3}, 1 <= n[l] <= 256,
 * 2 <= n_t <= 256, gamma > 0, nu > 0, precision one of STFD_FP64 / STFD_TF32 /
 * STFD_BF16 / STFD_DF32 / STFD_FP64TC / STFD_FP64TC7 (low precision: n[l] <= 128;
 * digit-sliced: n[l] <= 80). The factorisation runs on the host;
 * factors are uploaded on `stream` and the call synchronises that stream
 * before returning. Device memory held: the factors, one N-vector of
 * scratch and N_s Schur-complement reciprocals.
 * ------------------------------------------------------------------------ */
typedef struct stfd_fd stfd_fd;

int stfd_fd_setup(stfd_fd** out, int d, const int* n,
                  const double* const* K, const double* const* M,
                  const double* Wt, const double* Mt,
                  double gamma, double nu, int precision, void* stream);

/* s_dev = P^{-1} r_dev for nrhs right-hand sides (Algorithm 1, Steps 2-4):
 * s~ = (U_t^T (x) U_s^T) r, q~ = (gamma Delta_t (x) I + nu I (x) Lambda_s)^{-1} s~
 * by the block LU of eq. block_LU, s = (U_t (x) U_s) q~. r_dev and s_dev may
 * not overlap. Calls on one handle must not overlap in time (shared scratch). */
int stfd_fd_apply(const stfd_fd* h, const double* r_dev, double* s_dev, int nrhs, void* stream);

/* s_dev = P^{-T} r_dev, the transposed preconditioner, as used by the adjoint
 * solve. Not in the paper; it follows from its factorisation (Sec. 4.2-4.5):
 * P^{-T} = (U_t (x) U_s) (gamma Delta_t^T (x) I + nu I (x) Lambda_s)^{-1}
 * (U_t^T (x) U_s^T) with the same factors, and Delta_t^T is the arrowhead of
 * the Remark in Sec. 4.5 with lambda_j and g negated (the Schur complement is
 * unchanged). Arguments, precision and errors as stfd_fd_apply. */
int stfd_fd_apply_transpose(const stfd_fd* h, const double* r_dev, double* s_dev, int nrhs, void* stream);

/* Problem sizes of a handle: n[0..d] (array of d+1 ints) and *N_out. */
int stfd_fd_shape(const stfd_fd* h, int* d_out, int* n, long long* N_out);

void stfd_fd_destroy(stfd_fd* h);

/* ------------------------------------------------------------------------
 * System operator A = gamma W_t (x) M_s + nu M_t (x) K_s (eq. syst_mat) with
 * banded univariate factors (bandwidth 2p+1 is detected from the entries;
 * any dense factor works, only slower). Same size limits as stfd_fd_setup.
 * The factors are uploaded on `stream`, which is synchronised.
 * `arith` selects the arithmetic of the banded products:
 *   STFD_OP_FP64  FP64 fused multiply-adds (IEEE double throughout);
 *   STFD_OP_DF32  double-float on the FP32 pipes: every value is an unevaluated
 *                 pair hi + lo of floats (about 48 significant bits), products
 *                 split exactly by FMA, sums by error-free two-sum; FP64 input
 *                 and output. Agrees with STFD_OP_FP64 to about 1e-14 relative
 *                 and is several times faster on GPUs with low FP64 throughput.
 *                 The input is scaled exactly by a power of two (its largest
 *                 entry to [1, 2)) and the result scaled back, so FP32's exponent
 *                 range does not limit it (two extra passes over the vector and
 *                 one N-vector of scratch).
 *   STFD_OP_FX64  FP64 results, intermediates and inputs; each band product is
 *                 formed exactly in 64-bit integer arithmetic (every fibre of the
 *                 input and every band row written as 53-bit integers under their
 *                 own powers of two, 27-bit limbs, 3 integer multiply-adds per
 *                 tap, Karatsuba) and rounded once to FP64; an output summing two products
 *                 of different inputs sums them exactly and rounds once when their
 *                 scales are within 2^16 (else adds the two rounded FP64 values). Entries
 *                 far below their fibre's largest entry are rounded at 2^-53 of
 *                 that entry (normwise FP64 accuracy). A non-finite input entry
 *                 makes every output of the fibres it feeds NaN (the passes
 *                 carry it along whole fibres, so the result is NaN far beyond
 *                 the entry's band). Needs every half-bandwidth
 *                 in 1..4; otherwise the op uses the STFD_OP_FP64 passes.
 * ------------------------------------------------------------------------ */
typedef struct stfd_op stfd_op;
enum { STFD_OP_FP64 = 0, STFD_OP_DF32 = 1, STFD_OP_FX64 = 2 };

int stfd_op_create_kron(stfd_op** out, int d, const int* n,
                        const double* const* K, const double* const* M,
                        const double* Wt, const double* Mt,
                        double gamma, double nu, int arith, void* stream);

/* y_dev = A x_dev for nrhs vectors (matrix-free, sum-factorised through eq.
 * kron_vec_multi: 3d+1 banded mode products). x_dev and y_dev may not
 * overlap. Calls on one op must not overlap in time (shared scratch). */
int stfd_st_matvec(const stfd_op* A, const double* x_dev, double* y_dev, int nrhs, void* stream);

/* y_dev = A^T x_dev = (gamma W_t^T (x) M_s + nu M_t (x) K_s) x_dev (W_t is the
 * only non-symmetric factor, eq. time_mat). Used by the adjoint solve; not in
 * the paper. Arguments and errors as stfd_st_matvec. */
int stfd_st_matvec_transpose(const stfd_op* A, const double* x_dev, double* y_dev, int nrhs, void* stream);

void stfd_op_destroy(stfd_op* A);

/* ------------------------------------------------------------------------
 * Right-preconditioned flexible GMRES(restart) for A u = f with x0 = 0
 * (Sec. 4.5, Sec. 5: tolerance 1e-8, zero initial guess, Krylov dimension
 * 100). Classical Gram-Schmidt with one re-orthogonalisation, Givens
 * rotations on the host. Stops when the residual estimate
 * |g_{j+1}| <= tol ||f||, then computes the true residual ||f - A u|| / ||f||.
 * f_dev, u_dev: device N-vectors (one right-hand side). The call blocks the
 * host (one small device-to-host read per iteration) and returns when u_dev
 * is final. Krylov vectors (2 * restart + 1 N-vectors) are allocated on the
 * first call and cached in the op. `history` (optional, host, hist_cap
 * entries) receives the relative residual estimate per iteration.
 * ------------------------------------------------------------------------ */
typedef struct {
  double tol;        /* relative residual target, default 1e-8 */
  int restart;       /* Krylov dimension per cycle, default 100 */
  int max_it;        /* total iterations, default 1000 */
  int transpose;     /* 0: solve A u = f with P^{-1};  1: solve the adjoint
                        A^T u = f with P^{-T} (default 0) */
} stfd_gmres_opts;

typedef struct {
  int iters;              /* iterations done (preconditioner applications) */
  int converged;          /* 1 if the estimate reached tol */
  double rel_res_est;     /* |g_{j+1}| / ||f|| at exit */
  double rel_res_true;    /* ||f - A u|| / ||f|| at exit */
  double* history;        /* optional host array */
  int hist_cap;           /* its capacity */
  int hist_len;           /* entries written */
} stfd_gmres_info;

void stfd_gmres_default_opts(stfd_gmres_opts* opts);

int stfd_gmres_solve(const stfd_op* A, const stfd_fd* P, const double* f_dev, double* u_dev,
                     const stfd_gmres_opts* opts, stfd_gmres_info* info, void* stream);

/* ------------------------------------------------------------------------
 * Mapped domains and variable coefficients (Sec. 4.6 and 4.6.1).
 *
 * With a geometry map F of the parametric box (0,1)^d and time-independent
 * coefficients c(x) (heat capacity, gamma_s) and kappa(x) (conductivity,
 * nu_s), the system is A = gamma W_t (x) M_s + nu M_t (x) K_s with general
 * sparse spatial matrices (the parametric form of [A]_{ij} in Sec. 4.6):
 *     [M_s]_{ij} = int c(F) B^_i B^_j |det J|,
 *     [K_s]_{ij} = int kappa(F) grad^B^_i . J^{-1} J^{-T} grad^B^_j |det J|.
 *
 * Geometries (d = spatial dimension):
 *   STFD_GEOM_BOX              F = identity on (0,1)^d.
 *   STFD_GEOM_QUARTER_ANNULUS  F(eta) = (1 + eta_1) C(eta_2) [, eta_3], d in {2, 3}:
 *                              the quarter of the annulus with radii 1 and 2
 *                              (Sec. 5), C the exact rational quadratic (NURBS)
 *                              quarter circle with control points (1,0), (1,1),
 *                              (0,1) and weights 1, 1/sqrt(2), 1; extruded over
 *                              (0,1) in the third direction when d = 3.
 *   STFD_GEOM_REVOLVED_QUARTER_ANNULUS  d = 3: the planar quarter annulus
 *                              (a, b) = (1 + eta_1) C(eta_2) turned by a right
 *                              angle about the axis {(x_1, -1, 0)} (Sec. 5.1):
 *                              F = (a, -1 + (b+1) C_x(eta_3), (b+1) C_y(eta_3)).
 * The discrete space is the push-forward of the parametric splines (eq.
 * disc_space): degree p, n_el uniform elements and maximal smoothness per
 * direction, Dirichlet reduction in every direction (n_s = n_el + p - 2).
 *
 * Tensor-product stencil layout of a spatial matrix S (N_s x N_s with
 * N_s = n_s^d): in a tensor-product spline space S[i][j] = 0 unless
 * |i_l - j_l| <= p in every direction, so S is stored as (2p+1)^d arrays of
 * N_s values,  st[o * N_s + i] = S[i][i + sum_l (o_l - p) n_s^(l-1)]  with
 * o = sum_l o_l (2p+1)^(l-1), o_l in 0..2p (direction 1 fastest), and 0
 * wherever that column lies outside the box.
 *
 * Quadrature: nq Gauss points per element and direction (nq >= p + 1).
 * Points, elements and local functions are numbered colexicographically
 * (direction 1 fastest); point k of element e is entry e * nq^d + k.
 * ------------------------------------------------------------------------ */
enum { STFD_GEOM_BOX = 0, STFD_GEOM_QUARTER_ANNULUS = 1, STFD_GEOM_REVOLVED_QUARTER_ANNULUS = 2 };

/* Physical coordinates of the quadrature points (host): x[a * Q + k] for
 * coordinate a < d and point k < Q = n_el^d nq^d. The caller evaluates c and
 * kappa there for stfd_spatial_assemble. */
int stfd_spatial_quadrature_points(int d, int p, int n_el, int geom, int nq, double* x);

/* Physical coordinates of the element midpoints F((e + 1/2) / n_el) (host):
 * x[a * n_el^d + e]. Coefficient values there feed stfd_geo_separate. */
int stfd_spatial_element_midpoints(int d, int n_el, int geom, double* x);

/* Assemble M_s and K_s (host, multi-threaded) in the stencil layout; c_q and
 * kappa_q hold the coefficients at the Q quadrature points (NULL = 1). Ms and
 * Ks (either may be NULL) receive (2p+1)^d * N_s doubles each. */
int stfd_spatial_assemble(int d, int p, int n_el, int geom, int nq, const double* c_q, const double* kappa_q,
                          double* Ms, double* Ks);

/* Element stiffness matrices of unit conductivity (host): Ke receives n_el^d
 * blocks of (p+1)^d x (p+1)^d doubles, block e holding K_e[a][b] at
 * e * (p+1)^(2d) + a * (p+1)^d + b over the element's local functions
 * (including those removed by the Dirichlet reduction), so that
 * K_s = sum_e kappa_e K_e for a piecewise-constant conductivity. */
int stfd_spatial_element_stiffness(int d, int p, int n_el, int geom, int nq, double* Ke);

/* Separation of variables of eq. separation (host): the diagonal of the
 * coefficient matrix frak{C} -- kappa |det J| [J^{-1} J^{-T}]_{ll} for l <= d
 * and c |det J| -- is interpolated by its value at each element midpoint
 * (c_mid, kappa_mid: coefficient values there, NULL = 1) and fitted by
 *     C_{d+1} ~ phi_1 .. phi_d,   C_l ~ phi_1 .. Phi_l .. phi_d,
 * by least squares in log space on the element grid (univariate factors from
 * marginal means; the paper cites another work for its algorithm, this is the
 * reading used here). phi, Phi receive d x n_el values (phi[l * n_el + k]).
 * Returns STFD_ERR_ARG for non-positive data. */
int stfd_geo_separate(int d, int n_el, int geom, const double* c_mid, const double* kappa_mid, double* phi,
                      double* Phi);

/* Weighted univariate matrices of eq. over_A (host):
 * M[i,j] = int w_mass b_i b_j, K[i,j] = int w_stiff b'_i b'_j with weights
 * constant per element (n_el values each, NULL = 1); otherwise as
 * stfd_spline_matrices. */
int stfd_spline_matrices_weighted(int p, int n_el, double length, int bc, const double* w_mass,
                                  const double* w_stiff, double* M, double* K, int* n_out);

/* System operator with general spatial matrices: Ms, Ks host arrays in the
 * stencil layout with half-bandwidth p_s ((2p_s+1)^d * N_s doubles each),
 * n[0..d-1] = n_s per direction, n[d] = n_t, Wt and Mt the column-major time
 * factors. arith as stfd_op_create_kron (STFD_OP_DF32 keeps the coefficients
 * and intermediates as double-float pairs). STFD_OP_FX64: the time pass in
 * IEEE FP64, then every output of the spatial pass formed exactly in 64-bit
 * integers and rounded once to FP64 (each coefficient row written as 53-bit
 * integers under its largest entry's power of two, once, at creation; the
 * entries of each time slice that a block of 256 rows reads written under
 * their largest entry's power of two, so entries far below it are rounded at
 * 2^-53 of it; balanced 27-bit limbs, 3 integer multiply-adds per tap; the
 * mass and stiffness parts summed exactly and rounded once when their scales
 * are within 2^10, else added in FP64); needs (2p_s+1)^d <= 729, otherwise
 * the op uses IEEE FP64. A non-finite coefficient or input value gives NaN
 * where it is read. The op works with
 * stfd_st_matvec, stfd_st_matvec_transpose (A^T: M_s and K_s are symmetric)
 * and stfd_gmres_solve. Device memory: the two coefficient arrays (8 bytes
 * per entry in every arithmetic), two N-vectors of scratch and, for
 * STFD_OP_FX64, 2 N_s row exponents. */
int stfd_op_create_stencil(stfd_op** out, int d, const int* n, int p_s, const double* Ms, const double* Ks,
                           const double* Wt, const double* Mt, double gamma, double nu, int arith, void* stream);

/* Diagonal scaling of the geometry-aware preconditioner (eq. prec_geo):
 * after this call the handle applies P = D^{1/2} A~ D^{1/2}, where A~ is the
 * operator of its univariate factors and D = diag(A) / diag(A~) per dof, from
 * Ms_diag and Ks_diag (host, N_s each): the diagonals of the true spatial
 * matrices of A. Both NULL removes the scaling. Part of the set-up: not to be
 * called while an apply on the handle is in flight. Device memory: two
 * N-vectors. Synchronises `stream`. */
int stfd_fd_set_scaling(stfd_fd* h, const double* Ms_diag, const double* Ks_diag, void* stream);

/* Gradient of a loss with respect to a piecewise-constant conductivity
 * kappa_e (K_s = sum_e kappa_e K_e), not in the paper: with A u = f and the
 * adjoint solution lam of A^T lam = dL/du,
 *     g_e = dL/dkappa_e = -nu lam^T (M_t (x) K_e) u.
 * Ke_dev: device copy of stfd_spatial_element_stiffness's output for the
 * same (d, p, n_el); lam_dev, u_dev: device N-vectors; g_dev: device, n_el^d
 * values. Requires n_s = n_el + p - 2 in every direction of A and
 * (p+1)^(2d) doubles of shared memory per element (about 200 KiB at most).
 * Uses the op's scratch: not concurrent with other calls on A. */
int stfd_grad_kappa_elements(const stfd_op* A, int p, int n_el, const double* Ke_dev, const double* lam_dev,
                             const double* u_dev, double* g_dev, void* stream);

/* ------------------------------------------------------------------------
 * Batched solver: many independent small heat problems on the unit box
 * (0,1)^d x (0,T), constant coefficients gamma, nu, each with its own number
 * of elements n_el[k], degree p[k] (space and time) and number of right-hand
 * sides nrhs[k]. Not a section of the paper: it batches its method. On the
 * unit box the preconditioner of eq. prec_definition equals A (Sec. 4); each
 * item runs FD-preconditioned iterative refinement (see stfd_batch_create_ex)
 * with the true relative residual ||f - A u|| / ||f|| (eq. syst_mat,
 * sum-factorised) checked after every step, in IEEE FP64 or double-float.
 *
 * The work runs as ONE persistent kernel launch: every CTA repeatedly takes
 * the next (problem, right-hand side) item from a list sorted by size
 * (largest first) and solves it alone. stfd_batch_solve captures the launch
 * (with the reset of the work counter) into a CUDA graph bound to the given
 * pointers and replays it on later calls with the same pointers.
 *
 * Limits: d in {1,2,3}; 1 <= p[k] <= 10; n_s = n_el + p - 2 >= 1;
 * n_s, n_t <= 256; at most 2^20 dofs per problem; count >= 1.
 * autotune != 0 times every candidate CTA configuration (threads per CTA x
 * CTAs per SM, see stfd_batch_stats) on the batch with synthetic right-hand
 * sides and keeps the fastest; otherwise 256 threads x the largest of 4, 2, 1
 * CTAs per SM that fits.
 * Device memory: factors, 4 * max_N float pairs of scratch per CTA slot
 * (SMs x the largest CTAs-per-SM count that can be launched) and the work list.
 * ------------------------------------------------------------------------ */
typedef struct stfd_batch stfd_batch;

int stfd_batch_create(stfd_batch** out, int count, int d, const int* n_el, const int* p, const int* nrhs,
                      double T, double gamma, double nu, int autotune, void* stream);

/* As stfd_batch_create, with the arithmetic and the refinement of each item:
 * precision STFD_FP64 (IEEE FP64 on the FP64 pipe) or STFD_DF32 (double-float);
 * every item runs FD-preconditioned iterative refinement, u_0 = 0 and
 * u_{k+1} = u_k + P^{-1} (f - A u_k) by Algorithm 1, until the true relative
 * residual ||f - A u|| / ||f|| <= tol or max_it iterations (1 <= max_it <=
 * 1000, tol >= 0). stfd_batch_create is precision STFD_DF32, tol 0, max_it 1
 * (one application). Device memory: the factors in the chosen arithmetic, 5 x
 * max_N 8-byte entries of scratch per CTA slot and one int per item. */
int stfd_batch_create_ex(stfd_batch** out, int count, int d, const int* n_el, const int* p, const int* nrhs,
                         double T, double gamma, double nu, int precision, double tol, int max_it, int autotune,
                         void* stream);

/* After a solve has completed: iterations done per item (n_items ints, item
 * order as relres: problem-major, then right-hand side). An item whose
 * relres is still above tol used all max_it iterations. Synchronous. */
int stfd_batch_iterations(const stfd_batch* b, int* iters);

/* Packed vector layout: problem k's nrhs[k] right-hand sides (each of
 * N_k = n_s^d n_t dofs, vec order) start at offsets[k] (count + 1 entries,
 * offsets[count] = total). *n_items = sum of nrhs. Any output may be NULL. */
int stfd_batch_layout(const stfd_batch* b, long long* offsets, int* n_items, long long* total);

/* u_dev = P_k^{-1} f_dev per problem and right-hand side (packed layout);
 * relres_dev (optional, n_items doubles, problem-major then right-hand side)
 * receives ||f - A u|| / ||f||. f_dev and u_dev must not overlap. Calls on one
 * batch must not overlap in time (shared work counter and scratch). The first
 * call with a new (f, u, relres) pointer triple captures and instantiates the
 * graph. */
int stfd_batch_solve(stfd_batch* b, const double* f_dev, double* u_dev, double* relres_dev, void* stream);

/* After a solve has completed: per-problem solve time in microseconds (first
 * start to last end of its right-hand sides, device global timer) in
 * problem_us (count entries), the chosen configuration, and the autotuning
 * times in milliseconds per candidate (NaN if not run or infeasible; the 8
 * candidates are 128x2, 128x4, 128x8, 256x1, 256x2, 256x4, 512x1, 512x2
 * threads x CTAs per SM). Any output may be NULL. Synchronous. */
int stfd_batch_stats(const stfd_batch* b, double* problem_us, int* threads, int* ctas_per_sm, double* tune_ms,
                     int tune_cap);

/* Work-list order: item idx (0 <= idx < n_items) solves right-hand side *rhs
 * of problem *problem. */
int stfd_batch_item(const stfd_batch* b, int idx, int* problem, int* rhs);

void stfd_batch_destroy(stfd_batch* b);

/* ------------------------------------------------------------------------
 * Allocation-free system matvec. The paper has no counterpart: this entry
 * point serves callers that must not allocate device memory -- for example a
 * host application that owns every byte of device memory through its own
 * allocator and memory budget, or a latency-critical loop where cudaMalloc /
 * cudaFree would synchronise the device and stall other streams.
 *
 * Computes y_dev = A x_dev exactly like stfd_st_matvec (same sum-factorised
 * banded products), but takes the univariate matrices as caller-owned device
 * arrays and keeps its scratch (four partial-sum tensors) in one static device
 * array of 4 * STFD_NOALLOC_MAX_N doubles (16 MiB) that every GPU loading the
 * library holds until the process exits. It calls no allocating routine.
 *   n[0..d]   sizes as in stfd_op_create_kron; N = prod n must not exceed
 *             STFD_NOALLOC_MAX_N (else STFD_ERR_ARG, nothing launched)
 *   K_dev[l], M_dev[l]  device, column-major n[l] x n[l]; Wt_dev, Mt_dev n_t x n_t
 *   bw        host array of d+1 half-bandwidths (space directions, then time:
 *             max over the two matrices of that direction); NULL or a
 *             negative entry treats that direction as dense
 *   x_dev, y_dev        device N-vectors, must not overlap
 * The first call on a device looks up the static array's device address
 * (cudaGetSymbolAddress, with that device current) and caches it; make that
 * first call before any stream capture. All calls share the one array, which
 * keeps the last call's contents; every scratch element is written before it is
 * read within a call, so nothing needs clearing. Calls that overlap on the GPU
 * (concurrent streams, or several host threads) race on the scratch: order them.
 * ------------------------------------------------------------------------ */
#define STFD_NOALLOC_MAX_N 524288

int stfd_st_matvec_noalloc(int d, const int* n, const double* const* K_dev, const double* const* M_dev,
                           const double* Wt_dev, const double* Mt_dev, const int* bw,
                           double gamma, double nu, const double* x_dev, double* y_dev, void* stream);

#ifdef __cplusplus
}
#endif
#endif /* STFD_H */
