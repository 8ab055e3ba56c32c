"""Python binding of the C ABI in ``include/stfd.h`` (ctypes; marshalling only).

Every numerical step runs in ``lib/libstfd.so``: the host-side setup in its
C++ code and the apply / matvec / GMRES path in its CUDA kernels. This module
only converts arguments (numpy arrays for host data, torch CUDA tensors for
device data, torch's current stream) and raises on error codes. There is no
fallback: if the library is missing or fails to load, every call raises.
"""
import ctypes
import os

import numpy as np

from . import build as _build

STFD_OK = 0
STFD_NOT_CONVERGED = 1
STFD_FP64, STFD_TF32, STFD_BF16, STFD_DF32, STFD_FP64TC, STFD_FP64TC7 = 0, 1, 2, 3, 4, 5
STFD_BC_NONE, STFD_BC_INITIAL, STFD_BC_DIRICHLET = 0, 1, 2
STFD_NOALLOC_MAX_N = 524288
STFD_OP_FP64, STFD_OP_DF32, STFD_OP_FX64 = 0, 1, 2
STFD_GEOM_BOX, STFD_GEOM_QUARTER_ANNULUS, STFD_GEOM_REVOLVED_QUARTER_ANNULUS = 0, 1, 2

_c_int_p = ctypes.POINTER(ctypes.c_int)
_c_dbl_p = ctypes.POINTER(ctypes.c_double)
_c_dbl_pp = ctypes.POINTER(_c_dbl_p)
_lib = None


class StfdError(RuntimeError):
    def __init__(self, code, what):
        self.code = code
        super().__init__("%s failed: %s (%d)" % (what, _strerror(code), code))


class GmresOpts(ctypes.Structure):
    _fields_ = [("tol", ctypes.c_double), ("restart", ctypes.c_int), ("max_it", ctypes.c_int),
                ("transpose", ctypes.c_int)]


class GmresInfo(ctypes.Structure):
    _fields_ = [("iters", ctypes.c_int), ("converged", ctypes.c_int),
                ("rel_res_est", ctypes.c_double), ("rel_res_true", ctypes.c_double),
                ("history", _c_dbl_p), ("hist_cap", ctypes.c_int), ("hist_len", ctypes.c_int)]


# Exported symbols and their signatures: (restype, argtypes).
SIGNATURES = {
    "stfd_strerror": (ctypes.c_char_p, [ctypes.c_int]),
    "stfd_version": (ctypes.c_int, []),
    "stfd_device_status": (ctypes.c_int, []),
    "stfd_set_wait_limit": (ctypes.c_int, [ctypes.c_longlong]),
    "stfd_get_wait_limit": (ctypes.c_longlong, []),
    "stfd_spline_matrices": (ctypes.c_int, [ctypes.c_int, ctypes.c_int, ctypes.c_double, ctypes.c_int,
                                            _c_dbl_p, _c_dbl_p, _c_dbl_p, _c_int_p]),
    "stfd_spline_load_trig": (ctypes.c_int, [ctypes.c_int, ctypes.c_int, ctypes.c_double, ctypes.c_int,
                                             ctypes.c_double, ctypes.c_double, ctypes.c_double, _c_dbl_p]),
    "stfd_fd_factors": (ctypes.c_int, [ctypes.c_int, _c_int_p, _c_dbl_pp, _c_dbl_pp, _c_dbl_p, _c_dbl_p,
                                       _c_dbl_pp, _c_dbl_pp, _c_dbl_p, _c_dbl_p, _c_dbl_p, _c_dbl_p,
                                       _c_int_p, _c_int_p]),
    "stfd_fd_setup": (ctypes.c_int, [ctypes.POINTER(ctypes.c_void_p), ctypes.c_int, _c_int_p, _c_dbl_pp,
                                     _c_dbl_pp, _c_dbl_p, _c_dbl_p, ctypes.c_double, ctypes.c_double,
                                     ctypes.c_int, ctypes.c_void_p]),
    "stfd_fd_apply": (ctypes.c_int, [ctypes.c_void_p, ctypes.c_void_p, ctypes.c_void_p, ctypes.c_int,
                                     ctypes.c_void_p]),
    "stfd_fd_apply_transpose": (ctypes.c_int, [ctypes.c_void_p, ctypes.c_void_p, ctypes.c_void_p, ctypes.c_int,
                                               ctypes.c_void_p]),
    "stfd_fd_shape": (ctypes.c_int, [ctypes.c_void_p, _c_int_p, _c_int_p, ctypes.POINTER(ctypes.c_longlong)]),
    "stfd_fd_destroy": (None, [ctypes.c_void_p]),
    "stfd_op_create_kron": (ctypes.c_int, [ctypes.POINTER(ctypes.c_void_p), ctypes.c_int, _c_int_p, _c_dbl_pp,
                                           _c_dbl_pp, _c_dbl_p, _c_dbl_p, ctypes.c_double, ctypes.c_double,
                                           ctypes.c_int, ctypes.c_void_p]),
    "stfd_st_matvec": (ctypes.c_int, [ctypes.c_void_p, ctypes.c_void_p, ctypes.c_void_p, ctypes.c_int,
                                      ctypes.c_void_p]),
    "stfd_st_matvec_transpose": (ctypes.c_int, [ctypes.c_void_p, ctypes.c_void_p, ctypes.c_void_p, ctypes.c_int,
                                                ctypes.c_void_p]),
    "stfd_op_destroy": (None, [ctypes.c_void_p]),
    "stfd_gmres_default_opts": (None, [ctypes.POINTER(GmresOpts)]),
    "stfd_gmres_solve": (ctypes.c_int, [ctypes.c_void_p, ctypes.c_void_p, ctypes.c_void_p, ctypes.c_void_p,
                                        ctypes.POINTER(GmresOpts), ctypes.POINTER(GmresInfo), ctypes.c_void_p]),
    "stfd_st_matvec_noalloc": (ctypes.c_int, [ctypes.c_int, _c_int_p, ctypes.POINTER(ctypes.c_void_p),
                                              ctypes.POINTER(ctypes.c_void_p), ctypes.c_void_p, ctypes.c_void_p,
                                              _c_int_p, ctypes.c_double, ctypes.c_double, ctypes.c_void_p,
                                              ctypes.c_void_p, ctypes.c_void_p]),
    "stfd_spatial_quadrature_points": (ctypes.c_int, [ctypes.c_int, ctypes.c_int, ctypes.c_int, ctypes.c_int,
                                                      ctypes.c_int, _c_dbl_p]),
    "stfd_spatial_element_midpoints": (ctypes.c_int, [ctypes.c_int, ctypes.c_int, ctypes.c_int, _c_dbl_p]),
    "stfd_spatial_assemble": (ctypes.c_int, [ctypes.c_int, ctypes.c_int, ctypes.c_int, ctypes.c_int, ctypes.c_int,
                                             _c_dbl_p, _c_dbl_p, _c_dbl_p, _c_dbl_p]),
    "stfd_spatial_element_stiffness": (ctypes.c_int, [ctypes.c_int, ctypes.c_int, ctypes.c_int, ctypes.c_int,
                                                      ctypes.c_int, _c_dbl_p]),
    "stfd_geo_separate": (ctypes.c_int, [ctypes.c_int, ctypes.c_int, ctypes.c_int, _c_dbl_p, _c_dbl_p, _c_dbl_p,
                                         _c_dbl_p]),
    "stfd_spline_matrices_weighted": (ctypes.c_int, [ctypes.c_int, ctypes.c_int, ctypes.c_double, ctypes.c_int,
                                                     _c_dbl_p, _c_dbl_p, _c_dbl_p, _c_dbl_p, _c_int_p]),
    "stfd_op_create_stencil": (ctypes.c_int, [ctypes.POINTER(ctypes.c_void_p), ctypes.c_int, _c_int_p, ctypes.c_int,
                                              _c_dbl_p, _c_dbl_p, _c_dbl_p, _c_dbl_p, ctypes.c_double,
                                              ctypes.c_double, ctypes.c_int, ctypes.c_void_p]),
    "stfd_fd_set_scaling": (ctypes.c_int, [ctypes.c_void_p, _c_dbl_p, _c_dbl_p, ctypes.c_void_p]),
    "stfd_grad_kappa_elements": (ctypes.c_int, [ctypes.c_void_p, ctypes.c_int, ctypes.c_int, ctypes.c_void_p,
                                                ctypes.c_void_p, ctypes.c_void_p, ctypes.c_void_p, ctypes.c_void_p]),
    "stfd_batch_create": (ctypes.c_int, [ctypes.POINTER(ctypes.c_void_p), ctypes.c_int, ctypes.c_int, _c_int_p,
                                         _c_int_p, _c_int_p, ctypes.c_double, ctypes.c_double, ctypes.c_double,
                                         ctypes.c_int, ctypes.c_void_p]),
    "stfd_batch_create_ex": (ctypes.c_int, [ctypes.POINTER(ctypes.c_void_p), ctypes.c_int, ctypes.c_int, _c_int_p,
                                            _c_int_p, _c_int_p, ctypes.c_double, ctypes.c_double, ctypes.c_double,
                                            ctypes.c_int, ctypes.c_double, ctypes.c_int, ctypes.c_int,
                                            ctypes.c_void_p]),
    "stfd_batch_iterations": (ctypes.c_int, [ctypes.c_void_p, _c_int_p]),
    "stfd_batch_layout": (ctypes.c_int, [ctypes.c_void_p, ctypes.POINTER(ctypes.c_longlong), _c_int_p,
                                         ctypes.POINTER(ctypes.c_longlong)]),
    "stfd_batch_solve": (ctypes.c_int, [ctypes.c_void_p, ctypes.c_void_p, ctypes.c_void_p, ctypes.c_void_p,
                                        ctypes.c_void_p]),
    "stfd_batch_stats": (ctypes.c_int, [ctypes.c_void_p, _c_dbl_p, _c_int_p, _c_int_p, _c_dbl_p, ctypes.c_int]),
    "stfd_batch_item": (ctypes.c_int, [ctypes.c_void_p, ctypes.c_int, _c_int_p, _c_int_p]),
    "stfd_batch_destroy": (None, [ctypes.c_void_p]),
    # include/stfd_profile.h
    "stfd_profile_enable": (ctypes.c_int, [ctypes.c_int]),
    "stfd_profile_reset": (ctypes.c_int, []),
    "stfd_profile_count": (ctypes.c_int, []),
    "stfd_profile_get": (ctypes.c_int, [ctypes.c_int, ctypes.c_char_p, ctypes.c_int,
                                        ctypes.POINTER(ctypes.c_longlong), _c_dbl_p, _c_dbl_p, _c_dbl_p]),
    "stfd_launch_count": (ctypes.c_longlong, []),
    "stfd_probe_fp64_peak": (ctypes.c_int, [_c_dbl_p, ctypes.c_void_p]),
    "stfd_probe_imad_wide_peak": (ctypes.c_int, [_c_dbl_p, ctypes.c_void_p]),
    "stfd_probe_bounded_wait": (ctypes.c_int, [ctypes.c_int, ctypes.c_void_p]),
    "stfd_probe_convert": (ctypes.c_int, [ctypes.c_void_p, ctypes.c_longlong, ctypes.c_void_p, ctypes.c_void_p,
                                          ctypes.c_void_p, ctypes.c_void_p, ctypes.c_void_p]),
}


def library_path():
    return _build.LIB


def load(build_if_missing=True):
    """Load libstfd.so (building it first if it is absent and nvcc exists)."""
    global _lib
    if _lib is not None:
        return _lib
    path = library_path()
    if not os.path.exists(path):
        if not build_if_missing:
            raise RuntimeError("libstfd.so is not built (%s); run paper_1909_07309_gb300.build" % path)
        _build.build()
    lib = ctypes.CDLL(path)
    for name, (res, args) in SIGNATURES.items():
        fn = getattr(lib, name)
        fn.restype = res
        fn.argtypes = args
    _lib = lib
    return lib


def _strerror(code):
    try:
        return load().stfd_strerror(int(code)).decode()
    except Exception:   # the library itself is unavailable
        return "status"


def _check(rc, what, allow_not_converged=False):
    if rc == STFD_OK or (allow_not_converged and rc == STFD_NOT_CONVERGED):
        return rc
    raise StfdError(rc, what)


def _f64(a):
    return np.asfortranarray(np.asarray(a, dtype=np.float64))


def _dptr(a):
    return a.ctypes.data_as(_c_dbl_p)


def _ptr_array(arrs):
    return (_c_dbl_p * len(arrs))(*[_dptr(a) for a in arrs])


def _stream(stream):
    if stream is not None:
        return ctypes.c_void_p(int(stream))
    import torch
    return ctypes.c_void_p(torch.cuda.current_stream().cuda_stream)


def _dev(t, N, what):
    import torch
    if not isinstance(t, torch.Tensor) or not t.is_cuda or t.dtype != torch.float64 or not t.is_contiguous():
        raise TypeError("%s must be a contiguous float64 CUDA tensor" % what)
    if t.numel() % N != 0:
        raise ValueError("%s has %d entries, not a multiple of N = %d" % (what, t.numel(), N))
    return ctypes.c_void_p(t.data_ptr()), t.numel() // N


# ---------------------------------------------------------------------------
# host entry points
# ---------------------------------------------------------------------------

def stfd_spline_matrices(p, n_el, length=1.0, bc=STFD_BC_NONE):
    """(M, K, W) dense n x n univariate matrices (eq. time_mat / space_mat factors)."""
    lib = load()
    n = ctypes.c_int(0)
    _check(lib.stfd_spline_matrices(p, n_el, float(length), bc, None, None, None, ctypes.byref(n)),
           "stfd_spline_matrices")
    M, K, W = (np.zeros((n.value, n.value), order="F") for _ in range(3))
    _check(lib.stfd_spline_matrices(p, n_el, float(length), bc, _dptr(M), _dptr(K), _dptr(W), ctypes.byref(n)),
           "stfd_spline_matrices")
    return M, K, W


def stfd_spline_load_trig(p, n_el, length, bc, freq, c_sin, c_cos):
    lib = load()
    n = ctypes.c_int(0)
    _check(lib.stfd_spline_matrices(p, n_el, float(length), bc, None, None, None, ctypes.byref(n)),
           "stfd_spline_matrices")
    out = np.zeros(n.value)
    _check(lib.stfd_spline_load_trig(p, n_el, float(length), bc, float(freq), float(c_sin), float(c_cos),
                                     _dptr(out)), "stfd_spline_load_trig")
    return out


def stfd_fd_factors(K, M, Wt, Mt):
    """Host factors of Step 1 of Algorithm 1 (real arrowhead form), as a dict."""
    lib = load()
    d = len(K)
    K = [_f64(k) for k in K]
    M = [_f64(m) for m in M]
    Wt, Mt = _f64(Wt), _f64(Mt)
    n = [k.shape[0] for k in K] + [Wt.shape[0]]
    nt = n[-1]
    U = [np.zeros((nl, nl), order="F") for nl in n[:d]]
    lam = [np.zeros(nl) for nl in n[:d]]
    Ut = np.zeros((nt, nt), order="F")
    lamt = np.zeros(max(1, nt // 2))
    g = np.zeros(nt - 1)
    sigma = ctypes.c_double(0.0)
    npairs = ctypes.c_int(0)
    hz = ctypes.c_int(0)
    rc = lib.stfd_fd_factors(d, (ctypes.c_int * (d + 1))(*n), _ptr_array(K), _ptr_array(M), _dptr(Wt), _dptr(Mt),
                             _ptr_array(U), _ptr_array(lam), _dptr(Ut), _dptr(lamt), _dptr(g),
                             ctypes.byref(sigma), ctypes.byref(npairs), ctypes.byref(hz))
    _check(rc, "stfd_fd_factors")
    return {"U": U, "lam": lam, "Ut": Ut, "lamt": lamt[:npairs.value].copy(), "g": g,
            "sigma": sigma.value, "n_pairs": npairs.value, "has_zero": hz.value}


# ---------------------------------------------------------------------------
# device handles
# ---------------------------------------------------------------------------

class FD:
    """Preconditioner handle: ``stfd_fd_setup`` / ``stfd_fd_apply`` / ``stfd_fd_destroy``."""

    def __init__(self, K, M, Wt, Mt, gamma=1.0, nu=1.0, precision=STFD_FP64, stream=None):
        lib = load()
        self._lib = lib
        self.handle = ctypes.c_void_p()
        K = [_f64(k) for k in K]
        M = [_f64(m) for m in M]
        Wt, Mt = _f64(Wt), _f64(Mt)
        self.d = len(K)
        self.n = [k.shape[0] for k in K] + [Wt.shape[0]]
        self.N = int(np.prod(self.n))
        rc = lib.stfd_fd_setup(ctypes.byref(self.handle), self.d, (ctypes.c_int * (self.d + 1))(*self.n),
                               _ptr_array(K), _ptr_array(M), _dptr(Wt), _dptr(Mt), float(gamma), float(nu),
                               int(precision), _stream(stream))
        _check(rc, "stfd_fd_setup")

    def apply(self, r, s=None, stream=None, transpose=False):
        """s = P^{-1} r (or P^{-T} r) for r of shape (N,) or (nrhs, N); returns s."""
        import torch
        if s is None:
            s = torch.empty_like(r)
        rp, nrhs = _dev(r, self.N, "r")
        sp, nrhs2 = _dev(s, self.N, "s")
        if nrhs != nrhs2:
            raise ValueError("r and s hold different numbers of right-hand sides")
        name = "stfd_fd_apply_transpose" if transpose else "stfd_fd_apply"
        _check(getattr(self._lib, name)(self.handle, rp, sp, nrhs, _stream(stream)), name)
        return s

    def set_scaling(self, Ms_diag, Ks_diag, stream=None):
        """Diagonal scaling of eq. prec_geo from the diagonals of the true M_s, K_s
        (host arrays of N_s); None, None removes it."""
        if Ms_diag is None and Ks_diag is None:
            rc = self._lib.stfd_fd_set_scaling(self.handle, None, None, _stream(stream))
        else:
            a = np.ascontiguousarray(Ms_diag, dtype=np.float64)
            b = np.ascontiguousarray(Ks_diag, dtype=np.float64)
            if a.size * self.n[-1] != self.N or b.size != a.size:
                raise ValueError("diagonals must hold N_s entries")
            rc = self._lib.stfd_fd_set_scaling(self.handle, _dptr(a), _dptr(b), _stream(stream))
        _check(rc, "stfd_fd_set_scaling")

    def close(self):
        if self.handle:
            self._lib.stfd_fd_destroy(self.handle)
            self.handle = ctypes.c_void_p()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


class _Op:
    """Common part of the system operator handles: matvec, GMRES, gradient."""

    def grad_kappa_elements(self, p, n_el, Ke_dev, lam, u, g=None, stream=None):
        """g_e = -nu lam^T (M_t kron K_e) u per element (``stfd_grad_kappa_elements``)."""
        import torch
        if g is None:
            g = torch.empty(n_el ** self.d, dtype=torch.float64, device=u.device)
        lp, k1 = _dev(lam, self.N, "lam")
        up, k2 = _dev(u, self.N, "u")
        if k1 != 1 or k2 != 1 or g.numel() != n_el ** self.d or not g.is_contiguous():
            raise ValueError("one adjoint / state vector and n_el^d outputs")
        if Ke_dev.dtype != torch.float64 or not Ke_dev.is_cuda or not Ke_dev.is_contiguous():
            raise TypeError("Ke must be a contiguous float64 CUDA tensor")
        if Ke_dev.numel() != n_el ** self.d * (p + 1) ** (2 * self.d):
            raise ValueError("Ke must hold n_el^d blocks of (p+1)^d x (p+1)^d values")
        _check(self._lib.stfd_grad_kappa_elements(self.handle, int(p), int(n_el), ctypes.c_void_p(Ke_dev.data_ptr()),
                                                  lp, up, ctypes.c_void_p(g.data_ptr()), _stream(stream)),
               "stfd_grad_kappa_elements")
        return g


class KronOp(_Op):
    """System operator handle: ``stfd_op_create_kron`` / ``stfd_st_matvec`` / ``stfd_gmres_solve``."""

    def __init__(self, K, M, Wt, Mt, gamma=1.0, nu=1.0, arith=STFD_OP_FP64, stream=None):
        lib = load()
        self._lib = lib
        self.handle = ctypes.c_void_p()
        K = [_f64(k) for k in K]
        M = [_f64(m) for m in M]
        Wt, Mt = _f64(Wt), _f64(Mt)
        self.d = len(K)
        self.n = [k.shape[0] for k in K] + [Wt.shape[0]]
        self.N = int(np.prod(self.n))
        rc = lib.stfd_op_create_kron(ctypes.byref(self.handle), self.d, (ctypes.c_int * (self.d + 1))(*self.n),
                                     _ptr_array(K), _ptr_array(M), _dptr(Wt), _dptr(Mt), float(gamma),
                                     float(nu), int(arith), _stream(stream))
        _check(rc, "stfd_op_create_kron")

    def matvec(self, x, y=None, stream=None, transpose=False):
        """y = A x (or A^T x) for x of shape (N,) or (nrhs, N); returns y."""
        import torch
        if y is None:
            y = torch.empty_like(x)
        xp, nrhs = _dev(x, self.N, "x")
        yp, nrhs2 = _dev(y, self.N, "y")
        if nrhs != nrhs2:
            raise ValueError("x and y hold different numbers of vectors")
        name = "stfd_st_matvec_transpose" if transpose else "stfd_st_matvec"
        _check(getattr(self._lib, name)(self.handle, xp, yp, nrhs, _stream(stream)), name)
        return y

    def gmres(self, fd, f, u=None, tol=1e-8, restart=100, max_it=1000, hist_cap=1000, stream=None,
              transpose=False):
        """Solve A u = f (or the adjoint A^T u = f with P^{-T}) with FD-preconditioned
        flexible GMRES; returns (u, info dict)."""
        import torch
        if u is None:
            u = torch.empty_like(f)
        fp, k1 = _dev(f, self.N, "f")
        up, k2 = _dev(u, self.N, "u")
        if k1 != 1 or k2 != 1:
            raise ValueError("gmres solves one right-hand side")
        opts = GmresOpts(float(tol), int(restart), int(max_it), 1 if transpose else 0)
        hist = np.zeros(max(1, hist_cap))
        info = GmresInfo(0, 0, 0.0, 0.0, _dptr(hist), int(hist_cap), 0)
        rc = self._lib.stfd_gmres_solve(self.handle, fd.handle, fp, up, ctypes.byref(opts), ctypes.byref(info),
                                        _stream(stream))
        _check(rc, "stfd_gmres_solve", allow_not_converged=True)
        return u, {"iters": info.iters, "converged": bool(info.converged), "rel_res_est": info.rel_res_est,
                   "rel_res_true": info.rel_res_true, "history": hist[:info.hist_len].copy(), "status": rc}

    def close(self):
        if self.handle:
            self._lib.stfd_op_destroy(self.handle)
            self.handle = ctypes.c_void_p()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


class StencilOp(KronOp):
    """System operator with general spatial matrices in the stencil layout
    (``stfd_op_create_stencil``); matvec / transpose / GMRES as KronOp. The
    default arithmetic is FP64 with exact integer-limb row sums
    (STFD_OP_FX64); STFD_OP_FP64 (IEEE) and STFD_OP_DF32 (~48-bit) are the
    others."""

    def __init__(self, n, p_s, Ms, Ks, Wt, Mt, gamma=1.0, nu=1.0, arith=STFD_OP_FX64, stream=None):
        lib = load()
        self._lib = lib
        self.handle = ctypes.c_void_p()
        Wt, Mt = _f64(Wt), _f64(Mt)
        self.n = [int(v) for v in n]
        self.d = len(self.n) - 1
        self.N = int(np.prod(self.n))
        Ns = self.N // self.n[-1]
        Ms = np.ascontiguousarray(Ms, dtype=np.float64)
        Ks = np.ascontiguousarray(Ks, dtype=np.float64)
        if Ms.size != (2 * p_s + 1) ** self.d * Ns or Ks.size != Ms.size:
            raise ValueError("stencil arrays must hold (2p+1)^d * N_s values")
        rc = lib.stfd_op_create_stencil(ctypes.byref(self.handle), self.d, (ctypes.c_int * (self.d + 1))(*self.n),
                                        int(p_s), _dptr(Ms), _dptr(Ks), _dptr(Wt), _dptr(Mt), float(gamma),
                                        float(nu), int(arith), _stream(stream))
        _check(rc, "stfd_op_create_stencil")


class Batch:
    """Batched solver handle (``stfd_batch_*``): many small unit-box problems,
    one persistent graph-captured launch per solve."""

    CANDIDATES = [(128, 2), (128, 4), (128, 8), (256, 1), (256, 2), (256, 4), (512, 1), (512, 2)]

    def __init__(self, n_el, p, nrhs, d=2, T=1.0, gamma=1.0, nu=1.0, autotune=True, stream=None,
                 precision=STFD_DF32, tol=0.0, max_it=1):
        lib = load()
        self._lib = lib
        self.handle = ctypes.c_void_p()
        n_el, p, nrhs = (np.ascontiguousarray(a, dtype=np.int32) for a in (n_el, p, nrhs))
        if not (n_el.size == p.size == nrhs.size):
            raise ValueError("n_el, p and nrhs must have one entry per problem")
        self.count, self.d = int(n_el.size), int(d)
        self.n_el, self.p, self.nrhs = n_el, p, nrhs
        ip = ctypes.POINTER(ctypes.c_int)
        rc = lib.stfd_batch_create_ex(ctypes.byref(self.handle), self.count, self.d, n_el.ctypes.data_as(ip),
                                      p.ctypes.data_as(ip), nrhs.ctypes.data_as(ip), float(T), float(gamma),
                                      float(nu), int(precision), float(tol), int(max_it), 1 if autotune else 0,
                                      _stream(stream))
        _check(rc, "stfd_batch_create_ex")
        self.precision, self.tol, self.max_it = int(precision), float(tol), int(max_it)
        off = (ctypes.c_longlong * (self.count + 1))()
        ni = ctypes.c_int(0)
        tot = ctypes.c_longlong(0)
        _check(lib.stfd_batch_layout(self.handle, off, ctypes.byref(ni), ctypes.byref(tot)), "stfd_batch_layout")
        self.offsets = np.array(off[:], dtype=np.int64)
        self.n_items = ni.value
        self.total = tot.value

    def iterations(self):
        """Refinement iterations per item of the last completed solve (numpy int32)."""
        it = np.zeros(self.n_items, dtype=np.int32)
        _check(self._lib.stfd_batch_iterations(self.handle, it.ctypes.data_as(ctypes.POINTER(ctypes.c_int))),
               "stfd_batch_iterations")
        return it

    def sizes(self, k):
        """(n_s, n_t, N) of problem k."""
        ns = int(self.n_el[k] + self.p[k] - 2)
        nt = int(self.n_el[k] + self.p[k] - 1)
        return ns, nt, ns ** self.d * nt

    def solve(self, f, u=None, relres=None, stream=None):
        """u = P^{-1} f per problem / right-hand side (packed); returns (u, relres)."""
        import torch
        if u is None:
            u = torch.empty_like(f)
        if relres is None:
            relres = torch.empty(self.n_items, dtype=torch.float64, device=f.device)
        for t, n in ((f, self.total), (u, self.total), (relres, self.n_items)):
            if t.dtype != torch.float64 or not t.is_cuda or not t.is_contiguous() or t.numel() != n:
                raise ValueError("packed float64 CUDA vectors of the batch layout expected")
        _check(self._lib.stfd_batch_solve(self.handle, ctypes.c_void_p(f.data_ptr()), ctypes.c_void_p(u.data_ptr()),
                                          ctypes.c_void_p(relres.data_ptr()), _stream(stream)), "stfd_batch_solve")
        return u, relres

    def stats(self):
        """Per-problem solve time (us) of the last solve, chosen (threads, CTAs/SM), tuning table."""
        us = np.zeros(self.count)
        th, ct = ctypes.c_int(0), ctypes.c_int(0)
        tune = np.zeros(len(self.CANDIDATES))
        _check(self._lib.stfd_batch_stats(self.handle, _dptr(us), ctypes.byref(th), ctypes.byref(ct), _dptr(tune),
                                          len(self.CANDIDATES)), "stfd_batch_stats")
        return us, (th.value, ct.value), {"%dx%d" % c: (None if np.isnan(v) else float(v))
                                          for c, v in zip(self.CANDIDATES, tune)}

    def close(self):
        if self.handle:
            self._lib.stfd_batch_destroy(self.handle)
            self.handle = ctypes.c_void_p()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


# ---------------------------------------------------------------------------
# mapped domains (Sec. 4.6): host assembly and separation
# ---------------------------------------------------------------------------

def spatial_quadrature_points(d, p, n_el, geom, nq):
    """Physical quadrature points, shape (d, n_el^d nq^d)."""
    x = np.zeros((d, (n_el * nq) ** d))
    _check(load().stfd_spatial_quadrature_points(d, p, n_el, geom, nq, _dptr(x)), "stfd_spatial_quadrature_points")
    return x


def spatial_element_midpoints(d, n_el, geom):
    x = np.zeros((d, n_el ** d))
    _check(load().stfd_spatial_element_midpoints(d, n_el, geom, _dptr(x)), "stfd_spatial_element_midpoints")
    return x


def _opt(a, size, what):
    if a is None:
        return None, None
    a = np.ascontiguousarray(a, dtype=np.float64)
    if a.size != size:
        raise ValueError("%s must hold %d values" % (what, size))
    return a, _dptr(a)


def spatial_assemble(d, p, n_el, geom, nq, c_q=None, kappa_q=None):
    """(M_s, K_s) in the stencil layout, shape ((2p+1)^d, N_s) each."""
    Q = (n_el * nq) ** d
    c_keep, cp = _opt(c_q, Q, "c_q")
    k_keep, kp = _opt(kappa_q, Q, "kappa_q")
    Ns = (n_el + p - 2) ** d
    S = (2 * p + 1) ** d
    Ms = np.zeros((S, Ns))
    Ks = np.zeros((S, Ns))
    _check(load().stfd_spatial_assemble(d, p, n_el, geom, nq, cp, kp, _dptr(Ms), _dptr(Ks)), "stfd_spatial_assemble")
    return Ms, Ks


def spatial_element_stiffness(d, p, n_el, geom, nq):
    """Unit-conductivity element stiffness, shape (n_el^d, (p+1)^d, (p+1)^d)."""
    L = (p + 1) ** d
    Ke = np.zeros((n_el ** d, L, L))
    _check(load().stfd_spatial_element_stiffness(d, p, n_el, geom, nq, _dptr(Ke)), "stfd_spatial_element_stiffness")
    return Ke


def geo_separate(d, n_el, geom, c_mid=None, kappa_mid=None):
    """(phi, Phi), each (d, n_el): eq. separation on the element grid."""
    c_keep, cp = _opt(c_mid, n_el ** d, "c_mid")
    k_keep, kp = _opt(kappa_mid, n_el ** d, "kappa_mid")
    phi = np.zeros((d, n_el))
    Phi = np.zeros((d, n_el))
    _check(load().stfd_geo_separate(d, n_el, geom, cp, kp, _dptr(phi), _dptr(Phi)), "stfd_geo_separate")
    return phi, Phi


def spline_matrices_weighted(p, n_el, length, bc, w_mass=None, w_stiff=None):
    """(M, K) with per-element weights (eq. over_A), column-major n x n."""
    lib = load()
    n = ctypes.c_int(0)
    _check(lib.stfd_spline_matrices_weighted(p, n_el, float(length), bc, None, None, None, None, ctypes.byref(n)),
           "stfd_spline_matrices_weighted")
    wm_keep, wm = _opt(w_mass, n_el, "w_mass")
    ws_keep, ws = _opt(w_stiff, n_el, "w_stiff")
    M = np.zeros((n.value, n.value), order="F")
    K = np.zeros((n.value, n.value), order="F")
    _check(lib.stfd_spline_matrices_weighted(p, n_el, float(length), bc, wm, ws, _dptr(M), _dptr(K),
                                             ctypes.byref(n)), "stfd_spline_matrices_weighted")
    return M, K


def stencil_center(p, d):
    """Offset index of the diagonal in the stencil layout."""
    return sum(p * (2 * p + 1) ** l for l in range(d))


def _eval_coef(f, x, size):
    if f is None:
        return None
    if callable(f):
        return np.asarray(f(x), dtype=np.float64).reshape(size)
    return np.asarray(f, dtype=np.float64).reshape(size)


def mapped_problem(d, p, n_el, geom=STFD_GEOM_QUARTER_ANNULUS, c=None, kappa=None, kappa_elem=None, nq=None,
                   T=1.0):
    """Host data of the heat problem on a mapped domain (Sec. 4.6.1): stencil
    M_s, K_s, time factors, and the univariate factors of the geometry-aware
    preconditioner. c, kappa: callables of physical points x with x.shape ==
    (d, m) returning m values (None = 1); kappa_elem: per-element conductivity
    (overrides kappa)."""
    nq = p + 1 if nq is None else nq
    Q = (n_el * nq) ** d
    xq = spatial_quadrature_points(d, p, n_el, geom, nq) if (c is not None or kappa is not None) else None
    xm = spatial_element_midpoints(d, n_el, geom)
    c_q = _eval_coef(c, xq, Q) if c is not None else None
    if kappa_elem is not None:
        kappa_elem = np.asarray(kappa_elem, dtype=np.float64).reshape(n_el ** d)
        kappa_q = np.repeat(kappa_elem, nq ** d)
        kappa_mid = kappa_elem
    else:
        kappa_q = _eval_coef(kappa, xq, Q) if kappa is not None else None
        kappa_mid = _eval_coef(kappa, xm, n_el ** d) if kappa is not None else None
    c_mid = _eval_coef(c, xm, n_el ** d) if c is not None else None
    Ms, Ks = spatial_assemble(d, p, n_el, geom, nq, c_q, kappa_q)
    phi, Phi = geo_separate(d, n_el, geom, c_mid, kappa_mid)
    Kl, Ml = [], []
    for l in range(d):
        M_, K_ = spline_matrices_weighted(p, n_el, 1.0, STFD_BC_DIRICHLET, phi[l], Phi[l])
        Kl.append(K_)
        Ml.append(M_)
    Mt, _, Wt = stfd_spline_matrices(p, n_el, T, STFD_BC_INITIAL)
    ctr = stencil_center(p, d)
    n = [n_el + p - 2] * d + [Wt.shape[0]]
    return {"d": d, "p": p, "n_el": n_el, "geom": geom, "nq": nq, "n": n, "Ms": Ms, "Ks": Ks, "Wt": Wt, "Mt": Mt,
            "K_tilde": Kl, "M_tilde": Ml, "Ms_diag": Ms[ctr].copy(), "Ks_diag": Ks[ctr].copy()}


def geometry_preconditioner(prob, gamma=1.0, nu=1.0, precision=STFD_FP64, scaled=True, stream=None):
    """FD handle of A^G = D^{1/2} A~ D^{1/2} (eq. prec_geo), or of A~ alone."""
    P = FD(prob["K_tilde"], prob["M_tilde"], prob["Wt"], prob["Mt"], gamma, nu, precision=precision, stream=stream)
    if scaled:
        P.set_scaling(prob["Ms_diag"], prob["Ks_diag"], stream=stream)
    return P


# ---------------------------------------------------------------------------
# diagnostics (include/stfd_profile.h)
# ---------------------------------------------------------------------------

def stfd_profile_enable(on=True):
    _check(load().stfd_profile_enable(1 if on else 0), "stfd_profile_enable")


def stfd_profile_reset():
    _check(load().stfd_profile_reset(), "stfd_profile_reset")


def stfd_profile_records():
    """List of {name, launches, ms, flops, bytes} per kernel since the last reset."""
    lib = load()
    out = []
    for i in range(lib.stfd_profile_count()):
        name = ctypes.create_string_buffer(64)
        n = ctypes.c_longlong(0)
        ms, fl, by = ctypes.c_double(), ctypes.c_double(), ctypes.c_double()
        _check(lib.stfd_profile_get(i, name, 64, ctypes.byref(n), ctypes.byref(ms), ctypes.byref(fl),
                                    ctypes.byref(by)), "stfd_profile_get")
        out.append({"name": name.value.decode(), "launches": n.value, "ms": ms.value,
                    "flops": fl.value, "bytes": by.value})
    return out


def stfd_launch_count():
    return int(load().stfd_launch_count())


def stfd_probe_fp64_peak(stream=None):
    """Measured FP64 FMA throughput of the current device (FLOP/s)."""
    v = ctypes.c_double(0.0)
    _check(load().stfd_probe_fp64_peak(ctypes.byref(v), _stream(stream)), "stfd_probe_fp64_peak")
    return v.value


def stfd_probe_imad_wide_peak(stream=None):
    """Measured 32 x 32 -> 64-bit integer multiply-add throughput (operations/s)."""
    v = ctypes.c_double(0.0)
    _check(load().stfd_probe_imad_wide_peak(ctypes.byref(v), _stream(stream)), "stfd_probe_imad_wide_peak")
    return v.value


def heat_problem(d, p, n_el, T=1.0, lengths=None, p_t=None, n_el_t=None):
    """Univariate factors of the heat problem on a box x (0, T) from the library's own
    spline assembly: returns (K_list, M_list, W_t, M_t)."""
    lengths = [1.0] * d if lengths is None else list(lengths)
    p_t = p if p_t is None else p_t
    n_el_t = n_el if n_el_t is None else n_el_t
    K, M = [], []
    for l in range(d):
        Ml, Kl, _ = stfd_spline_matrices(p, n_el, lengths[l], STFD_BC_DIRICHLET)
        K.append(Kl)
        M.append(Ml)
    Mt, _, Wt = stfd_spline_matrices(p_t, n_el_t, T, STFD_BC_INITIAL)
    return K, M, Wt, Mt
