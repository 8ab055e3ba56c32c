"""CPU tests of the C-ABI library: it loads, exports every declared symbol, and
its host-side logic (univariate spline matrices, loads, Step 1 factors)
agrees with the oracle. No device compute is called here."""
import ctypes
import os
import re

import numpy as np
import pytest

from oracle import fd as ofd
from oracle import loads as oloads
from oracle import matrices as omat
from paper_1909_07309_gb300 import stfd

INCLUDE = os.path.join(os.path.dirname(os.path.dirname(os.path.abspath(__file__))), "include")


def _declared_symbols():
    names = set()
    for fn in sorted(os.listdir(INCLUDE)):
        if fn.endswith(".h"):
            text = re.sub(r"/\*.*?\*/", "", open(os.path.join(INCLUDE, fn)).read(), flags=re.S)
            names |= set(re.findall(r"\b(stfd_\w+)\s*\(", text))
    return sorted(names)


def test_library_exports_every_declared_symbol():
    lib = stfd.load()
    names = _declared_symbols()
    assert len(names) >= 12
    for name in names:
        assert hasattr(lib, name), name
        assert name in stfd.SIGNATURES, name
    # and nothing the binding wraps is missing from the header
    assert set(stfd.SIGNATURES) == set(names)
    assert lib.stfd_version() >= 1
    assert lib.stfd_strerror(-1).decode() == "invalid argument"


@pytest.mark.parametrize("p,n_el,L", [(1, 1, 1.0), (1, 6, 2.0), (2, 9, 1.0), (3, 8, 0.5), (4, 11, 1.0), (5, 3, 3.0)])
@pytest.mark.parametrize("bc", [0, 1, 2])
def test_spline_matrices_match_oracle(p, n_el, L, bc):
    f = omat.univariate_matrices(p, n_el, L)
    lo = 0 if bc == 0 else 1
    hi = f["M"].shape[0] - (1 if bc == 2 else 0)
    if hi - lo < 1:
        pytest.skip("empty reduced basis")
    M, K, W = stfd.stfd_spline_matrices(p, n_el, L, bc)
    for ours, ref in [(M, f["M"]), (K, f["K"]), (W, f["W"])]:
        ref = ref[lo:hi, lo:hi]
        assert ours.shape == ref.shape
        assert np.max(np.abs(ours - ref)) <= 1e-13 * max(1.0, np.max(np.abs(ref)))


@pytest.mark.parametrize("p,n_el", [(2, 5), (3, 64)])
def test_trig_load_matches_oracle(p, n_el):
    ours = stfd.stfd_spline_load_trig(p, n_el, 1.0, 2, np.pi, 1.0, 0.0)
    ref = oloads.load_1d(p, n_el, 1.0, lambda x: np.sin(np.pi * x), 12)
    np.testing.assert_allclose(ours, ref, rtol=1e-12, atol=1e-17)
    ours_t = stfd.stfd_spline_load_trig(p, n_el, 1.0, 1, 1.0, 3 * np.pi ** 2, 1.0)
    ref_t = oloads.load_1d(p, n_el, 1.0, lambda t: 3 * np.pi ** 2 * np.sin(t) + np.cos(t), 12, True, False)
    np.testing.assert_allclose(ours_t, ref_t, rtol=1e-12, atol=1e-17)


@pytest.mark.parametrize("d,p,n_el,T", [(1, 2, 1, 1.0), (2, 1, 2, 1.0), (1, 1, 4, 1.0), (2, 2, 8, 2.0), (3, 3, 9, 1.0), (1, 4, 7, 0.5), (2, 3, 64, 1.0)])
def test_fd_factors_identities_and_oracle_spectrum(d, p, n_el, T):
    """Step 1 on the host: U^T M U = I, U^T K U = Lambda (eq. space_eig);
    U_t^T M_t U_t = I and U_t^T W_t U_t = Delta_t real arrowhead with 2 x 2
    blocks [[0, lam], [-lam, 0]] (Remark of Sec. 4.5); the spectra equal the
    oracle's (lam_j = |Im| of its complex eigenvalues)."""
    K, M, Wt, Mt = stfd.heat_problem(d, p, n_el, T=T)
    fac = stfd.stfd_fd_factors(K, M, Wt, Mt)
    for l in range(d):
        U, lam = fac["U"][l], fac["lam"][l]
        assert np.max(np.abs(U.T @ M[l] @ U - np.eye(len(lam)))) < 1e-13
        assert np.max(np.abs(U.T @ K[l] @ U - np.diag(lam))) < 1e-13 * lam.max()
        ref = ofd.spatial_factorization(K[l], M[l])[1]
        np.testing.assert_allclose(np.sort(lam), np.sort(ref), rtol=1e-12)
    Ut = fac["Ut"]
    n = Ut.shape[0]
    assert fac["n_pairs"] * 2 + fac["has_zero"] == n - 1
    assert fac["has_zero"] == (n - 1) % 2
    assert np.max(np.abs(Ut.T @ Mt @ Ut - np.eye(n))) < 1e-13
    D = Ut.T @ Wt @ Ut
    E = np.zeros_like(D)
    for j, lam in enumerate(fac["lamt"]):
        E[2 * j, 2 * j + 1] = lam
        E[2 * j + 1, 2 * j] = -lam
    E[:-1, -1] = fac["g"]
    E[-1, :-1] = -fac["g"]
    E[-1, -1] = fac["sigma"]
    assert np.max(np.abs(D - E)) < 1e-12 * np.max(np.abs(D))
    ora = ofd.time_factorization(Wt, Mt)
    im = np.sort(ora["lam"].imag)
    np.testing.assert_allclose(np.sort(fac["lamt"]), im[im > 1e-9 * im.max()], rtol=1e-11)
    assert abs(np.linalg.cond(Ut) - np.linalg.cond(ora["Ut"])) < 1e-9 * np.linalg.cond(Ut)


def test_table3_through_library():
    """Table 3 (kappa_2(U_t), T = 1) reproduced by the library's own factors."""
    for p, val in [(2, "3.2e+00"), (3, "5.2e+00"), (4, "8.3e+00")]:
        K, M, Wt, Mt = stfd.heat_problem(1, p, 32)
        assert format(np.linalg.cond(stfd.stfd_fd_factors(K, M, Wt, Mt)["Ut"]), ".1e") == val


def test_argument_errors():
    lib = stfd.load()
    n = ctypes.c_int(0)
    assert lib.stfd_spline_matrices(0, 4, 1.0, 0, None, None, None, ctypes.byref(n)) == -1
    assert lib.stfd_spline_matrices(2, 0, 1.0, 0, None, None, None, ctypes.byref(n)) == -1
    assert lib.stfd_spline_matrices(1, 1, 1.0, 2, None, None, None, ctypes.byref(n)) == -1   # n = 0 after reduction
    assert lib.stfd_spline_matrices(2, 3, -1.0, 0, None, None, None, ctypes.byref(n)) == -1
    K, M, Wt, Mt = stfd.heat_problem(1, 2, 5)
    with pytest.raises(stfd.StfdError) as e:
        stfd.stfd_fd_factors(K, [-m for m in M], Wt, Mt)
    assert e.value.code == -2          # not SPD
    with pytest.raises(stfd.StfdError) as e:
        stfd.stfd_fd_factors(K, M, Wt, -Mt)
    assert e.value.code == -2
    big = np.eye(257)
    with pytest.raises(stfd.StfdError) as e:
        stfd.stfd_fd_factors([big], [big], Wt, Mt)
    assert e.value.code == -1


def test_argument_errors_of_the_device_entry_points():
    """Invalid arguments are rejected before any CUDA call (so this runs on a
    host without a GPU): NULL handles and pointers, bad sizes and options."""
    lib = stfd.load()
    vp = ctypes.c_void_p()
    n3 = (ctypes.c_int * 3)(4, 4, 5)
    z = np.zeros(25 * 16)
    dp = stfd._dptr(z)
    # stencil op: NULL out, NULL matrices, bad half-bandwidth, bad arithmetic
    assert lib.stfd_op_create_stencil(None, 2, n3, 1, dp, dp, dp, dp, 1.0, 1.0, 1, None) == -1
    assert lib.stfd_op_create_stencil(ctypes.byref(vp), 2, n3, 1, None, dp, dp, dp, 1.0, 1.0, 1, None) == -1
    assert lib.stfd_op_create_stencil(ctypes.byref(vp), 2, n3, -1, dp, dp, dp, dp, 1.0, 1.0, 1, None) == -1
    assert lib.stfd_op_create_stencil(ctypes.byref(vp), 2, n3, 1, dp, dp, dp, dp, 1.0, 1.0, 7, None) == -1
    assert lib.stfd_op_create_stencil(ctypes.byref(vp), 4, n3, 1, dp, dp, dp, dp, 1.0, 1.0, 1, None) == -1
    assert not vp.value
    # transposed applies / matvecs and gradients on NULL handles
    assert lib.stfd_fd_apply_transpose(None, None, None, 1, None) == -1
    assert lib.stfd_st_matvec_transpose(None, None, None, 1, None) == -1
    assert lib.stfd_fd_set_scaling(None, dp, dp, None) == -1
    assert lib.stfd_grad_kappa_elements(None, 2, 4, None, None, None, None, None) == -1
    # GMRES options: transpose must be 0 or 1 (checked with NULL vectors first -> -1 either way)
    assert lib.stfd_gmres_solve(None, None, None, None, None, None, None) == -1
    # batch: empty, bad sizes, unsupported dimension
    ints = (ctypes.c_int * 2)(4, 5)
    one = (ctypes.c_int * 2)(1, 1)
    assert lib.stfd_batch_create(ctypes.byref(vp), 0, 2, ints, ints, one, 1.0, 1.0, 1.0, 0, None) == -1
    assert lib.stfd_batch_create(ctypes.byref(vp), 2, 4, ints, ints, one, 1.0, 1.0, 1.0, 0, None) == -1
    assert lib.stfd_batch_create(ctypes.byref(vp), 2, 2, ints, ints, one, -1.0, 1.0, 1.0, 0, None) == -1
    assert lib.stfd_batch_solve(None, None, None, None, None) == -1
    assert lib.stfd_batch_item(None, 0, None, None) == -1
    # mapped-domain host entry points
    assert lib.stfd_spatial_assemble(2, 2, 3, 1, 0, None, None, dp, dp) == -1          # nq = 0
    assert lib.stfd_spatial_assemble(2, 2, 3, 2, 3, None, None, dp, dp) == -1          # revolved needs d = 3
    assert lib.stfd_spatial_element_midpoints(2, 3, 9, dp) == -1
    assert lib.stfd_spline_matrices_weighted(2, 3, 1.0, 5, None, None, None, None, None) == -1
