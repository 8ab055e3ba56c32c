"""Pins of the oracle's B-splines and univariate matrices (CPU only).

Each test checks the oracle against a fact fixed by the paper or by the
mathematics, not against a retyped copy of its own formulas.
"""
import os

import numpy as np
import pytest

from oracle import bspline, fd, matrices

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")
rng = np.random.default_rng(1234)


@pytest.mark.parametrize("p", [1, 2, 3, 4, 5])
@pytest.mark.parametrize("n_el", [1, 3, 8])
def test_partition_of_unity_and_support(p, n_el):
    """Sec. 2.1: B-splines on an open knot vector sum to one on [0, 1], are
    non-negative and b_i vanishes outside [xi_i, xi_{i+p+1}]."""
    kn = bspline.open_uniform_knots(p, n_el)
    x = np.concatenate([rng.random(200), [0.0, 1.0], kn])
    V = bspline.all_basis(kn, p, x)
    assert V.shape[1] == n_el + p                                  # m = n_el + p
    assert np.max(np.abs(V.sum(axis=1) - 1.0)) < 1e-14
    assert V.min() >= -1e-15
    for i in range(V.shape[1]):
        outside = (x < kn[i]) | (x > kn[i + p + 1])
        assert np.all(V[outside, i] == 0.0)


@pytest.mark.parametrize("p", [1, 2, 3, 4])
def test_derivative_matches_finite_differences(p):
    """The de Boor derivative formula agrees with central differences of the
    Cox-de Boor values away from knots, and sum_i b'_i = 0."""
    n_el = 5
    kn = bspline.open_uniform_knots(p, n_el)
    x = (np.arange(n_el) + rng.uniform(0.2, 0.8, n_el)) / n_el
    h = 1e-6
    D = bspline.all_basis_deriv(kn, p, x)
    Dfd = (bspline.all_basis(kn, p, x + h) - bspline.all_basis(kn, p, x - h)) / (2 * h)
    assert np.max(np.abs(D - Dfd)) < 1e-6 * max(1.0, np.abs(D).max())
    assert np.max(np.abs(D.sum(axis=1))) < 1e-12


def test_endpoint_value():
    """Reading of the half-open spans: b_m(1) = 1 and b_1(0) = 1 (open knots)."""
    for p in [1, 2, 3]:
        kn = bspline.open_uniform_knots(p, 4)
        V = bspline.all_basis(kn, p, np.array([0.0, 1.0]))
        assert V[0, 0] == 1.0 and V[1, -1] == 1.0


@pytest.mark.parametrize("p", [1, 2, 3, 4])
@pytest.mark.parametrize("L", [1.0, 2.5])
def test_full_basis_sums(p, L):
    """Full (un-reduced) basis on [0, L]: sum_ij M_ij = L (partition of unity
    integrates to the measure), K 1 = 0, and W 1 = 0 since row i of W is
    int (sum_j b_j)' b_i. The transposed index order would give W^T 1 != 0."""
    f = matrices.univariate_matrices(p, 7, L)
    assert abs(f["M"].sum() - L) < 1e-13 * L
    assert np.max(np.abs(f["K"] @ np.ones(len(f["K"])))) < 1e-11
    assert np.max(np.abs(f["W"] @ np.ones(len(f["W"])))) < 1e-13
    assert np.max(np.abs(f["W"].T @ np.ones(len(f["W"])))) > 0.5   # b_1(0) = b_m(L) = 1
    assert np.allclose(f["M"], f["M"].T, atol=1e-15) and np.allclose(f["K"], f["K"].T, atol=1e-12)


def test_closed_form_uniform_stencils():
    """Interior rows for uniform knots. With N_q the cardinal B-spline of
    degree q, int N_p(x-i) N_p(x-j) = N_{2p+1}(p+1+j-i) and
    int N_p'(x-i) N_p'(x-j) = -N_{2p+1}''(p+1+j-i) (textbook identities):
    p=1: M = h [1, 4, 1]/6, K = [-1, 2, -1]/h, W = [-1/2, 0, 1/2];
    p=2: M = h [1, 26, 66, 26, 1]/120, K = [-1, -2, 6, -2, -1]/(6h),
         W = [-1/24, -5/12, 0, 5/12, 1/24]."""
    n_el = 12
    h = 1.0 / n_el
    f1 = matrices.univariate_matrices(1, n_el)
    np.testing.assert_allclose(f1["M"][6, 5:8], h * np.array([1, 4, 1]) / 6, rtol=1e-14)
    np.testing.assert_allclose(f1["K"][6, 5:8], np.array([-1, 2, -1]) / h, rtol=1e-13)
    np.testing.assert_allclose(f1["W"][6, 5:8], [-0.5, 0.0, 0.5], atol=1e-14)
    f2 = matrices.univariate_matrices(2, n_el)
    np.testing.assert_allclose(f2["M"][6, 4:9], h * np.array([1, 26, 66, 26, 1]) / 120, rtol=1e-13)
    np.testing.assert_allclose(f2["K"][6, 4:9], np.array([-1, -2, 6, -2, -1]) / (6 * h), rtol=1e-12)
    np.testing.assert_allclose(f2["W"][6, 4:9], [-1 / 24, -5 / 12, 0.0, 5 / 12, 1 / 24], atol=1e-14)


@pytest.mark.parametrize("p,n_el,T", [(1, 6, 1.0), (2, 9, 2.0), (3, 8, 0.5), (4, 11, 1.0)])
def test_time_skew_identity(p, n_el, T):
    """eq. integral_W: W_t + W_t^T = e_n e_n^T on the reduced time basis,
    whatever T (b_i(T) = 0 except for the last function, b_i(0) = 0 for the
    kept ones). Also M_t = T * (M_t at T = 1) and W_t independent of T (Sec. 4)."""
    Wt, Mt = matrices.time_matrices(p, n_el, T)
    E = np.zeros_like(Wt)
    E[-1, -1] = 1.0
    assert np.max(np.abs(Wt + Wt.T - E)) < 1e-13
    W1, M1 = matrices.time_matrices(p, n_el, 1.0)
    assert np.max(np.abs(Wt - W1)) < 1e-13
    assert np.max(np.abs(Mt - T * M1)) < 1e-14 * T


def _golden(name):
    rows = []
    with open(os.path.join(GOLDEN, name)) as fh:
        for line in fh:
            if line.strip() and not line.startswith("#"):
                rows.append(line.split())
    return rows


@pytest.mark.parametrize("n_el", [32, 64])
def test_table1_kappa_spatial(n_el):
    """Table 1: kappa_2(U_l) for p_s = 2..8 printed to 2 significant figures,
    and kappa_2(U_l) = sqrt(kappa_2(M_l)) (Sec. 4.1)."""
    for p, val in _golden("table1_kappa_Ul.txt"):
        K, M = matrices.space_matrices(int(p), n_el)
        U, _ = fd.spatial_factorization(K, M)
        k = np.linalg.cond(U)
        assert format(k, ".1e") == val, (p, k, val)
        assert abs(k - np.sqrt(np.linalg.cond(M))) < 1e-8 * k


def test_table3_kappa_time():
    """Table 3: kappa_2(U_t) of the arrowhead factorisation (T = 1), and the
    identity kappa_2(U_t) = sqrt(kappa_2(M_t)) of Sec. 4.2.2."""
    for n_el, p, val in _golden("table3_kappa_Ut.txt"):
        Wt, Mt = matrices.time_matrices(int(p), int(n_el))
        tf = fd.time_factorization(Wt, Mt)
        k = np.linalg.cond(tf["Ut"])
        assert format(k, ".1e") == val, (n_el, p, k, val)
        assert abs(k - np.sqrt(np.linalg.cond(Mt))) < 1e-8 * k


def test_table_cond_number_direct_time_eigendecomposition():
    """Table cond_number (Sec. 4.2.1): the condition number of the M_t-normalised
    complex eigenvectors of (W_t, M_t) from the oracle's time matrices, to the
    printed two significant figures."""
    import os
    import scipy.linalg as sl
    path = os.path.join(os.path.dirname(__file__), "golden", "table2_kappa_U_direct.txt")
    for line in open(path):
        if not line.strip() or line.startswith("#"):
            continue
        n_el, p, val = line.split()
        Wt, Mt = matrices.time_matrices(int(p), int(n_el), 1.0)
        _, U = sl.eig(Wt, Mt)
        for j in range(U.shape[1]):
            U[:, j] /= np.sqrt(np.real(np.conj(U[:, j]) @ Mt @ U[:, j]))
        assert format(np.linalg.cond(U), ".1e") == val, (n_el, p)
