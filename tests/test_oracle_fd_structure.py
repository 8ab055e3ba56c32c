"""Pins of the oracle's space-time structure and of Algorithm 1 (CPU only)."""
import numpy as np
import pytest
import scipy.sparse.linalg as spla

from oracle import assemble, direct, fd, kron, matrices
from paper_1909_07309_gb300 import inputs

rng = np.random.default_rng(99)


def _factors(d, p, n_el, lengths, T, p_t=None, n_el_t=None):
    p_t = p if p_t is None else p_t
    n_el_t = n_el if n_el_t is None else n_el_t
    sm = [matrices.space_matrices(p, n_el, L) for L in lengths[:d]]
    Wt, Mt = matrices.time_matrices(p_t, n_el_t, T)
    return [k for k, _ in sm], [m for _, m in sm], Wt, Mt


CASES = [  # d, p, n_el, lengths, T, gamma, nu   (n_t - 1 = n_el + p - 2: both parities)
    (1, 1, 5, [1.0], 1.0, 1.0, 1.0),
    (1, 3, 4, [2.0], 1.5, 0.7, 2.0),
    (2, 2, 3, [1.0, 1.0], 1.0, 1.0, 1.0),
    (2, 2, 4, [1.0, 2.0], 0.5, 1.3, 0.4),
    (2, 3, 3, [0.5, 1.0], 2.0, 2.0, 1.0),
    (2, 4, 2, [1.0, 1.0], 1.0, 1.0, 3.0),
    (3, 2, 2, [1.0, 1.0, 1.0], 1.0, 1.0, 1.0),
    (3, 1, 3, [1.0, 0.5, 2.0], 1.2, 0.9, 1.1),
]


@pytest.mark.parametrize("d,p,n_el,lengths,T,gamma,nu", CASES)
def test_assembled_equals_kronecker(d, p, n_el, lengths, T, gamma, nu):
    """eq. syst_mat: the matrix assembled by (d+1)-D quadrature of the
    bilinear form equals gamma W_t kron M_s + nu M_t kron K_s, and the
    oracle's mode-product matvec (eq. kron_vec_multi) equals A x."""
    A = assemble.assemble_space_time(d, p, n_el, p, n_el, gamma, nu, lengths=lengths, T=T)
    K, M, Wt, Mt = _factors(d, p, n_el, lengths, T)
    Ak = kron.st_matrix_kron(K, M, Wt, Mt, gamma, nu)
    assert abs(A - Ak).max() <= 1e-14 * abs(A).max()
    x = rng.standard_normal(A.shape[0])
    y = kron.st_matvec(x, K, M, Wt, Mt, gamma, nu)
    assert np.max(np.abs(A @ x - y)) <= 1e-13 * np.max(np.abs(y))


def test_mixed_degrees_assembly():
    """Different degree / mesh in time than in space (p_t != p_s, n_el_t != n_el_s)."""
    d, p, n_el, p_t, n_el_t = 2, 2, 3, 3, 5
    A = assemble.assemble_space_time(d, p, n_el, p_t, n_el_t, 1.0, 1.0)
    K, M, Wt, Mt = _factors(d, p, n_el, [1.0, 1.0], 1.0, p_t, n_el_t)
    Ak = kron.st_matrix_kron(K, M, Wt, Mt)
    assert abs(A - Ak).max() <= 1e-14 * abs(A).max()


@pytest.mark.parametrize("d,p,n_el,T,gamma,nu", [(1, 2, 5, 1.0, 1.0, 1.0), (1, 3, 6, 2.0, 0.7, 1.3),
                                                   (2, 2, 3, 1.0, 1.0, 1.0), (2, 1, 4, 0.5, 2.0, 0.5),
                                                   (2, 3, 3, 1.0, 1.0, 1.0), (3, 1, 3, 1.0, 1.0, 1.0)])
def test_banded_lu_agrees_with_superlu(d, p, n_el, T, gamma, nu):
    """The oracle's own banded Gaussian elimination with partial pivoting and
    the library routine (SuperLU) solve the directly assembled A (and A^T)
    alike; in vec order A's bandwidth is p (1 + n_s + ... + n_s^d) on both
    sides of the diagonal (supports of p + 1 spans in every direction)."""
    A = assemble.assemble_space_time(d, p, n_el, p, n_el, gamma, nu, T=T)
    n_s = n_el + p - 2
    assert direct.bandwidths(A) == (p * sum(n_s ** l for l in range(d + 1)),) * 2
    for M_ in (A, A.T.tocsr()):
        r = rng.standard_normal(M_.shape[0])
        x = direct.banded_solve(direct.banded_lu(M_), r)
        x_ref = spla.spsolve(M_.tocsc(), r)
        assert np.linalg.norm(x - x_ref) <= 1e-12 * np.linalg.norm(x_ref)
        assert np.linalg.norm(M_ @ x - r) <= 1e-13 * np.linalg.norm(r)


@pytest.mark.parametrize("n,kl,ku", [(50, 3, 5), (60, 10, 10), (200, 4, 4), (40, 0, 6), (40, 6, 0)])
def test_banded_lu_pivots_on_random_band_matrices(n, kl, ku):
    """The space-time matrices happen not to need row interchanges, so the
    pivoting path is pinned on random band matrices with a small diagonal
    (interchanges at most steps): same solution as LAPACK's dense solve."""
    import scipy.sparse as sp
    g = np.random.default_rng(n + 7 * kl + 13 * ku)
    D = np.zeros((n, n))
    for i in range(n):
        for j in range(max(0, i - kl), min(n, i + ku + 1)):
            D[i, j] = g.standard_normal()
    D[np.arange(n), np.arange(n)] = 0.05 * D[np.arange(n), np.arange(n)] + (kl == 0 or ku == 0)
    b = g.standard_normal(n)
    fac = direct.banded_lu(sp.csr_matrix(D))
    assert direct.bandwidths(sp.csr_matrix(D)) == (kl, ku)
    if kl > 0:
        assert np.count_nonzero(fac[1] != np.arange(n)) > n // 4
    x = direct.banded_solve(fac, b)
    ref = np.linalg.solve(D, b)
    assert np.linalg.norm(x - ref) <= 1e-11 * np.linalg.norm(ref)


@pytest.mark.parametrize("d,p,n_el,lengths,T,gamma,nu", CASES)
def test_fd_equals_direct_solve(d, p, n_el, lengths, T, gamma, nu):
    """Algorithm 1 reproduces P^{-1} r: compared with a sparse direct solve
    (SuperLU) of the directly assembled matrix on the unit cube, where P = A."""
    K, M, Wt, Mt = _factors(d, p, n_el, [1.0] * d, T)
    P = assemble.assemble_space_time(d, p, n_el, p, n_el, gamma, nu, T=T)
    r = rng.standard_normal(P.shape[0])
    s_ref = spla.spsolve(P.tocsc(), r)
    fac = fd.setup(K, M, Wt, Mt)
    s, imag = fd.apply(fac, r, gamma, nu)
    assert imag < 1e-12 * np.max(np.abs(s))
    assert np.linalg.norm(s - s_ref) <= 1e-12 * np.linalg.norm(s_ref)


def test_fd_d1_equals_dense_solve():
    """d = 1: P is a dense n_s n_t system solved by numpy.linalg.solve."""
    K, M, Wt, Mt = _factors(1, 3, 6, [1.0], 1.0)
    P = 1.5 * np.kron(Wt, M[0]) + 0.8 * np.kron(Mt, K[0])
    r = rng.standard_normal(P.shape[0])
    s = fd.fd_solve(K, M, Wt, Mt, r, 1.5, 0.8)
    np.testing.assert_allclose(s, np.linalg.solve(P, r), rtol=1e-11, atol=1e-13)


def test_fd_small_workload_direct():
    """The small workload (d=2, p=2, 16 elements, gamma = nu = 1, T = 1):
    Algorithm 1 on f = (M_t kron M_s) c, c ~ N(0,1), equals SuperLU on P."""
    K, M, Wt, Mt = _factors(2, 2, 16, [1.0, 1.0], 1.0)
    P = kron.st_matrix_kron(K, M, Wt, Mt)
    c = inputs.standard_normal(P.shape[0], inputs.SMALL["rhs_seed"])
    f = kron.st_matvec(c, [m for m in M], M, Mt, Mt, 1.0, 0.0)    # (M_t kron M_s) c
    s = fd.fd_solve(K, M, Wt, Mt, f)
    s_ref = spla.spsolve(P.tocsc(), f)
    assert np.linalg.norm(s - s_ref) <= 1e-12 * np.linalg.norm(s_ref)


@pytest.mark.parametrize("p,n_el", [(1, 6), (2, 7), (3, 8), (4, 9), (3, 9)])
def test_setup_identities(p, n_el):
    """eq. space_eig: U^T K U = Lambda, U^T M U = I. eqs. time_eig, time_eig_2:
    U_t^* M_t U_t = I and U_t^* W_t U_t = Delta_t is arrowhead with last row
    -g^*, leading block purely imaginary (skew pencil), sigma = rho^2 / 2
    (from eq. integral_W: sigma = [r; rho]^T W_t [r; rho] = rho^2 b_n(T)^2 / 2)."""
    K, M = matrices.space_matrices(p, n_el)
    U, lam = fd.spatial_factorization(K, M)
    assert np.max(np.abs(U.T @ M @ U - np.eye(len(lam)))) < 1e-13
    assert np.max(np.abs(U.T @ K @ U - np.diag(lam))) < 1e-12 * lam.max()
    assert lam.min() > 0
    Wt, Mt = matrices.time_matrices(p, n_el, 1.0)
    tf = fd.time_factorization(Wt, Mt)
    Ut = tf["Ut"]
    n = Ut.shape[0]
    assert np.max(np.abs(Ut.conj().T @ Mt @ Ut - np.eye(n))) < 1e-13
    D = Ut.conj().T @ Wt @ Ut
    mask = np.eye(n, dtype=bool)
    mask[-1, :] = True
    mask[:, -1] = True
    assert np.max(np.abs(D[~mask])) < 1e-13 * np.max(np.abs(D))
    assert np.max(np.abs(D - tf["Delta"])) < 1e-12 * np.max(np.abs(D))
    assert np.max(np.abs(D[-1, :-1] + D[:-1, -1].conj())) < 1e-12 * np.max(np.abs(D))
    assert np.max(np.abs(tf["lam"].real)) < 1e-12 * np.max(np.abs(tf["lam"]))
    assert abs(tf["sigma"] - tf["rho"] ** 2 / 2) < 1e-12 * abs(tf["sigma"])
    # eigenvalues come in conjugate pairs plus a zero when n_t - 1 is odd (Sec. 4.2.2)
    im = np.sort(tf["lam"].imag)
    np.testing.assert_allclose(im, -im[::-1], atol=1e-12 * np.abs(im).max())
    if (n - 1) % 2 == 1:
        assert np.min(np.abs(im)) < 1e-10 * np.abs(im).max()
    # a square M-orthonormal U has U U^T = M^{-1}: its singular values are the
    # inverse square roots of M's eigenvalues, so kappa_2(U) = sqrt(kappa_2(M))
    # (the quantity Tables 1 and 3 report for the spatial and time factors)
    np.testing.assert_allclose(np.linalg.cond(U), np.sqrt(np.linalg.cond(M)), rtol=1e-9)
    np.testing.assert_allclose(np.linalg.cond(Ut), np.sqrt(np.linalg.cond(Mt)), rtol=1e-9)
