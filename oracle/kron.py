"""m-mode products and the Kronecker form of the space-time matrix.

Test infrastructure only (see ``oracle/__init__.py``).

Dof tensors are numpy arrays of shape (n_1, ..., n_d, n_t); ``vec`` stacks
them with i_1 fastest (Fortran order), exactly the vec of Sec. 2.3.
"""
import numpy as np


def to_tensor(v, shape):
    """Inverse of vec (Sec. 2.3): index j = i_1 + sum_k (i_k - 1) prod_{l<k} n_l."""
    return np.reshape(v, shape, order="F")


def vec(X):
    return np.reshape(X, -1, order="F")


def mode_product(X, J, m):
    """[X x_m J]_{..i_m..} = sum_j X_{..j..} J_{i_m, j}   (Sec. 2.3, 0-based m)."""
    Y = np.tensordot(X, J, axes=([m], [1]))   # contracted axis removed, new axis last
    return np.moveaxis(Y, -1, m)


def kron_apply(factors, v, shape):
    """(J_{d+1} kron ... kron J_1) vec(X) = vec(X x_1 J_1 ... x_{d+1} J_{d+1}), eq. kron_vec_multi.

    ``factors`` = [J_1, ..., J_{d+1}] (time last).
    """
    X = to_tensor(v, shape)
    for m, J in enumerate(factors):
        X = mode_product(X, J, m)
    return vec(X)


def st_matvec(x, K, M, Wt, Mt, gamma=1.0, nu=1.0):
    """y = (gamma W_t kron M_s + nu M_t kron K_s) x   (eqs. syst_mat, space_univ_par_mat).

    M_s = M_d kron ... kron M_1 and K_s = sum_l M_d kron .. K_l .. kron M_1, each
    applied through eq. kron_vec_multi. ``K`` and ``M`` are lists of the d
    spatial factors (direction 1 first).
    """
    d = len(K)
    shape = tuple(k.shape[0] for k in K) + (Wt.shape[0],)
    y = gamma * kron_apply(list(M) + [Wt], x, shape)
    for l in range(d):
        facs = [K[k] if k == l else M[k] for k in range(d)] + [Mt]
        y = y + nu * kron_apply(facs, x, shape)
    return y


def st_matrix_kron(K, M, Wt, Mt, gamma=1.0, nu=1.0):
    """Sparse gamma W_t kron M_s + nu M_t kron K_s built with scipy.sparse.kron (eq. syst_mat)."""
    import scipy.sparse as sp
    d = len(K)

    def kron_chain(mats):   # mats = [J_1, ..., J_{d+1}] -> J_{d+1} kron ... kron J_1
        out = sp.csr_matrix(mats[-1])
        for J in reversed(mats[:-1]):
            out = sp.kron(out, sp.csr_matrix(J), format="csr")
        return out

    A = gamma * kron_chain(list(M) + [Wt])
    for l in range(d):
        A = A + nu * kron_chain([K[k] if k == l else M[k] for k in range(d)] + [Mt])
    return A.tocsr()
