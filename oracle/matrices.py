"""Univariate spline matrices by element-wise Gauss-Legendre quadrature.

Test infrastructure only (see ``oracle/__init__.py``).

* Time (eq. time_mat, Sec. 3.3):   [W_t]_{ij} = int_0^T b'_j b_i dt,  [M_t]_{ij} = int_0^T b_i b_j dt.
* Space (Sec. 4, univariate factors of eq. space_univ_par_mat):
  [K_l]_{ij} = int b'_i b'_j,  [M_l]_{ij} = int b_i b_j.
* Initial/boundary reduction (Sec. 2.2): space keeps b_2..b_{m-1}
  (n_s = m - 2), time keeps b_2..b_m (n_t = m - 1).
"""
import numpy as np

from . import bspline


def gauss_points(a, b, nq):
    """nq-point Gauss-Legendre rule mapped to [a, b] (numpy's leggauss)."""
    t, w = np.polynomial.legendre.leggauss(nq)
    return 0.5 * (b - a) * t + 0.5 * (a + b), 0.5 * (b - a) * w


def element_quadrature(knots, nq):
    """Concatenated quadrature points/weights over all non-empty knot spans."""
    xs, ws = [], []
    for k in range(len(knots) - 1):
        if knots[k + 1] > knots[k]:
            x, w = gauss_points(knots[k], knots[k + 1], nq)
            xs.append(x)
            ws.append(w)
    return np.concatenate(xs), np.concatenate(ws)


def univariate_matrices(p, n_el, length=1.0, nq=None):
    """Full (un-reduced) m x m matrices M, K, W on [0, length].

    With nq = p + 1 points per element the rule is exact for the polynomial
    integrands of degree <= 2p here.
    """
    knots = bspline.open_uniform_knots(p, n_el, length)
    nq = p + 1 if nq is None else nq
    x, w = element_quadrature(knots, nq)
    V = bspline.all_basis(knots, p, x)          # V[q, i] = b_i(x_q)
    D = bspline.all_basis_deriv(knots, p, x)    # D[q, i] = b'_i(x_q)
    M = V.T @ (w[:, None] * V)                  # int b_i b_j
    K = D.T @ (w[:, None] * D)                  # int b'_i b'_j
    W = V.T @ (w[:, None] * D)                  # W[i, j] = int b'_j b_i  (index order of eq. time_mat)
    return {"M": M, "K": K, "W": W, "knots": knots}


def space_matrices(p, n_el, length=1.0):
    """Reduced spatial factors (K_l, M_l): drop the first and last function."""
    f = univariate_matrices(p, n_el, length)
    return f["K"][1:-1, 1:-1].copy(), f["M"][1:-1, 1:-1].copy()


def time_matrices(p, n_el, T=1.0):
    """Reduced time factors (W_t, M_t) on [0, T]: drop the first function."""
    f = univariate_matrices(p, n_el, T)
    return f["W"][1:, 1:].copy(), f["M"][1:, 1:].copy()
