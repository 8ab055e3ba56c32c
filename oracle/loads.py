"""Load vectors [f]_i = F(B_i) and point evaluation of discrete solutions (Sec. 3).

Test infrastructure only (see ``oracle/__init__.py``).
"""
import itertools

import numpy as np

from . import bspline
from .assemble import reduced_index_maps
from .matrices import element_quadrature


def load_1d(p, n_el, length, func, nq, drop_first=True, drop_last=True):
    """[F]_i = int_0^length func(x) b_i(x) dx over the reduced 1D basis."""
    knots = bspline.open_uniform_knots(p, n_el, length)
    x, w = element_quadrature(knots, nq)
    V = bspline.all_basis(knots, p, x)
    F = V.T @ (w * func(x))
    lo = 1 if drop_first else 0
    hi = F.size - 1 if drop_last else F.size
    return F[lo:hi].copy()


def load_separable(space_loads, time_load):
    """F for f(x, t) = prod_l f_l(x_l) * f_t(t): F = F_t kron F_d kron .. kron F_1 (vec order)."""
    out = np.ones(1)
    for F in list(space_loads) + [time_load]:
        out = np.outer(F, out).ravel()      # new direction varies slowest
    return out


def load_quadrature(d, p_s, n_el_s, p_t, n_el_t, func, lengths=None, T=1.0, nq=None):
    """F_i = int_0^T int_Omega f B_i by direct (d+1)-D tensor Gauss quadrature.

    ``func(x_1, ..., x_d, t)`` takes broadcastable arrays.
    """
    lengths = [1.0] * d if lengths is None else list(lengths)
    nq = max(p_s, p_t) + 3 if nq is None else nq
    maps, sizes = reduced_index_maps(p_s, n_el_s, d, p_t, n_el_t)
    strides = np.cumprod([1] + sizes[:-1])
    F = np.zeros(int(np.prod(sizes)))
    dirs = [(p_s, n_el_s, lengths[l]) for l in range(d)] + [(p_t, n_el_t, T)]
    tabs = []
    for (p, ne, L) in dirs:
        knots = bspline.open_uniform_knots(p, ne, L)
        rows = []
        for k in range(len(knots) - 1):
            if knots[k + 1] <= knots[k]:
                continue
            t_, w_ = np.polynomial.legendre.leggauss(nq)
            x = 0.5 * (knots[k + 1] - knots[k]) * t_ + 0.5 * (knots[k] + knots[k + 1])
            w = 0.5 * (knots[k + 1] - knots[k]) * w_
            act = np.arange(k - p, k + 1)
            V = np.stack([bspline.basis(knots, p, i, x) for i in act], axis=-1)
            rows.append((act, x, w, V))
        tabs.append(rows)
    for elems in itertools.product(*tabs):
        grids = np.meshgrid(*[e[1] for e in elems], indexing="ij")
        wq = np.ones(1)
        for e in elems:
            wq = np.outer(wq, e[2]).ravel()
        fq = func(*grids).ravel() * wq
        # local load: contract fq over all point axes with each direction's table
        loc = fq.reshape([len(e[1]) for e in elems])
        for ax, e in enumerate(elems):
            loc = np.tensordot(loc, e[3], axes=([0], [0]))   # consume point axis, append function axis
        loc = loc.ravel()                                      # direction 0 slowest
        gidx = np.zeros(1, dtype=np.int64)
        keep = np.ones(1, dtype=bool)
        for l, e in enumerate(elems):
            red = maps[l][e[0]]
            gidx = (gidx[:, None] + np.where(red >= 0, red, 0)[None, :] * strides[l]).ravel()
            keep = (keep[:, None] & (red >= 0)[None, :]).ravel()
        np.add.at(F, gidx[keep], loc[keep])
    return F


def evaluate(coeffs, d, p_s, n_el_s, p_t, n_el_t, points, lengths=None, T=1.0):
    """u_h(x, t) = sum_i c_i B_i(x, t) at points (array of shape (P, d+1))."""
    lengths = [1.0] * d if lengths is None else list(lengths)
    maps, sizes = reduced_index_maps(p_s, n_el_s, d, p_t, n_el_t)
    C = np.reshape(coeffs, sizes, order="F")
    tables = []
    for l in range(d + 1):
        p, ne, L = (p_s, n_el_s, lengths[l]) if l < d else (p_t, n_el_t, T)
        knots = bspline.open_uniform_knots(p, ne, L)
        V = bspline.all_basis(knots, p, points[:, l])         # (P, m)
        keep = maps[l] >= 0
        tables.append(V[:, keep])
    out = np.empty(points.shape[0])
    for k in range(points.shape[0]):
        X = C
        for l in range(d + 1):
            X = np.tensordot(tables[l][k], X, axes=([0], [0]))
        out[k] = X
    return out
