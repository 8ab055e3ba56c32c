"""Space-time Galerkin matrices assembled directly by quadrature (Sec. 3).

Test infrastructure only (see ``oracle/__init__.py``).

For a box Omega = prod_l (0, L_l) (identity-like map, so physical and
parametric bases differ only by scaling) and a time interval (0, T), this
module integrates the bilinear form of Sec. 3.1,

    A(w, v) = int_0^T int_Omega ( gamma d_t w v + nu grad w . grad v ),

element by element with tensor Gauss rules in d+1 dimensions, and returns
[A]_{ij} = A(B_j, B_i) (eq. sys_solve) over the reduced basis of Sec. 2.2 in
colexicographic order (i_1 fastest, time slowest, eq. kron_vec_multi's vec).
It never forms a Kronecker product of matrices: the Kronecker structure of
eq. syst_mat is *checked against* this module, not used by it.

On the unit cube this also assembles the preconditioner of eq.
prec_definition, which integrates the same form on the parametric domain.
"""
import itertools

import numpy as np
import scipy.sparse as sp

from . import bspline
from .matrices import gauss_points


def _direction_tables(p, n_el, length, nq):
    """Per element: active function indices, Gauss points/weights, values, derivatives."""
    knots = bspline.open_uniform_knots(p, n_el, length)
    m = bspline.n_basis(knots, p)
    out = []
    for k in range(len(knots) - 1):
        if knots[k + 1] <= knots[k]:
            continue
        x, w = gauss_points(knots[k], knots[k + 1], nq)
        active = list(range(k - p, k + 1))      # b_{k-p..k} are the ones non-zero on span k
        V = np.stack([bspline.basis(knots, p, i, x) for i in active], axis=-1)
        D = np.stack([bspline.basis_deriv(knots, p, i, x) for i in active], axis=-1)
        out.append((np.array(active), x, w, V, D))
    return out, m


def reduced_index_maps(p_s, n_el_s, d, p_t, n_el_t):
    """Maps from full 1D function index to reduced index (-1 when removed)."""
    m_s = n_el_s + p_s
    m_t = n_el_t + p_t
    smap = np.full(m_s, -1)
    smap[1:-1] = np.arange(m_s - 2)      # Dirichlet on the spatial boundary
    tmap = np.full(m_t, -1)
    tmap[1:] = np.arange(m_t - 1)        # zero initial condition
    return [smap] * d + [tmap], [m_s - 2] * d + [m_t - 1]


def assemble_space_time(d, p_s, n_el_s, p_t, n_el_t, gamma=1.0, nu=1.0,
                        lengths=None, T=1.0, nq=None):
    """Return the sparse N x N matrix [A]_{ij} = A(B_j, B_i) by (d+1)-D quadrature."""
    lengths = [1.0] * d if lengths is None else list(lengths)
    nq_s = p_s + 1 if nq is None else nq
    nq_t = p_t + 1 if nq is None else nq
    tabs = [_direction_tables(p_s, n_el_s, lengths[l], nq_s)[0] for l in range(d)]
    tabs.append(_direction_tables(p_t, n_el_t, T, nq_t)[0])
    maps, sizes = reduced_index_maps(p_s, n_el_s, d, p_t, n_el_t)
    strides = np.cumprod([1] + sizes[:-1])
    N = int(np.prod(sizes))
    rows, cols, vals = [], [], []
    for elems in itertools.product(*tabs):
        # elems[l] = (active, x, w, V, D) for direction l (time last).
        # Values of the tensor-product basis at the tensor Gauss points
        # (eq. tens-prod-space-parametric): outer products of 1D tables.
        Vs = [e[3] for e in elems]
        Ds = [e[4] for e in elems]
        ws = [e[2] for e in elems]
        nd = d + 1

        def tensor_table(factors):
            # T[(q_0..q_d), (i_0..i_d)] = prod_l f_l[q_l, i_l], direction 0 slowest.
            T_ = factors[0]
            for f in factors[1:]:
                T_ = np.einsum("ab,cd->acbd", T_, f).reshape(T_.shape[0] * f.shape[0],
                                                             T_.shape[1] * f.shape[1])
            return T_

        # Inside the local tables direction 0 varies slowest; the global index
        # map below uses the same nesting and colexicographic strides.
        val = tensor_table(Vs)                                   # B_i at points
        dt = tensor_table(Vs[:-1] + [Ds[-1]])                    # d_t B_i
        grads = [tensor_table([Ds[l] if k == l else Vs[k] for k in range(nd)]) for l in range(d)]
        wq = ws[0]
        for w_ in ws[1:]:
            wq = np.outer(wq, w_).ravel()
        # Local matrix  Loc[i, j] = A(B_j, B_i)
        loc = gamma * (val.T @ (wq[:, None] * dt))
        for g in grads:
            loc += nu * (g.T @ (wq[:, None] * g))
        # Global reduced indices of the local functions (same nesting as tensor_table).
        gidx = np.zeros(1, dtype=np.int64)
        keep = np.ones(1, dtype=bool)
        for l in range(nd):
            act = elems[l][0]
            red = maps[l][act]
            gidx = (gidx[:, None] + np.where(red >= 0, red, 0)[None, :] * strides[l]).ravel()
            keep = (keep[:, None] & (red >= 0)[None, :]).ravel()
        li = np.nonzero(keep)[0]
        gi = gidx[li]
        sub = loc[np.ix_(li, li)]
        rows.append(np.repeat(gi, len(gi)))
        cols.append(np.tile(gi, len(gi)))
        vals.append(sub.ravel())
    A = sp.coo_matrix((np.concatenate(vals), (np.concatenate(rows), np.concatenate(cols))), shape=(N, N))
    return A.tocsr()
