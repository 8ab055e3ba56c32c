"""Mapped-domain spatial matrices with variable coefficients, the
geometry-aware preconditioner and the adjoint gradient.

Test infrastructure only (see ``oracle/__init__.py``).

* Spatial matrices (Sec. 4.6, the parametric form of [A]_{ij}; Sec. 4.6.1 with
  gamma_s = c, nu_s = kappa):
      [M_s]_{ij} = int_Omega^ c(F) B^_i B^_j |det J|,
      [K_s]_{ij} = int_Omega^ kappa(F) grad^B^_i . J^{-1} J^{-T} grad^B^_j |det J|,
  by tensor Gauss quadrature on every parametric element, then the Dirichlet
  reduction of Sec. 2.2 (first and last function dropped in every direction).
  J^{-1} and det J are taken by numpy's general routines at each point.
* The space-time matrix A = gamma W_t (x) M_s + nu M_t (x) K_s (Sec. 4.6.1:
  the coefficients do not depend on time, so the time factors are exact).
* Geometry-aware preconditioner (Sec. 4.6, eqs. separation, over_A,
  prec_geo): the diagonal of the coefficient matrix frak{C} (with kappa in the
  spatial block and c in the last entry) is interpolated by its value at the
  element midpoint; its separation is the least-squares fit in log space, with
  the univariate factors given by marginal means (our reading: the paper
  cites another paper's appendix for this algorithm); weighted univariate
  matrices; D = diag(A) / diag(A~).
* Adjoint gradient of L(u) = 1/2 (u - u_obs)^T (M_t (x) M_s) (u - u_obs) with
  A u = f (not in the paper): lambda = A^{-T} dL/du, dL/df = lambda and
  dL/dkappa_e = -nu lambda^T (M_t (x) K_e) u for the element stiffness K_e of
  unit conductivity.

Elements and dofs are numbered colexicographically (direction 1 fastest).
"""
import itertools

import numpy as np
import scipy.sparse as sp
import scipy.sparse.linalg as spla

from . import bspline, geometry
from .matrices import gauss_points


def _tables(p, n_el, nq):
    """Per parametric element of (0, 1): (active full indices, points, weights, values, derivatives)."""
    knots = bspline.open_uniform_knots(p, n_el, 1.0)
    out = []
    for k in range(len(knots) - 1):
        if knots[k + 1] <= knots[k]:
            continue
        x, w = gauss_points(knots[k], knots[k + 1], nq)
        act = np.arange(k - p, k + 1)
        V = np.stack([bspline.basis(knots, p, i, x) for i in act], axis=-1)
        D = np.stack([bspline.basis_deriv(knots, p, i, x) for i in act], axis=-1)
        out.append((act, x, w, V, D))
    return out


def element_ids(d, n_el):
    """Element multi-indices (e_1, .., e_d) in colexicographic order."""
    return [tuple(reversed(e)) for e in itertools.product(range(n_el), repeat=d)]


def _element_data(d, p, n_el, nq, geom, e, tabs):
    """Points, weights, basis values and parametric gradients on element e.

    Local functions and points are numbered colexicographically too."""
    ts = [tabs[e[l]] for l in range(d)]
    # points: q = q_1 + nq q_2 + ...
    grids = np.meshgrid(*[t[1] for t in ts], indexing="ij")          # axis l = direction l
    eta = np.stack([g.transpose(tuple(reversed(range(d)))).ravel() for g in grids], axis=-1)
    wq = np.ones(1)
    for t in ts:
        wq = np.outer(t[2], wq).ravel()                                # direction 1 fastest
    def table(facs):
        T = np.ones((1, 1))
        for f in facs:
            T = np.einsum("qa,rb->rqba", T, f).reshape(T.shape[0] * f.shape[0], T.shape[1] * f.shape[1])
        return T
    V = table([t[3] for t in ts])
    G = np.stack([table([ts[k][4] if k == l else ts[k][3] for k in range(d)]) for l in range(d)], axis=-1)
    act = [t[0] for t in ts]
    x, J = geometry.MAPS[geom](eta)
    return eta, wq, V, G, act, x, J


def _global_reduced(d, p, n_el, act):
    """Reduced global index (or -1) of each local function."""
    n_s = n_el + p - 2
    idx = np.zeros(1, dtype=np.int64)
    keep = np.ones(1, dtype=bool)
    stride = 1
    for l in range(d):
        red = act[l] - 1
        ok = (red >= 0) & (red < n_s)
        idx = (np.where(ok, red, 0)[:, None] * stride + idx[None, :]).ravel()
        keep = (ok[:, None] & keep[None, :]).ravel()
        stride *= n_s
    return np.where(keep, idx, -1)


def spatial_matrices(d, p, n_el, geom="quarter_annulus", c=None, kappa=None, kappa_elem=None, nq=None,
                     element_stiffness=False):
    """Reduced sparse (M_s, K_s); c, kappa: callables of physical points x[..., d]
    (None = 1); kappa_elem: per-element conductivity (overrides kappa).
    With element_stiffness=True also returns [(global reduced indices, K_e)] for
    unit conductivity, one entry per element in colexicographic order."""
    nq = p + 1 if nq is None else nq
    tabs = _tables(p, n_el, nq)
    n_s = n_el + p - 2
    Ns = n_s ** d
    rows, cols, mv, kv = [], [], [], []
    elems = []
    for eid, e in enumerate(element_ids(d, n_el)):
        eta, wq, V, G, act, x, J = _element_data(d, p, n_el, nq, geom, e, tabs)
        detJ = np.linalg.det(J)
        Jinv = np.linalg.inv(J)
        Cmat = np.abs(detJ)[:, None, None] * np.einsum("qab,qcb->qac", Jinv, Jinv)   # J^{-1} J^{-T} |det J|
        cval = np.ones(len(wq)) if c is None else c(x)
        if kappa_elem is not None:
            kval = np.full(len(wq), float(kappa_elem[eid]))
        else:
            kval = np.ones(len(wq)) if kappa is None else kappa(x)
        Mloc = V.T @ ((wq * cval * np.abs(detJ))[:, None] * V)
        K0 = np.einsum("q,qia,qab,qjb->ij", wq, G, Cmat, G)
        Kloc = np.einsum("q,qia,qab,qjb->ij", wq * kval, G, Cmat, G)
        g = _global_reduced(d, p, n_el, act)
        li = np.nonzero(g >= 0)[0]
        gi = g[li]
        rows.append(np.repeat(gi, len(gi)))
        cols.append(np.tile(gi, len(gi)))
        mv.append(Mloc[np.ix_(li, li)].ravel())
        kv.append(Kloc[np.ix_(li, li)].ravel())
        if element_stiffness:
            elems.append((gi, K0[np.ix_(li, li)]))
    r, cc = np.concatenate(rows), np.concatenate(cols)
    Ms = sp.coo_matrix((np.concatenate(mv), (r, cc)), shape=(Ns, Ns)).tocsr()
    Ks = sp.coo_matrix((np.concatenate(kv), (r, cc)), shape=(Ns, Ns)).tocsr()
    if element_stiffness:
        return Ms, Ks, elems
    return Ms, Ks


def spatial_rows(d, p, n_el, rows, geom="quarter_annulus", c=None, kappa=None, nq=None):
    """Rows of the reduced M_s and K_s for the given reduced row indices, each
    by quadrature over the (at most (p+1)^d) elements in the row's support:
    returns {row: (columns, M values, K values)}. For sizes where the whole
    matrix is too large to assemble here."""
    nq = p + 1 if nq is None else nq
    tabs = _tables(p, n_el, nq)
    n_s = n_el + p - 2
    out = {}
    for row in rows:
        idx = [(row // n_s ** l) % n_s for l in range(d)]
        full = [i + 1 for i in idx]                      # full 1D index (the first function was dropped)
        ranges = [range(max(0, f - p), min(n_el, f + 1)) for f in full]   # elements where b_f is non-zero
        acc_m, acc_k = {}, {}
        for e_rev in itertools.product(*reversed(ranges)):
            e = tuple(reversed(e_rev))
            eta, wq, V, G, act, x, J = _element_data(d, p, n_el, nq, geom, e, tabs)
            detJ = np.linalg.det(J)
            Jinv = np.linalg.inv(J)
            Cmat = np.abs(detJ)[:, None, None] * np.einsum("qab,qcb->qac", Jinv, Jinv)
            cval = np.ones(len(wq)) if c is None else c(x)
            kval = np.ones(len(wq)) if kappa is None else kappa(x)
            # local index of the row's function in this element (colexicographic)
            a_loc = sum((full[l] - e[l]) * (p + 1) ** l for l in range(d))
            g = _global_reduced(d, p, n_el, act)
            mrow = V[:, a_loc] @ ((wq * cval * np.abs(detJ))[:, None] * V)
            krow = np.einsum("q,qa,qab,qjb->j", wq * kval, G[:, a_loc, :], Cmat, G)
            for j, gj in enumerate(g):
                if gj >= 0:
                    acc_m[gj] = acc_m.get(gj, 0.0) + mrow[j]
                    acc_k[gj] = acc_k.get(gj, 0.0) + krow[j]
        cols = np.array(sorted(acc_m))
        out[row] = (cols, np.array([acc_m[j] for j in cols]), np.array([acc_k[j] for j in cols]))
    return out


def full_spatial_matrices(d, p, n_el, geom="quarter_annulus", nq=None):
    """Unreduced (M, K) over all (n_el + p)^d functions, unit coefficients (for pins)."""
    nq = p + 1 if nq is None else nq
    tabs = _tables(p, n_el, nq)
    m = n_el + p
    M = np.zeros((m ** d, m ** d))
    K = np.zeros((m ** d, m ** d))
    for e in element_ids(d, n_el):
        eta, wq, V, G, act, x, J = _element_data(d, p, n_el, nq, geom, e, tabs)
        detJ = np.linalg.det(J)
        Jinv = np.linalg.inv(J)
        Cmat = np.abs(detJ)[:, None, None] * np.einsum("qab,qcb->qac", Jinv, Jinv)
        g = np.zeros(1, dtype=np.int64)
        for l in range(d):
            g = (act[l][:, None] * m ** l + g[None, :]).ravel()
        M[np.ix_(g, g)] += V.T @ ((wq * np.abs(detJ))[:, None] * V)
        K[np.ix_(g, g)] += np.einsum("q,qia,qab,qjb->ij", wq, G, Cmat, G)
    return M, K


def space_time(Ms, Ks, Wt, Mt, gamma=1.0, nu=1.0):
    """A = gamma W_t (x) M_s + nu M_t (x) K_s (time slowest in vec order)."""
    return (gamma * sp.kron(sp.csr_matrix(Wt), Ms) + nu * sp.kron(sp.csr_matrix(Mt), Ks)).tocsr()


def load(d, p, n_el, p_t, n_el_t, f, geom="quarter_annulus", T=1.0, nq=None):
    """[F]_i = int_0^T int_Omega f(x, t) B_i |det J| over the reduced space-time basis."""
    nq = p + 3 if nq is None else nq
    tabs = _tables(p, n_el, nq)
    knots_t = bspline.open_uniform_knots(p_t, n_el_t, T)
    n_s, n_t = n_el + p - 2, n_el_t + p_t - 1
    F = np.zeros(n_s ** d * n_t)
    t_tabs = []
    for k in range(len(knots_t) - 1):
        if knots_t[k + 1] > knots_t[k]:
            tq, tw = gauss_points(knots_t[k], knots_t[k + 1], nq)
            act = np.arange(k - p_t, k + 1)
            Vt = np.stack([bspline.basis(knots_t, p_t, i, tq) for i in act], axis=-1)
            t_tabs.append((act, tq, tw, Vt))
    for e in element_ids(d, n_el):
        eta, wq, V, G, act, x, J = _element_data(d, p, n_el, nq, geom, e, tabs)
        wdet = wq * np.abs(np.linalg.det(J))
        g = _global_reduced(d, p, n_el, act)
        for (act_t, tq, tw, Vt) in t_tabs:
            fx = f(x[:, None, :], tq[None, :])                       # (points, time points)
            loc = V.T @ ((wdet[:, None] * fx) * tw[None, :]) @ Vt      # (local space, local time)
            for a, it in enumerate(act_t):
                if it == 0:
                    continue                                           # zero initial condition
                ok = g >= 0
                np.add.at(F, (it - 1) * n_s ** d + g[ok], loc[ok, a])
    return F


def l2_error(u, d, p, n_el, p_t, n_el_t, exact, geom="quarter_annulus", T=1.0, nq=None):
    """|| u_h - exact ||_{L2(Omega x (0,T))} by quadrature."""
    nq = p + 3 if nq is None else nq
    tabs = _tables(p, n_el, nq)
    knots_t = bspline.open_uniform_knots(p_t, n_el_t, T)
    n_s = n_el + p - 2
    U = u.reshape(-1, n_s ** d)                                         # [time][space]
    err2 = 0.0
    for e in element_ids(d, n_el):
        eta, wq, V, G, act, x, J = _element_data(d, p, n_el, nq, geom, e, tabs)
        wdet = wq * np.abs(np.linalg.det(J))
        g = _global_reduced(d, p, n_el, act)
        Vr = V[:, g >= 0]
        gi = g[g >= 0]
        for k in range(len(knots_t) - 1):
            if knots_t[k + 1] <= knots_t[k]:
                continue
            tq, tw = gauss_points(knots_t[k], knots_t[k + 1], nq)
            act_t = np.arange(k - p_t, k + 1)
            Vt = np.stack([bspline.basis(knots_t, p_t, i, tq) for i in act_t], axis=-1)
            uh = np.zeros((len(wq), len(tq)))
            for a, it in enumerate(act_t):
                if it >= 1:
                    uh += np.outer(Vr @ U[it - 1, gi], Vt[:, a])
            diff = uh - exact(x[:, None, :], tq[None, :])
            err2 += float(wdet @ (diff ** 2) @ tw)
    return np.sqrt(err2)


# ---------------------------------------------------------------------------
# Geometry-aware preconditioner (Sec. 4.6)
# ---------------------------------------------------------------------------

def coefficient_diagonal(d, n_el, geom="quarter_annulus", c=None, kappa=None, kappa_elem=None):
    """Per element (colexicographic), the diagonal of frak{C} at the element
    midpoint: rows l < d: kappa |det J| [J^{-1} J^{-T}]_{ll}; row d: c |det J|."""
    ids = element_ids(d, n_el)
    eta = (np.array(ids, dtype=np.float64) + 0.5) / n_el          # (n_elem, d)
    x, J = geometry.MAPS[geom](eta)
    det = np.abs(np.linalg.det(J))
    Jinv = np.linalg.inv(J)
    Cm = det[:, None, None] * np.einsum("eab,ecb->eac", Jinv, Jinv)
    if kappa_elem is not None:
        kv = np.asarray(kappa_elem, dtype=np.float64)
    else:
        kv = np.ones(len(ids)) if kappa is None else kappa(x)
    cv = np.ones(len(ids)) if c is None else c(x)
    out = np.zeros((d + 1, len(ids)))
    for l in range(d):
        out[l] = kv * Cm[:, l, l]
    out[d] = cv * det
    return out


def separate(Cdiag, d, n_el):
    """Univariate factors (phi, Phi), each (d, n_el), of eq. separation:
    C_{d+1} ~ prod_l phi_l(e_l) and C_l ~ Phi_l(e_l) prod_{m != l} phi_m(e_m),
    least squares in log space on the element grid (marginal means)."""
    shape = (n_el,) * d
    def grid(v):   # colexicographic vector -> array indexed [e_1, .., e_d]
        return np.reshape(v, shape, order="F")
    logm = np.log(grid(Cdiag[d]))
    mean = logm.mean()
    logphi = []
    for l in range(d):
        axes = tuple(k for k in range(d) if k != l)
        logphi.append(logm.mean(axis=axes) - (d - 1) / d * mean)
    phi = np.exp(np.array(logphi))
    Phi = np.zeros((d, n_el))
    for l in range(d):
        rest = np.zeros(shape)
        for m in range(d):
            if m != l:
                sh = [1] * d
                sh[m] = n_el
                rest = rest + np.reshape(logphi[m], sh)
        axes = tuple(k for k in range(d) if k != l)
        Phi[l] = np.exp((np.log(grid(Cdiag[l])) - rest).mean(axis=axes))
    return phi, Phi


def weighted_matrices(p, n_el, w_mass, w_stiff):
    """Reduced M~_l = int phi_l b_i b_j, K~_l = int Phi_l b'_i b'_j with
    piecewise-constant weights per element (exact with p + 1 Gauss points)."""
    tabs = _tables(p, n_el, p + 1)
    m = n_el + p
    M = np.zeros((m, m))
    K = np.zeros((m, m))
    for e, (act, x, w, V, D) in enumerate(tabs):
        M[np.ix_(act, act)] += w_mass[e] * (V.T @ (w[:, None] * V))
        K[np.ix_(act, act)] += w_stiff[e] * (D.T @ (w[:, None] * D))
    return K[1:-1, 1:-1].copy(), M[1:-1, 1:-1].copy()


def kron_spatial(Kl, Ml):
    """M~_s = M_d (x) .. (x) M_1 and K~_s = sum_l M_d .. K_l .. M_1 as sparse matrices."""
    d = len(Kl)
    def chain(mats):
        out = sp.csr_matrix(mats[-1])
        for J in reversed(mats[:-1]):
            out = sp.kron(out, sp.csr_matrix(J), format="csr")
        return out
    Ms = chain(list(Ml))
    Ks = sum(chain([Kl[k] if k == l else Ml[k] for k in range(d)]) for l in range(d))
    return Ks.tocsr(), Ms.tocsr()


def diag_scaling(A, Atil):
    """D = diag(A) / diag(A~) (eq. prec_geo)."""
    return A.diagonal() / Atil.diagonal()


# ---------------------------------------------------------------------------
# Adjoint gradient
# ---------------------------------------------------------------------------

def geometry_preconditioner(A, d, p, n_el, Wt, Mt, geom="quarter_annulus", c=None, kappa=None, kappa_elem=None,
                            transpose=False):
    """v -> (A^G)^{-1} v (or (A^G)^{-T} v) with A^G = D^{1/2} A~ D^{1/2} (eq. prec_geo),
    A~^{-1} by the oracle's Algorithm 1 on the weighted univariate factors."""
    from . import fd as ofd
    Cd = coefficient_diagonal(d, n_el, geom, c=c, kappa=kappa, kappa_elem=kappa_elem)
    phi, Phi = separate(Cd, d, n_el)
    KM = [weighted_matrices(p, n_el, phi[l], Phi[l]) for l in range(d)]
    Kl, Ml = [k for k, _ in KM], [m for _, m in KM]
    Kt, Mtl = kron_spatial(Kl, Ml)
    sq = np.sqrt(diag_scaling(A, space_time(Mtl, Kt, Wt, Mt)))
    fac = ofd.setup(Kl, Ml, Wt.T.copy() if transpose else Wt, Mt)
    return lambda v: ofd.apply(fac, v / sq)[0] / sq


def loss_and_grads(kappa_elem, f, u_obs, d, p, n_el, p_t, n_el_t, geom="quarter_annulus", T=1.0, c=None,
                   gamma=1.0, nu=1.0, solver="direct", tol=1e-13):
    """L = 1/2 (u - u_obs)^T (M_t (x) M_s) (u - u_obs) with A(kappa) u = f;
    returns (L, u, dL/df, dL/dkappa). solver="direct": SuperLU; "gmres": the
    oracle's GMRES with the geometry-aware preconditioner (for sizes where a
    direct solve is too slow), to relative residual tol."""
    from .matrices import time_matrices
    from . import gmres as ogm
    Ms, Ks, elems = spatial_matrices(d, p, n_el, geom, c=c, kappa_elem=kappa_elem, element_stiffness=True)
    Wt, Mt = time_matrices(p_t, n_el_t, T)
    A = space_time(Ms, Ks, Wt, Mt, gamma, nu)
    if solver == "direct":
        lu = spla.splu(A.tocsc())
        solve = lambda b, tr: lu.solve(b, trans="T" if tr else "N")
    else:
        pre = {tr: geometry_preconditioner(A, d, p, n_el, Wt, Mt, geom, c=c, kappa_elem=kappa_elem, transpose=tr)
               for tr in (False, True)}
        AT = A.T.tocsr()

        def solve(b, tr):
            x, info = ogm.gmres((lambda v: AT @ v) if tr else (lambda v: A @ v), pre[tr], b, tol=tol)
            assert info["converged"]
            return x
    u = solve(f, False)
    Mst = sp.kron(sp.csr_matrix(Mt), Ms).tocsr()
    r = u - u_obs
    gu = Mst @ r
    L = 0.5 * float(r @ gu)
    lam = solve(gu, True)
    n_s = n_el + p - 2
    U = u.reshape(-1, n_s ** d)            # [time][space]
    Lm = lam.reshape(-1, n_s ** d)
    Ubar = Mt @ U                           # (M_t (x) I) u
    dk = np.zeros(len(elems))
    for e, (gi, Ke) in enumerate(elems):
        dk[e] = -nu * float(np.sum(Lm[:, gi] * (Ubar[:, gi] @ Ke.T)))
    return L, u, lam, dk
