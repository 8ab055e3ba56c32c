"""Pins of the oracle's discrete solution and GMRES (CPU only)."""
import numpy as np
import pytest
import scipy.sparse.linalg as spla

from oracle import assemble, fd, gmres, kron, loads, matrices

rng = np.random.default_rng(7)


@pytest.mark.parametrize("d,p,p_t,n_el,T,gamma,nu", [
    (1, 2, 1, 4, 1.0, 1.0, 1.0),
    (2, 2, 1, 3, 1.5, 2.0, 0.5),
    (2, 3, 2, 3, 1.0, 1.0, 1.0),
    (3, 2, 2, 2, 0.7, 1.0, 1.3),
])
def test_manufactured_polynomial_is_exact(d, p, p_t, n_el, T, gamma, nu):
    """u = t * prod_l x_l (1 - x_l) lies in the spline space for p_s >= 2,
    p_t >= 1, vanishes on the spatial boundary and at t = 0, so the Galerkin
    solution of Sec. 3.2 equals u. f = gamma u_t - nu Lap u (eq. problem).
    This pins the basis, the matrices and their index order, the assembly,
    the load vector and the boundary reduction together."""
    def bubble(xs):
        out = 1.0
        for x in xs:
            out = out * x * (1.0 - x)
        return out

    def f(*args):
        xs, t = args[:-1], args[-1]
        val = gamma * bubble(xs)
        for l in range(d):
            others = bubble([xs[k] for k in range(d) if k != l])
            val = val + nu * t * 2.0 * others
        return val + 0.0 * t

    A = assemble.assemble_space_time(d, p, n_el, p_t, n_el, gamma, nu, T=T)
    F = loads.load_quadrature(d, p, n_el, p_t, n_el, f, T=T)
    c = spla.spsolve(A.tocsc(), F)
    pts = rng.random((25, d + 1))
    pts[:, d] *= T
    uh = loads.evaluate(c, d, p, n_el, p_t, n_el, pts, T=T)
    u = pts[:, d] * bubble([pts[:, l] for l in range(d)])
    assert np.max(np.abs(uh - u)) <= 1e-10 * np.max(np.abs(u))


@pytest.mark.parametrize("p", [2, 3])
def test_l2_convergence_rate(p):
    """Sec. 5.1: optimal L2 order O(h^{p+1}) (here d = 1, u = sin(pi x) sin t):
    the error ratio per halving of h approaches 2^{p+1}."""
    errs = []
    for n_el in [4, 8, 16]:
        K, M = matrices.space_matrices(p, n_el)
        Wt, Mt = matrices.time_matrices(p, n_el)
        A = kron.st_matrix_kron([K], [M], Wt, Mt)
        Fx = loads.load_1d(p, n_el, 1.0, lambda x: np.sin(np.pi * x), 10)
        Ft = loads.load_1d(p, n_el, 1.0, lambda t: np.cos(t) + np.pi ** 2 * np.sin(t), 10, True, False)
        c = spla.spsolve(A.tocsc(), loads.load_separable([Fx], Ft))
        # L2 error by a tensor Gauss rule on every space-time element
        g, w = np.polynomial.legendre.leggauss(p + 3)
        pts, wts = [], []
        for ex in range(n_el):
            for et in range(n_el):
                xs = (ex + 0.5 * (g + 1)) / n_el
                ts = (et + 0.5 * (g + 1)) / n_el
                X, Tt = np.meshgrid(xs, ts, indexing="ij")
                pts.append(np.stack([X.ravel(), Tt.ravel()], axis=1))
                wts.append(np.outer(w, w).ravel() / (4 * n_el * n_el))
        pts = np.concatenate(pts)
        wts = np.concatenate(wts)
        uh = loads.evaluate(c, 1, p, n_el, p, n_el, pts)
        u = np.sin(np.pi * pts[:, 0]) * np.sin(pts[:, 1])
        errs.append(np.sqrt(np.sum(wts * (uh - u) ** 2)))
    rate = np.log2(errs[-2] / errs[-1])
    assert p + 0.6 < rate < p + 1.6, errs


def test_separable_load_equals_quadrature_load():
    """For separable f the Kronecker product of 1D loads equals the direct
    (d+1)-D quadrature load (both oracle routes, different code)."""
    d, p, n_el = 2, 2, 3
    fx = lambda x: np.sin(np.pi * x)
    ft = lambda t: np.cos(t) + 3 * np.sin(t)
    F1 = loads.load_separable([loads.load_1d(p, n_el, 1.0, fx, 8)] * d,
                              loads.load_1d(p, n_el, 1.0, ft, 8, True, False))
    F2 = loads.load_quadrature(d, p, n_el, p, n_el, lambda x, y, t: fx(x) * fx(y) * ft(t), nq=8)
    np.testing.assert_allclose(F1, F2, rtol=1e-13, atol=1e-16)


def _problem(d, p, n_el, gamma=1.0, nu=1.0):
    K, M = zip(*[matrices.space_matrices(p, n_el)] * d)
    Wt, Mt = matrices.time_matrices(p, n_el)
    return list(K), list(M), Wt, Mt


def test_gmres_unit_cube_one_iteration():
    """Unit cube, T = 1, constant coefficients: P = A (Sec. 4 with F = id), so
    FD-preconditioned GMRES converges in one iteration."""
    K, M, Wt, Mt = _problem(2, 2, 6)
    fac = fd.setup(K, M, Wt, Mt)
    f = rng.standard_normal(K[0].shape[0] ** 2 * Wt.shape[0])
    x, info = gmres.gmres(lambda v: kron.st_matvec(v, K, M, Wt, Mt),
                          lambda v: fd.apply(fac, v)[0], f)
    assert info["converged"] and info["iters"] == 1
    res = np.linalg.norm(f - kron.st_matvec(x, K, M, Wt, Mt)) / np.linalg.norm(f)
    assert res < 1e-12


def test_gmres_mismatched_preconditioner():
    """nu_A = 2 vs nu_P = 1: several iterations, monotone residual history,
    true residual <= 1e-8 and agreement with a direct solve."""
    K, M, Wt, Mt = _problem(2, 3, 5)
    fac = fd.setup(K, M, Wt, Mt)
    A = kron.st_matrix_kron(K, M, Wt, Mt, 1.0, 2.0)
    f = rng.standard_normal(A.shape[0])
    x, info = gmres.gmres(lambda v: A @ v, lambda v: fd.apply(fac, v, 1.0, 1.0)[0], f, restart=3)
    h = np.array(info["history"])
    assert info["converged"] and info["iters"] > 3      # at least one restart
    assert np.all(np.diff(h) <= 1e-15)
    # it stops at the first step whose residual estimate relative to ||f|| is below the tolerance
    assert h[-1] <= 1e-8 < h[-2]
    assert np.linalg.norm(f - A @ x) / np.linalg.norm(f) <= 1e-8
    xd = spla.spsolve(A.tocsc(), f)
    assert np.linalg.norm(x - xd) / np.linalg.norm(xd) < 1e-6


def test_gmres_minimises_the_residual_over_the_krylov_space():
    """GMRES's defining property: after j steps x_j = P^{-1} V_j y minimises
    ||f - A x|| over x in P^{-1} K_j(A P^{-1}, f). Checked against a least-squares
    solve on the explicit (power) Krylov basis, for j = 1..4 and restarted runs:
    a restart cycle minimises from the current residual instead."""
    g = np.random.default_rng(17)
    n = 60
    A = np.eye(n) * 3.0 + g.standard_normal((n, n)) / np.sqrt(n)
    Pm = np.eye(n) * 3.0 + np.triu(g.standard_normal((n, n)) / np.sqrt(n))
    f = g.standard_normal(n)
    AP = A @ np.linalg.inv(Pm)
    for j in range(1, 5):
        x, info = gmres.gmres(lambda v: A @ v, lambda v: np.linalg.solve(Pm, v), f, tol=1e-30, max_it=j)
        assert info["iters"] == j and not info["converged"]
        Kb = np.stack([np.linalg.matrix_power(AP, i) @ f for i in range(j)], axis=1)
        c = np.linalg.lstsq(AP @ Kb, f, rcond=None)[0]
        best = np.linalg.norm(f - AP @ Kb @ c)
        np.testing.assert_allclose(np.linalg.norm(f - A @ x), best, rtol=1e-10)
        np.testing.assert_allclose(info["history"][-1] * np.linalg.norm(f), best, rtol=1e-10)
    # GMRES(2) for 4 steps: two cycles, the second from r_2 = f - A x_2
    x2, _ = gmres.gmres(lambda v: A @ v, lambda v: np.linalg.solve(Pm, v), f, tol=1e-30, restart=2, max_it=2)
    x4, info = gmres.gmres(lambda v: A @ v, lambda v: np.linalg.solve(Pm, v), f, tol=1e-30, restart=2, max_it=4)
    r2 = f - A @ x2
    Kb = np.stack([r2, AP @ r2], axis=1)
    c = np.linalg.lstsq(AP @ Kb, r2, rcond=None)[0]
    np.testing.assert_allclose(np.linalg.norm(f - A @ x4), np.linalg.norm(r2 - AP @ Kb @ c), rtol=1e-10)
    assert np.all(np.diff(info["history"]) <= 1e-15)


def test_gmres_finite_termination_on_a_low_rank_perturbation():
    """Textbook termination: for A = I + U W^T of rank r (and P = I) the Krylov
    space has dimension at most r + 1, so GMRES reaches the solution in at
    most r + 1 steps."""
    g = np.random.default_rng(23)
    n, r = 80, 3
    A = np.eye(n) + g.standard_normal((n, r)) @ g.standard_normal((r, n)) / n
    f = g.standard_normal(n)
    x, info = gmres.gmres(lambda v: A @ v, lambda v: v, f, tol=1e-12)
    assert info["converged"] and info["iters"] <= r + 1
    np.testing.assert_allclose(x, np.linalg.solve(A, f), rtol=1e-10, atol=1e-12)
