"""Right-preconditioned GMRES, zero initial guess (Sec. 4.5 and the Sec. 5 set-up).

Test infrastructure only (see ``oracle/__init__.py``).

Arnoldi with modified Gram-Schmidt, Givens rotations on the Hessenberg
matrix, restart length ``restart`` (the paper's "maximum dimension of the
Krylov subspace", 100, or 25 at n_el = 128). The preconditioned directions
z_j = P^{-1} v_j are stored (the flexible form), which for a fixed P is the
same iterate as x = P^{-1} V y. Stops when the unpreconditioned residual
estimate |g_{j+1}| <= tol * ||f|| (reading: the paper states a tolerance of
1e-8 but not the norm; with right preconditioning this is ||f - A x|| / ||f||).
"""
import numpy as np


def gmres(matvec, precond, f, tol=1e-8, restart=100, max_it=1000):
    f = np.asarray(f, dtype=np.float64)
    n = f.size
    x = np.zeros(n)
    fnorm = np.linalg.norm(f)
    history = [1.0]
    if fnorm == 0.0:
        return x, {"iters": 0, "history": history, "converged": True}
    total = 0
    r = f.copy()
    while total < max_it:
        beta = np.linalg.norm(r)
        V = np.zeros((restart + 1, n))
        Z = np.zeros((restart, n))
        H = np.zeros((restart + 1, restart))
        cs = np.zeros(restart)
        sn = np.zeros(restart)
        g = np.zeros(restart + 1)
        g[0] = beta
        V[0] = r / beta
        j_done = 0
        converged = False
        for j in range(restart):
            Z[j] = precond(V[j])
            w = matvec(Z[j])
            for i in range(j + 1):                 # modified Gram-Schmidt
                H[i, j] = w @ V[i]
                w = w - H[i, j] * V[i]
            H[j + 1, j] = np.linalg.norm(w)
            if H[j + 1, j] != 0.0:
                V[j + 1] = w / H[j + 1, j]
            for i in range(j):                     # previous rotations
                t = cs[i] * H[i, j] + sn[i] * H[i + 1, j]
                H[i + 1, j] = -sn[i] * H[i, j] + cs[i] * H[i + 1, j]
                H[i, j] = t
            den = np.hypot(H[j, j], H[j + 1, j])
            cs[j] = H[j, j] / den
            sn[j] = H[j + 1, j] / den
            H[j, j] = den
            H[j + 1, j] = 0.0
            g[j + 1] = -sn[j] * g[j]
            g[j] = cs[j] * g[j]
            total += 1
            j_done = j + 1
            history.append(abs(g[j + 1]) / fnorm)
            if abs(g[j + 1]) <= tol * fnorm or total >= max_it:
                converged = abs(g[j + 1]) <= tol * fnorm
                break
        y = np.zeros(j_done)
        for i in range(j_done - 1, -1, -1):        # back substitution
            y[i] = (g[i] - H[i, i + 1:j_done] @ y[i + 1:]) / H[i, i]
        x = x + Z[:j_done].T @ y
        if converged:
            return x, {"iters": total, "history": history, "converged": True}
        r = f - matvec(x)
    return x, {"iters": total, "history": history, "converged": False}
