"""Algorithm 1 (extended Fast Diagonalization) in complex arithmetic, as written.

Test infrastructure only (see ``oracle/__init__.py``).

Solves  P s = r  with  P = gamma W_t kron M_s + nu M_t kron K_s  (eq.
prec_definition; M_s, K_s of eq. space_univ_par_mat) in the order of Sec. 4:

1. factorisations: spatial pencils (eq. space_eig) and the time pencil
   through the arrowhead factorisation (eqs. arrow, U_t, split,
   factorization_first_block, syst_v, time_eig_2);
2. s~ = (U_t^* kron U_s^T) r;
3. q~ = (gamma Delta_t kron I + nu I kron Lambda_s)^{-1} s~ by the block LU
   of eq. block_LU;
4. s = (U_t kron U_s) q~.

Reading of Algorithm 1: its lines name the input s and the output r while
eq. prec_appl writes P s = r; we take the residual r as input and return
s = P^{-1} r.
"""
import numpy as np
import scipy.linalg as sla

from .kron import mode_product, to_tensor, vec


def spatial_factorization(K, M):
    """K U = M U Lambda with U^T M U = I (eq. space_eig), via scipy's generalized eigh."""
    lam, U = sla.eigh(K, M)
    return U, lam


def time_factorization(Wt, Mt):
    """Arrowhead factorisation W_t U_t = M_t U_t Delta_t, U_t^* M_t U_t = I (Sec. 4.2.2).

    Returns dict with U_t (complex n_t x n_t), Lambda (complex eigenvalues of
    the leading block, purely imaginary), g, sigma, Delta_t, r, rho, v.
    """
    n = Wt.shape[0]
    # eq. split
    W0 = Wt[:n - 1, :n - 1]
    w = Wt[:n - 1, n - 1]
    M0 = Mt[:n - 1, :n - 1]
    m = Mt[:n - 1, n - 1]
    # eq. factorization_first_block: W0 is skew-symmetric and M0 SPD. With
    # M0 = L L^T, S = L^{-1} W0 L^{-T} is real skew, so i S is Hermitian:
    # i S Z = Z diag(theta)  =>  S Z = Z diag(-i theta), and U0 = L^{-T} Z
    # gives W0 U0 = M0 U0 diag(-i theta) with U0^* M0 U0 = Z^* Z = I.
    L = np.linalg.cholesky(M0)
    Linv = sla.solve_triangular(L, np.eye(n - 1), lower=True)
    S = Linv @ W0 @ Linv.T
    theta, Z = np.linalg.eigh(1j * S)
    U0 = Linv.T @ Z
    lam0 = -1j * theta
    # eq. syst_v and the normalisation in the M_t norm
    v = np.linalg.solve(M0, -m)
    vv = np.concatenate([v, [1.0]])
    nrm = np.sqrt(vv @ Mt @ vv)
    r = v / nrm
    rho = 1.0 / nrm
    Ut = np.zeros((n, n), dtype=complex)
    Ut[:n - 1, :n - 1] = U0
    Ut[:n - 1, n - 1] = r
    Ut[n - 1, n - 1] = rho
    # eq. time_eig_2
    rr = np.concatenate([r, [rho]])
    g = U0.conj().T @ (np.hstack([W0, w[:, None]]) @ rr)
    sigma = rr @ Wt @ rr
    Delta = np.zeros((n, n), dtype=complex)
    Delta[:n - 1, :n - 1] = np.diag(lam0)
    Delta[:n - 1, n - 1] = g
    Delta[n - 1, :n - 1] = -g.conj()
    Delta[n - 1, n - 1] = sigma
    return {"Ut": Ut, "lam": lam0, "g": g, "sigma": sigma, "Delta": Delta,
            "r": r, "rho": rho, "v": v}


def setup(K, M, Wt, Mt):
    """Step 1 of Algorithm 1: all factorisations."""
    sp = [spatial_factorization(Kl, Ml) for Kl, Ml in zip(K, M)]
    tf = time_factorization(Wt, Mt)
    return {"U": [u for u, _ in sp], "lam_s": [l for _, l in sp], "time": tf}


def lambda_s(lam_s):
    """Diagonal of Lambda_s = sum_l I kron .. Lambda_l .. kron I, as a tensor (i_1 fastest)."""
    d = len(lam_s)
    shape = tuple(len(l) for l in lam_s)
    out = np.zeros(shape)
    for l, lam in enumerate(lam_s):
        sh = [1] * d
        sh[l] = len(lam)
        out = out + lam.reshape(sh)
    return out


def apply(fac, r_vec, gamma=1.0, nu=1.0):
    """Steps 2-4 of Algorithm 1: return s = P^{-1} r (real part; imaginary part ~ 0)."""
    U = fac["U"]
    tf = fac["time"]
    d = len(U)
    n_t = tf["Ut"].shape[0]
    shape = tuple(u.shape[0] for u in U) + (n_t,)
    X = to_tensor(np.asarray(r_vec, dtype=complex), shape)
    # Step 2: s~ = (U_t^* kron U_s^T) r  via eq. kron_vec_multi
    for l in range(d):
        X = mode_product(X, U[l].T, l)
    X = mode_product(X, tf["Ut"].conj().T, d)
    # Step 3: block LU of eq. block_LU, blocks indexed by the time index.
    Ls = lambda_s(fac["lam_s"])                       # diagonal of Lambda_s, spatial shape
    lam, g, sigma = tf["lam"], tf["g"], tf["sigma"]
    H = [gamma * lam[i] + nu * Ls for i in range(n_t - 1)]
    B = [gamma * g[i] for i in range(n_t - 1)]        # B_i = gamma g_i I
    Hn = gamma * sigma + nu * Ls
    Sdiag = Hn + sum(np.conj(B[i]) * B[i] / H[i] for i in range(n_t - 1))
    # forward: lower block factor (identity blocks, last row -B_i^* H_i^{-1})
    y_last = X[..., n_t - 1] + sum(np.conj(B[i]) * X[..., i] / H[i] for i in range(n_t - 1))
    Q = np.empty_like(X)
    Q[..., n_t - 1] = y_last / Sdiag
    for i in range(n_t - 1):
        Q[..., i] = (X[..., i] - B[i] * Q[..., n_t - 1]) / H[i]
    # Step 4: s = (U_t kron U_s) q~
    for l in range(d):
        Q = mode_product(Q, U[l], l)
    Q = mode_product(Q, tf["Ut"], d)
    out = vec(Q)
    return out.real, np.max(np.abs(out.imag)) if out.size else 0.0


def fd_solve(K, M, Wt, Mt, r_vec, gamma=1.0, nu=1.0):
    """Convenience: setup + apply, returns the real solution only."""
    return apply(setup(K, M, Wt, Mt), r_vec, gamma, nu)[0]
