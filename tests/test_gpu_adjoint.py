"""GPU parity of the adjoint building blocks against the oracle: the
transposed preconditioner P^{-T}, the transposed system matvec A^T and the
adjoint (transposed) FGMRES solve.

The oracle's P^{-T} r is its own Algorithm 1 run on the transposed pencil
(W_t^T in place of W_t: P^T = gamma W_t^T (x) M_s + nu M_t (x) K_s), pinned in
the CPU tests against a direct solve with the assembled P^T.
"""
import numpy as np
import pytest
import scipy.sparse.linalg as spla

from oracle import assemble, fd as ofd, kron as okron, matrices as omat
from paper_1909_07309_gb300 import inputs, stfd

pytestmark = pytest.mark.gpu
torch = pytest.importorskip("torch")


def dev(x):
    return torch.as_tensor(np.ascontiguousarray(x), dtype=torch.float64, device="cuda")


def host(t):
    torch.cuda.synchronize()
    return t.detach().cpu().numpy()


def oracle_factors(d, p, n_el, T=1.0):
    sm = [omat.space_matrices(p, n_el) for _ in range(d)]
    Wt, Mt = omat.time_matrices(p, n_el, T)
    return [k for k, _ in sm], [m for _, m in sm], Wt, Mt


CASES = [  # d, p, n_el, T, gamma, nu, nrhs (n_t - 1 odd and even)
    (1, 2, 9, 1.0, 1.0, 1.0, 1),
    (2, 2, 16, 1.0, 1.0, 1.0, 2),
    (2, 3, 21, 2.0, 0.7, 1.9, 1),
    (3, 3, 13, 1.0, 1.3, 0.6, 1),
    (3, 4, 10, 1.5, 1.0, 1.0, 1),
]


@pytest.mark.parametrize("prec", [stfd.STFD_FP64, stfd.STFD_DF32, stfd.STFD_FP64TC])
@pytest.mark.parametrize("d,p,n_el,T,gamma,nu,nrhs", CASES)
def test_fd_apply_transpose_matches_oracle(d, p, n_el, T, gamma, nu, nrhs, prec):
    K, M, Wt, Mt = stfd.heat_problem(d, p, n_el, T=T)
    P = stfd.FD(K, M, Wt, Mt, gamma, nu, precision=prec)
    r = inputs.standard_normal(P.N, seed=40 + d + p, batch=nrhs).reshape(nrhs, P.N)
    s = host(P.apply(dev(r), transpose=True))
    oK, oM, oWt, oMt = oracle_factors(d, p, n_el, T)
    fac_t = ofd.setup(oK, oM, oWt.T.copy(), oMt)
    for k in range(nrhs):
        ref, _ = ofd.apply(fac_t, r[k], gamma, nu)
        assert np.linalg.norm(s[k] - ref) <= 1e-11 * np.linalg.norm(ref)
    # the forward apply of the same handle is unchanged and differs from P^{-T}
    s_fwd = host(P.apply(dev(r)))
    assert np.linalg.norm(s_fwd - s) > 1e-6 * np.linalg.norm(s)


@pytest.mark.parametrize("prec,tol", [(stfd.STFD_TF32, 2e-3), (stfd.STFD_BF16, 2e-2)])
def test_fd_apply_transpose_low_precision(prec, tol):
    d, p, n_el = 3, 3, 12
    K, M, Wt, Mt = stfd.heat_problem(d, p, n_el)
    P = stfd.FD(K, M, Wt, Mt, precision=prec)
    r = inputs.standard_normal(P.N, seed=77)
    s = host(P.apply(dev(r), transpose=True))
    oK, oM, oWt, oMt = oracle_factors(d, p, n_el)
    ref, _ = ofd.apply(ofd.setup(oK, oM, oWt.T.copy(), oMt), r)
    assert np.linalg.norm(s - ref) <= tol * np.linalg.norm(ref)


@pytest.mark.parametrize("d,p,n_el", [(1, 3, 5), (2, 2, 4), (3, 2, 3)])
def test_fd_apply_transpose_matches_direct_solve(d, p, n_el):
    K, M, Wt, Mt = stfd.heat_problem(d, p, n_el)
    P = stfd.FD(K, M, Wt, Mt)
    r = inputs.standard_normal(P.N, seed=6)
    s = host(P.apply(dev(r), transpose=True))
    A = assemble.assemble_space_time(d, p, n_el, p, n_el)
    ref = spla.spsolve(A.T.tocsc(), r)
    assert np.linalg.norm(s - ref) <= 1e-11 * np.linalg.norm(ref)


@pytest.mark.parametrize("arith", [stfd.STFD_OP_FP64, stfd.STFD_OP_DF32])
@pytest.mark.parametrize("d,p,n_el,T,gamma,nu,nrhs", CASES)
def test_st_matvec_transpose_matches_oracle(d, p, n_el, T, gamma, nu, nrhs, arith):
    K, M, Wt, Mt = stfd.heat_problem(d, p, n_el, T=T)
    A = stfd.KronOp(K, M, Wt, Mt, gamma, nu, arith=arith)
    x = inputs.standard_normal(A.N, seed=9, batch=nrhs).reshape(nrhs, A.N)
    y = host(A.matvec(dev(x), transpose=True))
    oK, oM, oWt, oMt = oracle_factors(d, p, n_el, T)
    Ao = okron.st_matrix_kron(oK, oM, oWt, oMt, gamma, nu)
    for k in range(nrhs):
        ref = Ao.T @ x[k]
        assert np.max(np.abs(y[k] - ref)) <= 1e-13 * np.max(np.abs(ref))


def test_adjoint_identity_on_device():
    """<z, A x> = <A^T z, x> and <z, P^{-1} x> = <P^{-T} z, x> to rounding."""
    K, M, Wt, Mt = stfd.heat_problem(2, 3, 14)
    A = stfd.KronOp(K, M, Wt, Mt, 1.0, 1.7, arith=stfd.STFD_OP_DF32)
    P = stfd.FD(K, M, Wt, Mt, 1.0, 1.7, precision=stfd.STFD_FP64TC)
    x = dev(inputs.standard_normal(A.N, seed=1))
    z = dev(inputs.standard_normal(A.N, seed=2))
    for fwd, bwd in ((A.matvec(x), A.matvec(z, transpose=True)), (P.apply(x), P.apply(z, transpose=True))):
        lhs = float(torch.dot(z, fwd))
        rhs = float(torch.dot(bwd, x))
        assert abs(lhs - rhs) <= 1e-12 * float(torch.linalg.norm(z) * torch.linalg.norm(fwd))


@pytest.mark.parametrize("prec", [stfd.STFD_FP64, stfd.STFD_FP64TC, stfd.STFD_BF16])
def test_adjoint_gmres_matches_direct_solve(prec):
    """A^T lam = g with P^{-T} (nu_A = 2, nu_P = 1, several iterations); true
    residual <= 1e-8 and the SuperLU solution of the transposed system."""
    d, p, n_el = 2, 3, 10
    K, M, Wt, Mt = stfd.heat_problem(d, p, n_el)
    A = stfd.KronOp(K, M, Wt, Mt, 1.0, 2.0, arith=stfd.STFD_OP_DF32)
    P = stfd.FD(K, M, Wt, Mt, 1.0, 1.0, precision=prec)
    g = inputs.standard_normal(A.N, seed=12)
    lam, info = A.gmres(P, dev(g), transpose=True)
    assert info["converged"] and info["rel_res_true"] <= 1e-8 and info["iters"] > 1
    oK, oM, oWt, oMt = oracle_factors(d, p, n_el)
    Ao = okron.st_matrix_kron(oK, oM, oWt, oMt, 1.0, 2.0)
    ref = spla.spsolve(Ao.T.tocsc(), g)
    assert np.linalg.norm(host(lam) - ref) <= 1e-6 * np.linalg.norm(ref)
    # the forward solve of the same system gives a different vector
    u, _ = A.gmres(P, dev(g))
    assert np.linalg.norm(host(u) - host(lam)) > 1e-3 * np.linalg.norm(ref)
