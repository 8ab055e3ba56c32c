"""Element-by-element parity at the sizes the bench times.

The workload at scale (unit cube x (0, 1), d = 3, p = 3, 64 elements,
N = 18,125,250) in the launch configuration bench.py uses: the whole
P^{-1} r of every preconditioner arithmetic the bench reports against the
oracle's Algorithm 1 (complex arithmetic, Sec. 4.3), and the whole A x of
both matvec arithmetics against the oracle's sum-factorised Kronecker matvec
(eq. kron_vec_multi). Tolerances: the 1e-11 relative error the preconditioner
must meet, in the 2-norm and in the max-norm, and 1e-13 of the largest entry
for the FP64 matvec (1e-12 for the double-float one, whose products round at
about 2^-47 of |A||x|).

The tensor-core digit-sliced preconditioner is also compared at its largest
univariate sizes (n = 80 and n = 65/66) on 2D problems.
"""
import numpy as np
import pytest

from oracle import fd as ofd, kron as okron, matrices as omat
from paper_1909_07309_gb300 import inputs, stfd

pytestmark = pytest.mark.gpu
torch = pytest.importorskip("torch")


def _oracle_factors(d, p, n_el):
    K, M = omat.space_matrices(p, n_el)
    Wt, Mt = omat.time_matrices(p, n_el)
    return [K] * d, [M] * d, Wt, Mt


@pytest.fixture(scope="module")
def scale():
    cfg = inputs.SCALE
    d, p, n_el = cfg["d"], cfg["p"], cfg["n_el"]
    oK, oM, oWt, oMt = _oracle_factors(d, p, n_el)
    r = inputs.standard_normal(inputs.sizes(cfg)[2], cfg["rhs_seed"])
    fac = ofd.setup(oK, oM, oWt, oMt)
    s_ref, _ = ofd.apply(fac, r, cfg["gamma"], cfg["nu"])
    y_ref = okron.st_matvec(r, oK, oM, oWt, oMt, cfg["gamma"], cfg["nu"])
    return dict(cfg=cfg, r=r, s_ref=s_ref, y_ref=y_ref, mats=stfd.heat_problem(d, p, n_el))


def _check_rel(s, ref, tol):
    err2 = np.linalg.norm(s - ref) / np.linalg.norm(ref)
    errm = np.max(np.abs(s - ref)) / np.max(np.abs(ref))
    assert err2 <= tol and errm <= tol, (err2, errm)
    return err2, errm


# every preconditioner arithmetic the bench times (the 7-digit one once built)
PRECS = [stfd.STFD_FP64, stfd.STFD_DF32, stfd.STFD_FP64TC] + (
    [stfd.STFD_FP64TC7] if hasattr(stfd, "STFD_FP64TC7") else [])
TC_PRECS = [stfd.STFD_FP64TC] + ([stfd.STFD_FP64TC7] if hasattr(stfd, "STFD_FP64TC7") else [])


@pytest.mark.parametrize("prec", PRECS)
def test_fd_apply_full_size_matches_oracle(scale, prec):
    cfg = scale["cfg"]
    K, M, Wt, Mt = scale["mats"]
    P = stfd.FD(K, M, Wt, Mt, cfg["gamma"], cfg["nu"], precision=prec)
    r = torch.as_tensor(scale["r"], device="cuda")
    s = torch.empty_like(r)
    P.apply(r, s)
    torch.cuda.synchronize()
    _check_rel(s.cpu().numpy(), scale["s_ref"], 1e-11)
    P.close()


@pytest.mark.parametrize("arith,tol", [(stfd.STFD_OP_FP64, 1e-13), (stfd.STFD_OP_FX64, 1e-13), (stfd.STFD_OP_DF32, 1e-12)])
def test_st_matvec_full_size_matches_oracle(scale, arith, tol):
    cfg = scale["cfg"]
    K, M, Wt, Mt = scale["mats"]
    A = stfd.KronOp(K, M, Wt, Mt, cfg["gamma"], cfg["nu"], arith=arith)
    x = torch.as_tensor(scale["r"], device="cuda")
    y = torch.empty_like(x)
    A.matvec(x, y)
    torch.cuda.synchronize()
    ref = scale["y_ref"]
    assert np.max(np.abs(y.cpu().numpy() - ref)) <= tol * np.max(np.abs(ref))
    A.close()


@pytest.mark.parametrize("prec", TC_PRECS)
@pytest.mark.parametrize("p,n_el", [(3, 78), (3, 64)])   # n = 79 / 80 and n = 65 / 66
def test_digit_sliced_at_largest_sizes(prec, p, n_el):
    d = 2
    K, M, Wt, Mt = stfd.heat_problem(d, p, n_el)
    P = stfd.FD(K, M, Wt, Mt, 1.0, 1.0, precision=prec)
    r = inputs.standard_normal(P.N, 17)
    s = P.apply(torch.as_tensor(r, device="cuda")).cpu().numpy()
    oK, oM, oWt, oMt = _oracle_factors(d, p, n_el)
    ref, _ = ofd.apply(ofd.setup(oK, oM, oWt, oMt), r)
    _check_rel(s, ref, 1e-11)
