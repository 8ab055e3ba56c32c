"""The seven-digit tensor-core Algorithm 1 (STFD_FP64TC7) is FP64-grade.

Its mode products keep every digit pair down to 2^-48 of the row scales,
accumulate them exactly and round once, with FP64 intermediates and an IEEE
FP64 Step 3, so it agrees with the IEEE-FP64 path to within a few FP64
roundings per entry (far inside the 1e-11 target), and it is exactly
homogeneous under power-of-two scaling of the input over the whole FP64
range (row scaling by the entries' own exponents, 64-bit integer
recombination): P^{-1}(2^s r) = 2^s P^{-1} r bit for bit while the result
stays normal.
"""
import numpy as np
import pytest

from oracle import fd as ofd, matrices as omat
from paper_1909_07309_gb300 import inputs, stfd

pytestmark = pytest.mark.gpu
torch = pytest.importorskip("torch")


@pytest.mark.parametrize("d,p,n_el", [(1, 3, 60), (2, 2, 30), (3, 3, 13), (3, 2, 9)])
def test_agrees_with_ieee_fp64_path(d, p, n_el):
    K, M, Wt, Mt = stfd.heat_problem(d, p, n_el)
    P7 = stfd.FD(K, M, Wt, Mt, precision=stfd.STFD_FP64TC7)
    P64 = stfd.FD(K, M, Wt, Mt, precision=stfd.STFD_FP64)
    r = torch.as_tensor(inputs.standard_normal(P7.N, 41), device="cuda")
    s7, s64 = P7.apply(r), P64.apply(r)
    err = float(torch.linalg.norm(s7 - s64) / torch.linalg.norm(s64))
    assert err <= 2e-15, err
    # and the oracle (Algorithm 1 in complex arithmetic, whose eigenvector basis is
    # ill-conditioned (Table 2), so it is itself only good to about 1e-13 here)
    sm = [omat.space_matrices(p, n_el) for _ in range(d)]
    oWt, oMt = omat.time_matrices(p, n_el)
    ref, _ = ofd.apply(ofd.setup([k for k, _ in sm], [m for _, m in sm], oWt, oMt), r.cpu().numpy())
    assert np.linalg.norm(s7.cpu().numpy() - ref) <= 1e-11 * np.linalg.norm(ref)


@pytest.mark.parametrize("shift", [100, -100, 900, -900])
def test_exact_power_of_two_homogeneity(shift):
    K, M, Wt, Mt = stfd.heat_problem(3, 3, 10)
    P = stfd.FD(K, M, Wt, Mt, precision=stfd.STFD_FP64TC7)
    r = torch.as_tensor(inputs.standard_normal(P.N, 42), device="cuda")
    s = P.apply(r)
    s_sc = P.apply(torch.ldexp(r, torch.tensor(shift, device="cuda")))
    assert torch.equal(torch.ldexp(s, torch.tensor(shift, device="cuda")), s_sc)


def test_nonfinite_input_row_gives_nan():
    K, M, Wt, Mt = stfd.heat_problem(2, 2, 8)
    P = stfd.FD(K, M, Wt, Mt, precision=stfd.STFD_FP64TC7)
    r = torch.as_tensor(inputs.standard_normal(P.N, 43), device="cuda")
    r[5] = float("inf")
    s = P.apply(r)
    assert bool(torch.isnan(s).any())


@pytest.mark.parametrize("d,p,n_el,T,gamma,nu", [(1, 3, 60, 1.0, 1.0, 1.0), (2, 2, 30, 0.5, 2.0, 0.3),
                                                 (3, 3, 13, 1.0, 1.0, 1.0), (3, 4, 9, 1.5, 0.7, 1.9),
                                                 (2, 1, 40, 1.0, 1.0, 1.0)])
def test_integer_limb_matvec_agrees_with_ieee_fp64(d, p, n_el, T, gamma, nu):
    """STFD_OP_FX64 forms every band product exactly and rounds once: it agrees
    with the IEEE-FP64 matvec within a few FP64 roundings, for both A and A^T."""
    K, M, Wt, Mt = stfd.heat_problem(d, p, n_el, T=T)
    Ax = stfd.KronOp(K, M, Wt, Mt, gamma, nu, arith=stfd.STFD_OP_FX64)
    A64 = stfd.KronOp(K, M, Wt, Mt, gamma, nu, arith=stfd.STFD_OP_FP64)
    x = torch.as_tensor(inputs.standard_normal(Ax.N, 44), device="cuda")
    for tr in (False, True):
        y, y64 = Ax.matvec(x, transpose=tr), A64.matvec(x, transpose=tr)
        err = float(torch.max(torch.abs(y - y64)) / torch.max(torch.abs(y64)))
        assert err <= 1e-15, (tr, err)


@pytest.mark.parametrize("shift", [100, -100, 900, -900])
def test_integer_limb_matvec_power_of_two_homogeneity(shift):
    K, M, Wt, Mt = stfd.heat_problem(3, 3, 10)
    A = stfd.KronOp(K, M, Wt, Mt, arith=stfd.STFD_OP_FX64)
    x = torch.as_tensor(inputs.standard_normal(A.N, 45), device="cuda")
    two = torch.tensor(shift, device="cuda")
    assert torch.equal(torch.ldexp(A.matvec(x), two), A.matvec(torch.ldexp(x, two)))


@pytest.mark.parametrize("shift", [100, -100, -1000, 1000])
@pytest.mark.parametrize("which", ["fd_df32", "fd_tc48", "mv_df32"])
def test_double_float_paths_scale_exactly(which, shift):
    """The double-float paths (FP32 exponent range) work on the input scaled by
    a power of two and scale back: inputs at 2^+-100 and 2^+-1000 give the
    unscaled result times the same power of two, bit for bit."""
    K, M, Wt, Mt = stfd.heat_problem(3, 3, 10)
    if which == "mv_df32":
        op = stfd.KronOp(K, M, Wt, Mt, arith=stfd.STFD_OP_DF32).matvec
    else:
        prec = stfd.STFD_DF32 if which == "fd_df32" else stfd.STFD_FP64TC
        op = stfd.FD(K, M, Wt, Mt, precision=prec).apply
    x = torch.as_tensor(inputs.standard_normal(int(np.prod([k.shape[0] for k in K]) * Wt.shape[0]), 46),
                        device="cuda")
    two = torch.tensor(shift, device="cuda")
    y = op(x)
    ys = op(torch.ldexp(x, two))
    assert torch.equal(torch.ldexp(y, two), ys)
    assert bool(torch.isfinite(ys).all())
