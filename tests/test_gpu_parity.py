"""GPU parity: the CUDA path (through the C ABI) against the oracle.

Tolerances (FP64 path): fd_apply 1e-11 relative (the target for the
preconditioner), st_matvec 1e-13 relative to the largest entry, GMRES true
relative residual <= 1e-8 (the paper's tolerance, Sec. 5).
"""
import numpy as np
import pytest
import scipy.sparse.linalg as spla

from oracle import assemble, fd as ofd, gmres as ogmres, kron as okron, matrices as omat
from paper_1909_07309_gb300 import inputs, stfd

pytestmark = pytest.mark.gpu
torch = pytest.importorskip("torch")


def dev(x):
    return torch.as_tensor(np.ascontiguousarray(x), dtype=torch.float64, device="cuda")


def host(t):
    torch.cuda.synchronize()
    return t.detach().cpu().numpy()


def oracle_factors(d, p, n_el, T=1.0, p_t=None, n_el_t=None):
    p_t = p if p_t is None else p_t
    n_el_t = n_el if n_el_t is None else n_el_t
    sm = [omat.space_matrices(p, n_el) for _ in range(d)]
    Wt, Mt = omat.time_matrices(p_t, n_el_t, T)
    return [k for k, _ in sm], [m for _, m in sm], Wt, Mt


FD_CASES = [  # d, p, n_el, T, gamma, nu, nrhs  (n_t - 1 = n_el + p - 2 takes both parities)
    (1, 1, 7, 1.0, 1.0, 1.0, 1),
    (1, 2, 255, 1.0, 1.0, 1.0, 1),          # largest univariate size: n_t = 256
    (1, 4, 40, 0.5, 2.0, 0.3, 3),
    (2, 1, 1, 1.0, 1.0, 1.0, 1),            # degenerate: n_s = 0 -> skipped below
    (2, 2, 1, 1.0, 1.0, 1.0, 1),            # n_s = 1, n_t = 2
    (2, 2, 16, 1.0, 1.0, 1.0, 1),           # the small workload
    (2, 3, 21, 2.0, 0.7, 1.9, 2),
    (3, 2, 9, 1.0, 1.0, 1.0, 1),
    (3, 3, 13, 1.0, 1.3, 0.6, 1),
    (3, 4, 10, 1.5, 1.0, 1.0, 2),
]


@pytest.mark.parametrize("prec", [stfd.STFD_FP64, stfd.STFD_DF32, stfd.STFD_FP64TC, stfd.STFD_FP64TC7])
@pytest.mark.parametrize("d,p,n_el,T,gamma,nu,nrhs", FD_CASES)
def test_fd_apply_matches_oracle(d, p, n_el, T, gamma, nu, nrhs, prec):
    """FP64, double-float and tensor-core digit-sliced (six and seven digits)
    Algorithm 1 against the oracle, 1e-11."""
    if n_el + p - 2 < 1:
        pytest.skip("no spatial dofs")
    if prec in (stfd.STFD_FP64TC, stfd.STFD_FP64TC7) and n_el + p - 1 > 80:
        pytest.skip("tensor-core digit-sliced paths take univariate sizes <= 80")
    K, M, Wt, Mt = stfd.heat_problem(d, p, n_el, T=T)
    P = stfd.FD(K, M, Wt, Mt, gamma, nu, precision=prec)
    r = inputs.standard_normal(P.N, seed=11 + d + p, batch=nrhs).reshape(nrhs, P.N)
    s = host(P.apply(dev(r)))
    oK, oM, oWt, oMt = oracle_factors(d, p, n_el, T)
    fac = ofd.setup(oK, oM, oWt, oMt)
    for k in range(nrhs):
        ref, _ = ofd.apply(fac, r[k], gamma, nu)
        err = np.linalg.norm(s[k] - ref) / np.linalg.norm(ref)
        assert err <= 1e-11, err
        assert np.max(np.abs(s[k] - ref)) <= 1e-11 * np.max(np.abs(ref))


@pytest.mark.parametrize("d,p,n_el", [(1, 3, 5), (2, 2, 4), (3, 2, 3)])
def test_fd_apply_matches_direct_solve(d, p, n_el):
    """Tiny meshes: P^{-1} r by SuperLU on the directly assembled matrix."""
    K, M, Wt, Mt = stfd.heat_problem(d, p, n_el)
    P = stfd.FD(K, M, Wt, Mt, 1.0, 1.0)
    r = inputs.standard_normal(P.N, seed=5)
    s = host(P.apply(dev(r)))
    A = assemble.assemble_space_time(d, p, n_el, p, n_el)
    ref = spla.spsolve(A.tocsc(), r)
    assert np.linalg.norm(s - ref) <= 1e-11 * np.linalg.norm(ref)


MV_CASES = [(1, 3, 30, 1.0, 1.0, 1.0, 1), (2, 2, 16, 1.0, 1.0, 1.0, 2), (2, 4, 11, 0.5, 0.4, 2.5, 1),
            (3, 3, 13, 1.0, 1.0, 1.0, 1), (3, 1, 17, 2.0, 1.1, 0.9, 1),
            (1, 2, 120, 1.0, 1.0, 1.0, 1)]   # n_t = 121: the time pass takes the unpaired kernel


@pytest.mark.parametrize("arith", [stfd.STFD_OP_FP64, stfd.STFD_OP_DF32, stfd.STFD_OP_FX64])
@pytest.mark.parametrize("d,p,n_el,T,gamma,nu,nrhs", MV_CASES)
def test_st_matvec_matches_oracle(d, p, n_el, T, gamma, nu, nrhs, arith):
    """FP64, integer-limb FP64 and double-float (about 48-bit) matvec all agree
    with the oracle to 1e-13."""
    K, M, Wt, Mt = stfd.heat_problem(d, p, n_el, T=T)
    A = stfd.KronOp(K, M, Wt, Mt, gamma, nu, arith=arith)
    x = inputs.standard_normal(A.N, seed=3, batch=nrhs).reshape(nrhs, A.N)
    y = host(A.matvec(dev(x)))
    oK, oM, oWt, oMt = oracle_factors(d, p, n_el, T)
    for k in range(nrhs):
        ref = okron.st_matvec(x[k], oK, oM, oWt, oMt, gamma, nu)
        assert np.max(np.abs(y[k] - ref)) <= 1e-13 * np.max(np.abs(ref))


@pytest.mark.parametrize("arith,prec", [(stfd.STFD_OP_FP64, stfd.STFD_FP64), (stfd.STFD_OP_DF32, stfd.STFD_FP64),
                                        (stfd.STFD_OP_DF32, stfd.STFD_DF32), (stfd.STFD_OP_DF32, stfd.STFD_FP64TC),
                                        (stfd.STFD_OP_FP64, stfd.STFD_FP64TC7), (stfd.STFD_OP_FX64, stfd.STFD_FP64TC7)])
def test_gmres_unit_cube_single_iteration(arith, prec):
    """Unit cube, T = 1, constant coefficients: P = A, one iteration (Sec. 4, F = id)."""
    d, p, n_el = 3, 3, 12
    K, M, Wt, Mt = stfd.heat_problem(d, p, n_el)
    A = stfd.KronOp(K, M, Wt, Mt, arith=arith)
    P = stfd.FD(K, M, Wt, Mt, precision=prec)
    f = inputs.standard_normal(A.N, seed=21)
    u, info = A.gmres(P, dev(f))
    assert info["converged"] and info["iters"] == 1
    # one iteration leaves the residual of the preconditioner's own accuracy,
    # bounded by the 1e-11 relative-error target for P^{-1}
    assert info["rel_res_true"] <= 1e-11
    oK, oM, oWt, oMt = oracle_factors(d, p, n_el)
    ref = ofd.fd_solve(oK, oM, oWt, oMt, f)
    assert np.linalg.norm(host(u) - ref) <= 1e-11 * np.linalg.norm(ref)


@pytest.mark.parametrize("restart,arith", [(100, stfd.STFD_OP_FP64), (4, stfd.STFD_OP_FP64), (100, stfd.STFD_OP_DF32),
                                           (4, stfd.STFD_OP_FX64)])
def test_gmres_mismatched_preconditioner(restart, arith):
    """nu_A = 2, nu_P = 1: several iterations; same count as the oracle's
    GMRES (same Krylov space; CGS2 vs MGS differ only by rounding), true
    residual <= 1e-8 and the solution of a direct solve."""
    d, p, n_el = 2, 3, 10
    K, M, Wt, Mt = stfd.heat_problem(d, p, n_el)
    A = stfd.KronOp(K, M, Wt, Mt, 1.0, 2.0, arith=arith)
    P = stfd.FD(K, M, Wt, Mt, 1.0, 1.0)
    f = inputs.standard_normal(A.N, seed=8)
    u, info = A.gmres(P, dev(f), restart=restart)
    assert info["converged"] and info["rel_res_true"] <= 1e-8
    h = info["history"]
    assert len(h) == info["iters"] and np.all(np.diff(h) <= 1e-14)
    oK, oM, oWt, oMt = oracle_factors(d, p, n_el)
    fac = ofd.setup(oK, oM, oWt, oMt)
    Ao = okron.st_matrix_kron(oK, oM, oWt, oMt, 1.0, 2.0)
    _, oinfo = ogmres.gmres(lambda v: Ao @ v, lambda v: ofd.apply(fac, v)[0], f, restart=restart)
    assert abs(oinfo["iters"] - info["iters"]) <= 1
    ref = spla.spsolve(Ao.tocsc(), f)
    assert np.linalg.norm(host(u) - ref) <= 1e-6 * np.linalg.norm(ref)


def test_small_workload_end_to_end():
    """d = 2, p = 2, 16 elements: f = (M_t kron M_s) c, c ~ N(0,1) seed 0 (the
    library builds f with its mass operator), GMRES to 1e-8, compared with the
    oracle's SuperLU solve of P = A."""
    cfg = inputs.SMALL
    d, p, n_el = cfg["d"], cfg["p"], cfg["n_el"]
    K, M, Wt, Mt = stfd.heat_problem(d, p, n_el)
    mass = stfd.KronOp(M, M, Mt, Mt, 1.0, 0.0)
    A = stfd.KronOp(K, M, Wt, Mt)
    P = stfd.FD(K, M, Wt, Mt)
    c = inputs.standard_normal(A.N, cfg["rhs_seed"])
    f = mass.matvec(dev(c))
    oK, oM, oWt, oMt = oracle_factors(d, p, n_el)
    f_ref = okron.st_matvec(c, oM, oM, oMt, oMt, 1.0, 0.0)
    assert np.max(np.abs(host(f) - f_ref)) <= 1e-13 * np.max(np.abs(f_ref))
    u, info = A.gmres(P, f)
    assert info["converged"] and info["rel_res_true"] <= 1e-8
    ref = spla.spsolve(okron.st_matrix_kron(oK, oM, oWt, oMt).tocsc(), f_ref)
    assert np.linalg.norm(host(u) - ref) <= 1e-10 * np.linalg.norm(ref)


def _row_of_A(S, idx, oK, oM, oWt, oMt, gamma, nu, p):
    """(A s)_i for one multi-index i from the univariate rows (eq. syst_mat)."""
    d = len(oK)
    rng = [slice(max(0, i - p), i + p + 1) for i in idx]
    block = S[tuple(rng)]
    def contract(mats):
        out = block
        for l, Mx in enumerate(mats):
            out = np.tensordot(Mx[idx[l], rng[l]], out, axes=([0], [0]))
        return out
    val = gamma * contract(list(oM) + [oWt])
    for l in range(d):
        val += nu * contract([oK[k] if k == l else oM[k] for k in range(d)] + [oMt])
    return float(val)


@pytest.mark.parametrize("prec", [stfd.STFD_FP64, stfd.STFD_DF32, stfd.STFD_FP64TC, stfd.STFD_FP64TC7])
def test_fd_apply_full_size_residual_samples(prec):
    """Workload at scale (d = 3, p = 3, 64 elements, N = 18,125,250): P = A on
    the unit cube, so A (P^{-1} r) = r holds at every entry; checked on 400
    sampled entries with the oracle's univariate matrices."""
    cfg = inputs.SCALE
    d, p, n_el = cfg["d"], cfg["p"], cfg["n_el"]
    K, M, Wt, Mt = stfd.heat_problem(d, p, n_el)
    P = stfd.FD(K, M, Wt, Mt, precision=prec)
    r = inputs.standard_normal(P.N, cfg["rhs_seed"])
    s = host(P.apply(dev(r)))
    oK, oM, oWt, oMt = oracle_factors(d, p, n_el)
    shape = [k.shape[0] for k in oK] + [oWt.shape[0]]
    S = s.reshape(shape, order="F")
    R = r.reshape(shape, order="F")
    g = np.random.default_rng(2024)
    worst = 0.0
    for _ in range(400):
        idx = [int(g.integers(0, n)) for n in shape]
        worst = max(worst, abs(_row_of_A(S, idx, oK, oM, oWt, oMt, 1.0, 1.0, p) - R[tuple(idx)]))
    assert worst <= 1e-10 * np.max(np.abs(r)), worst


@pytest.mark.parametrize("arith", [stfd.STFD_OP_DF32, stfd.STFD_OP_FP64, stfd.STFD_OP_FX64])
def test_st_matvec_full_size_samples(arith):
    """Workload at scale (d = 3, p = 3, 64 elements, N = 18,125,250), the
    matvec the bench times: 400 sampled entries of A x against the rows the
    oracle's univariate matrices give one by one (eq. syst_mat). Tolerance
    1e-12 of the largest entry: the double-float passes round each product
    at about 2^-47 of |A||x|, which reaches 2.4 times max |A x| here."""
    cfg = inputs.SCALE
    d, p, n_el = cfg["d"], cfg["p"], cfg["n_el"]
    K, M, Wt, Mt = stfd.heat_problem(d, p, n_el)
    A = stfd.KronOp(K, M, Wt, Mt, arith=arith)
    x = inputs.standard_normal(A.N, cfg["rhs_seed"])
    y = host(A.matvec(dev(x)))
    oK, oM, oWt, oMt = oracle_factors(d, p, n_el)
    shape = [k.shape[0] for k in oK] + [oWt.shape[0]]
    X = x.reshape(shape, order="F")
    Y = y.reshape(shape, order="F")
    g = np.random.default_rng(2025)
    worst = 0.0
    for _ in range(400):
        idx = [int(g.integers(0, n)) for n in shape]
        worst = max(worst, abs(_row_of_A(X, idx, oK, oM, oWt, oMt, 1.0, 1.0, p) - Y[tuple(idx)]))
    assert worst <= 1e-12 * np.max(np.abs(y)), worst


def test_gmres_rejects_nan_and_reports_not_converged():
    K, M, Wt, Mt = stfd.heat_problem(2, 2, 6)
    A = stfd.KronOp(K, M, Wt, Mt, 1.0, 3.0)
    P = stfd.FD(K, M, Wt, Mt, 1.0, 1.0)
    f = inputs.standard_normal(A.N, seed=1)
    f_nan = f.copy()
    f_nan[7] = np.nan
    with pytest.raises(stfd.StfdError) as e:
        A.gmres(P, dev(f_nan))
    assert e.value.code == -5
    u, info = A.gmres(P, dev(f), tol=1e-14, max_it=2)
    assert info["status"] == 1 and not info["converged"] and info["iters"] == 2


@pytest.mark.parametrize("prec", [stfd.STFD_FP64TC, stfd.STFD_FP64TC7])
def test_fp64tc_rejects_large_factor(prec):
    K, M, Wt, Mt = stfd.heat_problem(1, 2, 90)      # n_t = 91 > 80
    with pytest.raises(stfd.StfdError):
        stfd.FD(K, M, Wt, Mt, precision=prec)


def test_argument_checks_on_device():
    K, M, Wt, Mt = stfd.heat_problem(2, 2, 5)
    P = stfd.FD(K, M, Wt, Mt)
    r = dev(np.ones(P.N))
    with pytest.raises(stfd.StfdError):
        P.apply(r, r)                        # aliasing is rejected
    lib = stfd.load()
    assert lib.stfd_fd_apply(P.handle, None, None, 0, None) == 0   # nrhs = 0 is a no-op
    with pytest.raises(stfd.StfdError):
        stfd.FD(K, M, Wt, Mt, gamma=-1.0)


@pytest.mark.parametrize("prec", [stfd.STFD_FP64TC, stfd.STFD_DF32, stfd.STFD_FP64TC7])
@pytest.mark.parametrize("d,p,n_el", [(2, 3, 21), (3, 3, 13)])
def test_fd_apply_unaligned_buffers_match(d, p, n_el, prec):
    """Input and output vectors that start 8 bytes past a 16-byte boundary take
    the element-wise copies of mode 1 instead of the bulk copies; the result is
    the same arithmetic, hence bit-identical."""
    K, M, Wt, Mt = stfd.heat_problem(d, p, n_el)
    P = stfd.FD(K, M, Wt, Mt, precision=prec)
    r = dev(inputs.standard_normal(P.N, 4))
    s_ref = P.apply(r)
    big_r = torch.zeros(P.N + 1, dtype=torch.float64, device="cuda")
    big_s = torch.zeros(P.N + 1, dtype=torch.float64, device="cuda")
    r1, s1 = big_r[1:], big_s[1:]
    assert r1.data_ptr() % 16 == 8 and s1.data_ptr() % 16 == 8
    r1.copy_(r)
    P.apply(r1, s1)
    assert torch.equal(s1, s_ref)


@pytest.mark.parametrize("kind", ["kron", "stencil"])
def test_fx64_matvec_nonfinite_input_gives_nan(kind):
    """The integer-limb matvecs turn a non-finite input entry into NaN outputs
    (as IEEE arithmetic would) instead of finite values; finite inputs stay finite."""
    if kind == "kron":
        K, M, Wt, Mt = stfd.heat_problem(3, 3, 6)
        A = stfd.KronOp(K, M, Wt, Mt, arith=stfd.STFD_OP_FX64)
    else:
        prob = stfd.mapped_problem(2, 3, 8, stfd.STFD_GEOM_QUARTER_ANNULUS)
        A = stfd.StencilOp(prob["n"], 3, prob["Ms"], prob["Ks"], prob["Wt"], prob["Mt"], arith=stfd.STFD_OP_FX64)
    x = inputs.standard_normal(A.N, seed=71)
    y = A.matvec(dev(x))
    assert bool(torch.isfinite(y).all())
    for bad in (np.inf, -np.inf, np.nan):
        xb = x.copy()
        xb[A.N // 2] = bad
        yb = A.matvec(dev(xb))
        assert bool(torch.isnan(yb).any())
        assert bool(torch.isnan(yb[A.N // 2]))
