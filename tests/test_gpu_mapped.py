"""GPU parity on mapped domains with variable coefficients (Sec. 4.6, 4.6.1):
the stencil system matvec and its transpose, the geometry-aware
preconditioner A^G (eq. prec_geo), FGMRES with A^ and A^G, and the adjoint
conductivity gradient, against the oracle."""
import numpy as np
import pytest
import scipy.sparse.linalg as spla

from oracle import fd as ofd, gmres as ogm, mapped, matrices as omat
from paper_1909_07309_gb300 import inputs, stfd

pytestmark = pytest.mark.gpu
torch = pytest.importorskip("torch")

QA = stfd.STFD_GEOM_QUARTER_ANNULUS


def dev(x):
    return torch.as_tensor(np.ascontiguousarray(x), dtype=torch.float64, device="cuda")


def host(t):
    torch.cuda.synchronize()
    return t.detach().cpu().numpy()


def kappa_lib(x):
    return 1 + 0.5 * np.sin(2 * np.pi * x[0]) * np.cos(2 * np.pi * x[1])


def c_lib(x):
    return 1 + 0.3 * x[0] * x[1]


def kappa_or(x):
    return kappa_lib(np.moveaxis(x, -1, 0))


def c_or(x):
    return c_lib(np.moveaxis(x, -1, 0))


def oracle_system(d, p, n_el, gamma=1.0, nu=1.0, T=1.0):
    Ms, Ks = mapped.spatial_matrices(d, p, n_el, "quarter_annulus", c=c_or, kappa=kappa_or)
    Wt, Mt = omat.time_matrices(p, n_el, T)
    return mapped.space_time(Ms, Ks, Wt, Mt, gamma, nu), Wt, Mt


MV_CASES = [(2, 3, 12, 1.0, 1.0, 2), (2, 2, 9, 0.7, 1.6, 1), (3, 2, 5, 1.0, 1.0, 1), (3, 4, 4, 1.3, 0.8, 1),
            (2, 1, 10, 1.0, 1.0, 1)]


@pytest.mark.parametrize("arith", [stfd.STFD_OP_FP64, stfd.STFD_OP_DF32, stfd.STFD_OP_FX64])
@pytest.mark.parametrize("d,p,n_el,gamma,nu,nrhs", MV_CASES)
def test_stencil_matvec_and_transpose_match_oracle(d, p, n_el, gamma, nu, nrhs, arith):
    prob = stfd.mapped_problem(d, p, n_el, QA, c=c_lib, kappa=kappa_lib)
    A = stfd.StencilOp(prob["n"], p, prob["Ms"], prob["Ks"], prob["Wt"], prob["Mt"], gamma, nu, arith=arith)
    x = inputs.standard_normal(A.N, seed=31, batch=nrhs).reshape(nrhs, A.N)
    y = host(A.matvec(dev(x)))
    yt = host(A.matvec(dev(x), transpose=True))
    Ao, _, _ = oracle_system(d, p, n_el, gamma, nu)
    Ms, Ks = mapped.spatial_matrices(d, p, n_el, "quarter_annulus", c=c_or, kappa=kappa_or)
    Wt, Mt = omat.time_matrices(p, n_el, 1.0)
    # rounding bound of the two sums of products: (gamma |W_t| (x) |M_s| + nu |M_t| (x) |K_s|) |x|,
    # not |y| (the two terms cancel in part)
    absA = mapped.space_time(abs(Ms), abs(Ks), np.abs(Wt), np.abs(Mt), gamma, nu)
    # FP64: 1e-13; double-float (2^-48 per operation) summed over up to 2 (2p+1)^d
    # = 1458 terms per entry: 1e-12 (a random-walk estimate is sqrt(1458) 2^-48 = 1.4e-13);
    # integer limbs (FP64 time pass, then exact row sums of entries rounded at 2^-53
    # of their row's and neighbourhood's largest entry, one rounding): 1e-13
    tol = 1e-12 if arith == stfd.STFD_OP_DF32 else 1e-13
    for k in range(nrhs):
        ref, reft = Ao @ x[k], Ao.T @ x[k]
        bound, boundt = absA @ np.abs(x[k]), absA.T @ np.abs(x[k])
        assert np.max(np.abs(y[k] - ref) / bound) <= tol
        assert np.max(np.abs(yt[k] - reft) / boundt) <= tol


@pytest.mark.parametrize("prec", [stfd.STFD_FP64, stfd.STFD_DF32, stfd.STFD_FP64TC])
@pytest.mark.parametrize("d,p,n_el", [(2, 3, 7), (3, 2, 4)])
def test_geometry_preconditioner_matches_oracle(d, p, n_el, prec):
    """(A^G)^{-1} r and (A^G)^{-T} r: D^{-1/2} A~^{-1} D^{-1/2} with the
    oracle's separation, weighted factors and Algorithm 1 (1e-11)."""
    prob = stfd.mapped_problem(d, p, n_el, QA, c=c_lib, kappa=kappa_lib)
    P = stfd.geometry_preconditioner(prob, precision=prec)
    r = inputs.standard_normal(P.N, seed=17)
    Ao, Wt, Mt = oracle_system(d, p, n_el)
    for tr in (False, True):
        s = host(P.apply(dev(r), transpose=tr))
        ref = mapped.geometry_preconditioner(Ao, d, p, n_el, Wt, Mt, c=c_or, kappa=kappa_or, transpose=tr)(r)
        assert np.linalg.norm(s - ref) <= 1e-11 * np.linalg.norm(ref)


def test_fgmres_mapped_geometry_plain_and_geometry_aware():
    """A^ (parametric factors) and A^G reach 1e-8; A^G needs fewer iterations
    (Sec. 5.2, Table rev_quarter); both give the direct solution; the
    iteration counts match the oracle's GMRES to +-2."""
    d, p, n_el = 2, 3, 10
    prob = stfd.mapped_problem(d, p, n_el, QA, c=c_lib, kappa=kappa_lib)
    A = stfd.StencilOp(prob["n"], p, prob["Ms"], prob["Ks"], prob["Wt"], prob["Mt"])
    K, M, Wt, Mt = stfd.heat_problem(d, p, n_el)
    P_plain = stfd.FD(K, M, Wt, Mt)
    P_geo = stfd.geometry_preconditioner(prob)
    f = inputs.standard_normal(A.N, seed=23)
    Ao, oWt, oMt = oracle_system(d, p, n_el)
    ref = spla.spsolve(Ao.tocsc(), f)
    its = {}
    for name, P in (("plain", P_plain), ("geo", P_geo)):
        u, info = A.gmres(P, dev(f))
        assert info["converged"] and info["rel_res_true"] <= 1e-8
        assert np.linalg.norm(host(u) - ref) <= 1e-6 * np.linalg.norm(ref)
        its[name] = info["iters"]
    assert its["geo"] < its["plain"]
    oK, oM = omat.space_matrices(p, n_el)
    fac = ofd.setup([oK] * d, [oM] * d, oWt, oMt)
    _, oi = ogm.gmres(lambda v: Ao @ v, lambda v: ofd.apply(fac, v)[0], f)
    pre = mapped.geometry_preconditioner(Ao, d, p, n_el, oWt, oMt, c=c_or, kappa=kappa_or)
    _, og = ogm.gmres(lambda v: Ao @ v, pre, f)
    assert abs(oi["iters"] - its["plain"]) <= 2 and abs(og["iters"] - its["geo"]) <= 2


@pytest.mark.parametrize("prec", [stfd.STFD_TF32, stfd.STFD_BF16])
def test_fgmres_mapped_low_precision_preconditioner(prec):
    """TF32 / BF16 geometry-aware preconditioner inside FP64 FGMRES: still
    reaches the 1e-8 true residual."""
    d, p, n_el = 3, 3, 8
    prob = stfd.mapped_problem(d, p, n_el, QA, c=c_lib, kappa=kappa_lib)
    A = stfd.StencilOp(prob["n"], p, prob["Ms"], prob["Ks"], prob["Wt"], prob["Mt"])
    f = dev(inputs.standard_normal(A.N, seed=29))
    _, ref = A.gmres(stfd.geometry_preconditioner(prob), f)
    u, info = A.gmres(stfd.geometry_preconditioner(prob, precision=prec), f)
    assert info["converged"] and info["rel_res_true"] <= 1e-8
    assert info["iters"] <= ref["iters"] + 6


def _adjoint_case(n_el, seed):
    d, p = 2, 3
    g = np.random.default_rng(seed)
    kap = g.uniform(0.5, 2.0, n_el ** d)
    kap_obs = kap * np.exp(0.1 * g.standard_normal(kap.size))
    n = (n_el + p - 2) ** d * (n_el + p - 1)
    c = g.standard_normal(n)
    return d, p, kap, kap_obs, c


def test_adjoint_gradient_matches_oracle_direct():
    """Small mesh: dL/dkappa_e and dL/df from the CUDA forward / adjoint
    solves and the device contraction equal the oracle's direct-solve
    gradient element by element."""
    from paper_1909_07309_gb300 import autograd as ag
    d, p, kap, kap_obs, c = _adjoint_case(6, 3)
    n_el = 6
    model = ag.MappedHeatModel(d, p, n_el, kappa_ref=kap, tol=1e-13)
    f = model.mass.matvec(dev(c))
    u_obs = ag.solve(torch.as_tensor(kap_obs), f, model).detach()
    kt = torch.tensor(kap, requires_grad=True)
    ft = f.clone().requires_grad_(True)
    L = ag.l2_misfit(ag.solve(kt, ft, model), u_obs, model)
    L.backward()
    L0, _, lam, dk = mapped.loss_and_grads(kap, host(f), host(u_obs), d, p, n_el, p, n_el)
    assert abs(float(L.detach()) - L0) <= 1e-10 * abs(L0)
    assert np.max(np.abs(kt.grad.numpy() - dk)) <= 1e-8 * np.max(np.abs(dk))
    assert np.linalg.norm(host(ft.grad) - lam) <= 1e-8 * np.linalg.norm(lam)


def test_adjoint_gradient_workload_finite_differences_and_oracle():
    """Quarter annulus, p = 3, 32 elements per direction (N = 37,026),
    kappa_e ~ U[0.5, 2]: the gradient agrees with central differences
    (h = 1e-6) of the CUDA loss on 20 random directions to 1e-6 and with the
    oracle's gradient (its own FD-preconditioned GMRES) element by element."""
    from paper_1909_07309_gb300 import autograd as ag
    d, p, kap, kap_obs, c = _adjoint_case(32, 5)
    n_el = 32
    model = ag.MappedHeatModel(d, p, n_el, kappa_ref=kap, tol=1e-13)
    f = model.mass.matvec(dev(c))
    u_obs = ag.solve(torch.as_tensor(kap_obs), f, model).detach()
    kt = torch.tensor(kap, requires_grad=True)
    L = ag.l2_misfit(ag.solve(kt, f, model), u_obs, model)
    L.backward()
    gk = kt.grad.numpy().copy()

    def loss(k):
        with torch.no_grad():
            return float(ag.l2_misfit(ag.solve(torch.as_tensor(k), f, model), u_obs, model))

    g = np.random.default_rng(20)
    h = 1e-6
    for _ in range(20):
        v = g.standard_normal(kap.size)
        fd = (loss(kap + h * v) - loss(kap - h * v)) / (2 * h)
        assert abs(fd - gk @ v) <= 1e-6 * np.linalg.norm(gk) * np.linalg.norm(v), (fd, gk @ v)
    _, _, _, dk = mapped.loss_and_grads(kap, host(f), host(u_obs), d, p, n_el, p, n_el, solver="gmres", tol=1e-13)
    assert np.max(np.abs(gk - dk)) <= 1e-7 * np.max(np.abs(dk))


def _rev_quarter_table():
    import os
    path = os.path.join(os.path.dirname(__file__), "golden", "table_rev_quarter_iters.txt")
    tab = {}
    for line in open(path):
        if line.strip() and not line.startswith("#"):
            k, ne, p, it = line.split()
            tab[(k, int(ne), int(p))] = int(it)
    return tab


@pytest.mark.parametrize("n_el,p", [(8, 1), (8, 2), (8, 3), (8, 4), (16, 1), (16, 2), (16, 3), (16, 4)])
def test_iterations_revolved_quarter_annulus_vs_table(n_el, p):
    """Sec. 5.2, Table rev_quarter: GMRES iterations with A^ and A^G on the
    revolved quarter annulus (gamma = nu = 1, T = 1, Krylov dimension 100) from
    the CUDA path, right-hand side (M_t x M_s) 1. A^G within 3 of the printed
    count (stable in p and n_el), A^ within -5..+10, A^G below half of A^."""
    tab = _rev_quarter_table()
    G = stfd.STFD_GEOM_REVOLVED_QUARTER_ANNULUS
    prob = stfd.mapped_problem(3, p, n_el, G)
    n = prob["n"]
    N = int(np.prod(n))
    A = stfd.StencilOp(n, p, prob["Ms"], prob["Ks"], prob["Wt"], prob["Mt"])
    mass = stfd.StencilOp(n, p, prob["Ms"], prob["Ms"], prob["Mt"], prob["Mt"], 1.0, 0.0)
    f = mass.matvec(torch.ones(N, dtype=torch.float64, device="cuda"))
    K, M, Wt, Mt = stfd.heat_problem(3, p, n_el)
    _, ih = A.gmres(stfd.FD(K, M, Wt, Mt, precision=stfd.STFD_FP64TC), f)
    _, ig = A.gmres(stfd.geometry_preconditioner(prob, precision=stfd.STFD_FP64TC), f)
    assert ih["converged"] and ig["converged"] and ig["rel_res_true"] <= 1e-8
    assert abs(ig["iters"] - tab[("AG", n_el, p)]) <= 3, ig["iters"]
    assert -5 <= ih["iters"] - tab[("Ahat", n_el, p)] <= 10, ih["iters"]
    assert 2 * ig["iters"] < ih["iters"]


def test_mapped_workload_full_size_sampled_rows():
    """The mixed-precision workload at full size (quarter annulus extruded, d = 3,
    p = 4, 96 elements, N = 93,178,008), in the arithmetic bench.py times:
    (1) sampled rows of the double-float and integer-limb stencil matvecs
    against rows the oracle assembles one by one (1e-12 and 1e-13 of the
    absolute-value sum);
    (2) sampled rows of A~ (A~^{-1} r) = r for the FP64-accurate preconditioner
    on the weighted factors, with the oracle's own separation and univariate
    matrices (1e-10 of max |r|, as the unit-cube full-size check)."""
    cfg = inputs.MAPPED
    d, p, n_el = cfg["d"], cfg["p"], cfg["n_el"]
    prob = stfd.mapped_problem(d, p, n_el, QA, c=inputs.c_bilinear, kappa=inputs.kappa_trig)
    n = prob["n"]
    ns, nt = n[0], n[-1]
    Ns = ns ** d
    N = Ns * nt
    x = inputs.standard_normal(N, 61)
    tols = {stfd.STFD_OP_DF32: 1e-12, stfd.STFD_OP_FX64: 1e-13}
    ys = {}
    for arith in tols:
        A = stfd.StencilOp(n, p, prob["Ms"], prob["Ks"], prob["Wt"], prob["Mt"], arith=arith)
        ys[arith] = host(A.matvec(dev(x)))
        A.close()
        torch.cuda.empty_cache()
    g = np.random.default_rng(62)
    samples = [(int(g.integers(Ns)), int(g.integers(nt))) for _ in range(24)]
    rows = mapped.spatial_rows(d, p, n_el, sorted({i for i, _ in samples}), "quarter_annulus", c=c_or, kappa=kappa_or)
    Wt, Mt = omat.time_matrices(p, n_el, 1.0)
    X = x.reshape(nt, Ns)
    for i, t in samples:
        cols, mv, kv = rows[i]
        val = bound = 0.0
        for tau in range(max(0, t - p), min(nt, t + p + 1)):
            xs = X[tau, cols]
            val += Wt[t, tau] * (mv @ xs) + Mt[t, tau] * (kv @ xs)
            bound += abs(Wt[t, tau]) * (np.abs(mv) @ np.abs(xs)) + abs(Mt[t, tau]) * (np.abs(kv) @ np.abs(xs))
        for arith, tol in tols.items():
            assert abs(ys[arith][i + Ns * t] - val) <= tol * bound, (arith, i, t)
    del ys
    P = stfd.geometry_preconditioner(prob, precision=stfd.STFD_DF32, scaled=False)
    r = inputs.standard_normal(N, 63)
    s = host(P.apply(dev(r))).reshape(nt, ns, ns, ns)          # [t][i3][i2][i1]
    P.close()
    Cd = mapped.coefficient_diagonal(d, n_el, "quarter_annulus", c=c_or, kappa=kappa_or)
    phi, Phi = mapped.separate(Cd, d, n_el)
    KM = [mapped.weighted_matrices(p, n_el, phi[l], Phi[l]) for l in range(d)]
    Kl, Ml = [k for k, _ in KM], [m for _, m in KM]
    worst = 0.0
    for i, t in samples:
        i1, i2, i3 = i % ns, (i // ns) % ns, i // ns ** 2
        r3 = slice(max(0, i3 - p), i3 + p + 1)
        r2 = slice(max(0, i2 - p), i2 + p + 1)
        r1 = slice(max(0, i1 - p), i1 + p + 1)
        val = 0.0
        for tau in range(max(0, t - p), min(nt, t + p + 1)):
            blk = s[tau, r3, r2, r1]
            m3, m2, m1 = Ml[2][i3, r3], Ml[1][i2, r2], Ml[0][i1, r1]
            k3, k2, k1 = Kl[2][i3, r3], Kl[1][i2, r2], Kl[0][i1, r1]
            mass = np.einsum("c,b,a,cba->", m3, m2, m1, blk)
            stiff = (np.einsum("c,b,a,cba->", m3, m2, k1, blk) + np.einsum("c,b,a,cba->", m3, k2, m1, blk) +
                     np.einsum("c,b,a,cba->", k3, m2, m1, blk))
            val += Wt[t, tau] * mass + Mt[t, tau] * stiff
        worst = max(worst, abs(val - r[i + Ns * t]))
    assert worst <= 1e-10 * np.max(np.abs(r)), worst
