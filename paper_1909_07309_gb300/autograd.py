"""torch.autograd wrappers of the space-time solve (argument marshalling only).

The forward pass solves A(kappa) u = f with FD-preconditioned flexible GMRES
in the CUDA library; the backward pass solves the adjoint system
A^T lam = dL/du with the transposed preconditioner P^{-T} (same factors,
transposed arrowhead) and contracts the per-element conductivity gradient
dL/dkappa_e = -nu lam^T (M_t (x) K_e) u on the device; dL/df = lam. Neither
is in the paper: both follow from its factorisation and its matrices
(Sec. 3.3, 4.3, 4.6.1). The Krylov bases live in the operator handles and are
not kept between forward and backward: the backward pass re-solves (the
adjoint Krylov space differs from the forward one anyway).
"""
import numpy as np
import torch

from . import stfd


class MappedHeatModel:
    """Heat problem on a mapped domain with piecewise-constant conductivity
    kappa_e per parametric element (colexicographic order) and heat capacity
    c(x): A(kappa) = gamma W_t (x) M_s[c] + nu M_t (x) K_s[kappa].

    The geometry-aware preconditioner (eq. prec_geo) is built once from the
    reference conductivity ``kappa_ref``; it only changes the iteration count.
    """

    def __init__(self, d, p, n_el, geom=stfd.STFD_GEOM_QUARTER_ANNULUS, c=None, kappa_ref=None, T=1.0,
                 gamma=1.0, nu=1.0, arith=stfd.STFD_OP_FX64, precision=stfd.STFD_FP64, tol=1e-10, nq=None,
                 restart=100, max_it=1000):
        self.d, self.p, self.n_el, self.geom = d, p, n_el, geom
        self.gamma, self.nu, self.arith, self.tol = gamma, nu, arith, tol
        self.restart, self.max_it = restart, max_it
        self.nq = p + 1 if nq is None else nq
        self.n_elem = n_el ** d
        kref = np.ones(self.n_elem) if kappa_ref is None else np.asarray(kappa_ref, dtype=np.float64)
        prob = stfd.mapped_problem(d, p, n_el, geom, c=c, kappa_elem=kref, nq=self.nq, T=T)
        self.prob = prob
        self.n = prob["n"]
        self.N = int(np.prod(self.n))
        self.P = stfd.geometry_preconditioner(prob, gamma, nu, precision=precision)
        self.Ms = prob["Ms"]
        zero = np.zeros_like(self.Ms)
        # (M_t (x) M_s) for the L2 misfit: gamma W_t (x) M_s with W_t := M_t, no stiffness
        self.mass = stfd.StencilOp(self.n, p, self.Ms, zero, prob["Mt"], prob["Mt"], 1.0, 0.0, arith=arith)
        self.Ke = torch.as_tensor(stfd.spatial_element_stiffness(d, p, n_el, geom, self.nq), device="cuda")
        self.iters = []

    def operator(self, kappa):
        """StencilOp of A(kappa) (host assembly of K_s = sum_e kappa_e K_e)."""
        k = np.asarray(kappa, dtype=np.float64).reshape(self.n_elem)
        _, Ks = stfd.spatial_assemble(self.d, self.p, self.n_el, self.geom, self.nq, None,
                                      np.repeat(k, self.nq ** self.d))
        return stfd.StencilOp(self.n, self.p, self.Ms, Ks, self.prob["Wt"], self.prob["Mt"], self.gamma, self.nu,
                              arith=self.arith)

    def solve(self, op, rhs, transpose=False):
        x, info = op.gmres(self.P, rhs.contiguous(), tol=self.tol, restart=self.restart, max_it=self.max_it,
                           transpose=transpose)
        if not info["converged"]:
            raise RuntimeError("GMRES did not converge: %r" % (info,))
        self.iters.append(info["iters"])
        return x


class _Solve(torch.autograd.Function):
    @staticmethod
    def forward(ctx, kappa, f, model):
        op = model.operator(kappa.detach().cpu().numpy())
        u = model.solve(op, f.detach())
        ctx.model, ctx.op = model, op
        ctx.kappa_device = kappa.device
        ctx.save_for_backward(u)
        return u

    @staticmethod
    def backward(ctx, grad_u):
        (u,) = ctx.saved_tensors
        model, op = ctx.model, ctx.op
        lam = model.solve(op, grad_u.detach(), transpose=True)
        gk = op.grad_kappa_elements(model.p, model.n_el, model.Ke, lam, u)
        return gk.to(ctx.kappa_device), lam, None


class _Mass(torch.autograd.Function):
    @staticmethod
    def forward(ctx, r, model):
        ctx.model = model
        return model.mass.matvec(r.detach().contiguous())

    @staticmethod
    def backward(ctx, g):
        return ctx.model.mass.matvec(g.detach().contiguous()), None


def solve(kappa, f, model):
    """u = A(kappa)^{-1} f, differentiable in kappa (per element) and f."""
    return _Solve.apply(kappa, f, model)


def l2_misfit(u, u_obs, model):
    """L = 1/2 (u - u_obs)^T (M_t (x) M_s) (u - u_obs), differentiable in u."""
    r = u - u_obs
    return 0.5 * torch.dot(r, _Mass.apply(r, model))
