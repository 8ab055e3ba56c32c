"""Seeded synthetic inputs shared by the CUDA path's tests/bench and the oracle.

This module holds workload shapes and random numbers only -- none of the
method's arithmetic (no basis functions, matrices, loads or solves). The
paper's experiments are analytic (unit cube / box domains, uniform knots,
manufactured solutions), so every input is synthetic.
"""
import numpy as np

# The small workload: heat equation on the unit square x (0, 1), d = 2,
# p = 2, 16 elements per direction, gamma = nu = 1, coefficients c ~ N(0, 1)
# with seed 0 projected to the right-hand side f = (M_t kron M_s) c.
SMALL = dict(name="unit square x (0,1), d=2, p=2, n_el=16", d=2, p=2, n_el=16,
             T=1.0, gamma=1.0, nu=1.0, rhs_seed=0)

# The workload at scale: unit cube x (0, 1), d = 3, p = 3, 64 elements per
# direction (n_s = 65, n_t = 66, N = 18,125,250), manufactured solution
# u = sin(pi x) sin(pi y) sin(pi z) sin(t); fd_apply timing input r ~ N(0, 1), seed 1.
SCALE = dict(name="unit cube x (0,1), d=3, p=3, n_el=64", d=3, p=3, n_el=64,
             T=1.0, gamma=1.0, nu=1.0, rhs_seed=1)


# Mixed-precision workload on a mapped domain: quarter annulus with radii 1
# and 2 (exact NURBS map) extruded over (0, 1), d = 3, p = 4, 96 elements per
# direction (n_s = 98, n_t = 99, N = 93,178,008), conductivity kappa and heat
# capacity c below, right-hand side f = (M_t kron M_s) c_rhs with c_rhs ~ N(0, 1)
# from seed 3.
MAPPED = dict(name="quarter annulus (NURBS, extruded) x (0,1), d=3, p=4, n_el=96, variable kappa, c",
              d=3, p=4, n_el=96, T=1.0, gamma=1.0, nu=1.0, rhs_seed=3)

# Adjoint workload: planar quarter annulus x (0, 1), d = 2, p = 3, 32 elements
# per direction (N = 37,026), piecewise-constant conductivity kappa_e ~ U[0.5, 2]
# per element (seed 5); observations from kappa_e * exp(0.1 xi_e), xi ~ N(0, 1)
# (same generator); f = (M_t kron M_s) c_rhs with c_rhs ~ N(0, 1) (same generator).
ADJOINT = dict(name="quarter annulus x (0,1), d=2, p=3, n_el=32, kappa_e ~ U[0.5,2]", d=2, p=3, n_el=32,
               T=1.0, gamma=1.0, nu=1.0, seed=5)


# Batched workload: 512 independent problems on the unit square x (0, 1),
# d = 2, n_el ~ U{8..48}, p ~ U{1..4}, nrhs ~ U{1..8} per problem, constant
# coefficients, right-hand sides with i.i.d. N(0, 1) entries; all draws from
# default_rng(4) in this order.
BATCH = dict(name="512 problems, unit square x (0,1), d=2, n_el~U{8..48}, p~U{1..4}, nrhs~U{1..8}",
             count=512, d=2, T=1.0, gamma=1.0, nu=1.0, seed=4)


def batch_draws(cfg):
    """(n_el, p, nrhs) arrays of the batched workload and a generator for its right-hand sides."""
    g = np.random.default_rng(cfg["seed"])
    n = cfg["count"]
    return g.integers(8, 49, n), g.integers(1, 5, n), g.integers(1, 9, n), g


def kappa_trig(x):
    """kappa(x) = 1 + 0.5 sin(2 pi x_1) cos(2 pi x_2); x has shape (d, m)."""
    return 1.0 + 0.5 * np.sin(2 * np.pi * x[0]) * np.cos(2 * np.pi * x[1])


def c_bilinear(x):
    """c(x) = 1 + 0.3 x_1 x_2; x has shape (d, m)."""
    return 1.0 + 0.3 * x[0] * x[1]


def adjoint_draws(cfg):
    """(kappa_e, kappa_obs_e, c_rhs) of the adjoint workload."""
    g = np.random.default_rng(cfg["seed"])
    n_e = cfg["n_el"] ** cfg["d"]
    kap = g.uniform(0.5, 2.0, n_e)
    kap_obs = kap * np.exp(0.1 * g.standard_normal(n_e))
    _, _, N = sizes(cfg)
    return kap, kap_obs, g.standard_normal(N)


def sizes(cfg):
    """(n_s, n_t, N) for uniform maximal-smoothness knots: n_s = n_el + p - 2, n_t = n_el + p - 1."""
    n_s = cfg["n_el"] + cfg["p"] - 2
    n_t = cfg["n_el"] + cfg["p"] - 1
    return n_s, n_t, n_s ** cfg["d"] * n_t


def standard_normal(n, seed, batch=1):
    """i.i.d. N(0, 1) FP64 vector(s) from numpy's default_rng(seed), shape (batch, n) or (n,)."""
    g = np.random.default_rng(seed)
    out = g.standard_normal((batch, n))
    return out[0] if batch == 1 else out


def uniform_points(n, dim, seed):
    """Uniform random points in [0, 1)^dim (evaluation sites for tests)."""
    return np.random.default_rng(seed).random((n, dim))
