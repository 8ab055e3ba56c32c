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
