"""Geometry maps F: (0,1)^d -> Omega of the mapped-domain problems (Sec. 2.2,
Sec. 4.6 and the quarter-annulus domain of Sec. 5).

Test infrastructure only (see ``oracle/__init__.py``).

The quarter annulus with radii 1 and 2 is the exact NURBS map: radial
direction eta_1 linear, angular direction eta_2 the rational quadratic
quarter circle with control points (1,0), (1,1), (0,1) and weights 1,
1/sqrt(2), 1. For d = 3 the annulus is extruded in eta_3 over (0, 1).

Each map returns the physical points and the Jacobian J[..., a, b] =
d x_a / d eta_b computed from the closed form below (quotient rule for the
rational curve); nothing here is shared with the CUDA library.
"""
import numpy as np

W1 = 1.0 / np.sqrt(2.0)
CTRL = np.array([[1.0, 0.0], [1.0, 1.0], [0.0, 1.0]])
WTS = np.array([1.0, W1, 1.0])


def quarter_circle(t):
    """Point C(t) and derivative C'(t) of the rational quadratic quarter circle."""
    t = np.asarray(t, dtype=np.float64)
    bern = np.stack([(1 - t) ** 2, 2 * t * (1 - t), t ** 2], axis=-1)        # Bernstein basis
    dbern = np.stack([-2 * (1 - t), 2 - 4 * t, 2 * t], axis=-1)
    w = bern @ WTS
    dw = dbern @ WTS
    num = (bern * WTS) @ CTRL
    dnum = (dbern * WTS) @ CTRL
    C = num / w[..., None]
    dC = (dnum - C * dw[..., None]) / w[..., None]
    return C, dC


def box(eta, lengths=None):
    """x = diag(L) eta."""
    eta = np.asarray(eta, dtype=np.float64)
    d = eta.shape[-1]
    L = np.ones(d) if lengths is None else np.asarray(lengths, dtype=np.float64)
    J = np.zeros(eta.shape + (d,))
    for a in range(d):
        J[..., a, a] = L[a]
    return eta * L, J


def quarter_annulus(eta):
    """F(eta) = (1 + eta_1) C(eta_2) [, eta_3] for eta of shape (..., d), d in {2, 3}."""
    eta = np.asarray(eta, dtype=np.float64)
    d = eta.shape[-1]
    r = 1.0 + eta[..., 0]
    C, dC = quarter_circle(eta[..., 1])
    x = np.zeros(eta.shape)
    J = np.zeros(eta.shape + (d,))
    x[..., 0] = r * C[..., 0]
    x[..., 1] = r * C[..., 1]
    J[..., 0, 0] = C[..., 0]
    J[..., 1, 0] = C[..., 1]
    J[..., 0, 1] = r * dC[..., 0]
    J[..., 1, 1] = r * dC[..., 1]
    if d == 3:
        x[..., 2] = eta[..., 2]
        J[..., 2, 2] = 1.0
    return x, J


MAPS = {"box": box, "quarter_annulus": quarter_annulus}
