"""Geometry maps F: (0,1)^d -> Omega of the mapped-domain problems (Sec. 2.2,
Sec. 4.6 and the quarter-annulus domain of Sec. 5).

Test infrastructure only (see ``oracle/__init__.py``).

The quarter annulus with radii 1 and 2 is the exact NURBS map: radial
direction eta_1 linear, angular direction eta_2 the rational quadratic
quarter circle with control points (1,0), (1,1), (0,1) and weights 1,
1/sqrt(2), 1. For d = 3 the annulus is extruded in eta_3 over (0, 1).
The revolved quarter annulus of Sec. 5.1 turns that planar annulus by a
right angle about the axis {(x_1, -1, 0)}, the angle following the same
rational quarter circle in eta_3.

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


def revolved_quarter_annulus(eta):
    """(a, b) = (1 + eta_1) C(eta_2);  F = (a, -1 + (b + 1) C_x(eta_3), (b + 1) C_y(eta_3))."""
    eta = np.asarray(eta, dtype=np.float64)
    r = 1.0 + eta[..., 0]
    C2, dC2 = quarter_circle(eta[..., 1])
    C3, dC3 = quarter_circle(eta[..., 2])
    a, b = r * C2[..., 0], r * C2[..., 1]
    da = np.stack([C2[..., 0], r * dC2[..., 0], np.zeros_like(r)], axis=-1)     # d a / d eta
    db = np.stack([C2[..., 1], r * dC2[..., 1], np.zeros_like(r)], axis=-1)     # d b / d eta
    x = np.stack([a, -1.0 + (b + 1.0) * C3[..., 0], (b + 1.0) * C3[..., 1]], axis=-1)
    J = np.zeros(eta.shape + (3,))
    J[..., 0, :] = da
    J[..., 1, :] = db * C3[..., 0, None]
    J[..., 2, :] = db * C3[..., 1, None]
    J[..., 1, 2] += (b + 1.0) * dC3[..., 0]
    J[..., 2, 2] += (b + 1.0) * dC3[..., 1]
    return x, J


MAPS = {"box": box, "quarter_annulus": quarter_annulus, "revolved_quarter_annulus": revolved_quarter_annulus}
