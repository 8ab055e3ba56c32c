"""Univariate B-splines (Sec. 2.1): open uniform knot vectors and Cox-de Boor.

Test infrastructure only (see ``oracle/__init__.py``).

Indices are 0-based here: the paper's b_{i,p} for i = 1..m is ``basis(..., i-1, ...)``.
"""
import numpy as np


def open_uniform_knots(p, n_el, length=1.0):
    """Open knot vector with maximal smoothness on [0, length] (Sec. 2.1, Sec. 5).

    xi_1 = .. = xi_{p+1} = 0, xi_m = .. = xi_{m+p+1} = length, interior knots
    simple and uniform, so m = n_el + p basis functions.
    """
    interior = [length * k / n_el for k in range(1, n_el)]
    return np.array([0.0] * (p + 1) + interior + [float(length)] * (p + 1))


def n_basis(knots, p):
    """m = len(knots) - p - 1 (the knot vector has m + p + 1 entries)."""
    return len(knots) - p - 1


def _last_nonempty_span(knots):
    for i in range(len(knots) - 2, -1, -1):
        if knots[i] < knots[i + 1]:
            return i
    raise ValueError("degenerate knot vector")


def _ratio(num, den):
    """The 0/0 = 0 convention of the Cox-de Boor recursion (Sec. 2.1).

    ``num`` is an array; ``den`` a scalar knot difference. When den == 0 the
    term multiplies a degree p-1 B-spline on an empty span, which vanishes,
    so the whole term is taken as 0.
    """
    if den == 0.0:
        return np.zeros_like(num)
    return num / den


def basis(knots, p, i, x):
    """b_{i,p}(x) by the Cox-de Boor recursion, evaluated at an array x.

    Degree 0 uses the half-open spans [xi_i, xi_{i+1}) of Sec. 2.1. The right
    end point x = xi_last would make every function vanish; we close the last
    non-empty span on the right (our reading; it only matters for point
    evaluation at the end point, e.g. b_{n_t}(T) = 1).
    """
    x = np.asarray(x, dtype=np.float64)
    if p == 0:
        lo, hi = knots[i], knots[i + 1]
        val = ((x >= lo) & (x < hi)).astype(np.float64)
        if i == _last_nonempty_span(knots):
            val = np.where(x == hi, 1.0, val)
        return val
    left = _ratio(x - knots[i], knots[i + p] - knots[i]) * basis(knots, p - 1, i, x)
    right = _ratio(knots[i + p + 1] - x, knots[i + p + 1] - knots[i + 1]) * basis(knots, p - 1, i + 1, x)
    return left + right


def basis_deriv(knots, p, i, x):
    """b'_{i,p}(x) by the textbook de Boor derivative formula (not in the paper).

    b'_{i,p} = p/(xi_{i+p}-xi_i) b_{i,p-1} - p/(xi_{i+p+1}-xi_{i+1}) b_{i+1,p-1},
    with the same 0/0 = 0 convention.
    """
    x = np.asarray(x, dtype=np.float64)
    if p == 0:
        return np.zeros_like(x)
    a = knots[i + p] - knots[i]
    b = knots[i + p + 1] - knots[i + 1]
    ta = (p / a) * basis(knots, p - 1, i, x) if a != 0.0 else np.zeros_like(x)
    tb = (p / b) * basis(knots, p - 1, i + 1, x) if b != 0.0 else np.zeros_like(x)
    return ta - tb


def all_basis(knots, p, x):
    """Matrix V[k, i] = b_{i,p}(x_k) for every basis function i = 0..m-1."""
    m = n_basis(knots, p)
    return np.stack([basis(knots, p, i, x) for i in range(m)], axis=-1)


def all_basis_deriv(knots, p, x):
    """Matrix D[k, i] = b'_{i,p}(x_k)."""
    m = n_basis(knots, p)
    return np.stack([basis_deriv(knots, p, i, x) for i in range(m)], axis=-1)
