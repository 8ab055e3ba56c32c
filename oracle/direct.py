"""Banded Gaussian elimination with partial pivoting, the oracle's own direct
solver for the assembled space-time matrices (Sec. 3.3, eq. sys_solve).

Test infrastructure only (see ``oracle/__init__.py``).

The space-time matrix of eq. syst_mat in vec order (i_1 fastest, time
slowest) is banded: an entry (i, j) is non-zero only if every coordinate of
i and j differs by at most the degree, so |i - j| <= p * (1 + n_1 + ... ) --
about p N_s. This module solves A x = b by the textbook algorithm (LU with
row interchanges, then forward and back substitution), restricted to the band:
with lower bandwidth kl and upper bandwidth ku, eliminating column k touches
rows k+1 .. k+kl, and row interchanges widen the upper part of U to kl + ku.
It serves as an independent check of the library routine (SuperLU) that the
other oracle modules use; it is slow (dense storage, one Python step per
column) and meant for tiny meshes only.
"""
import numpy as np


def bandwidths(A):
    """(kl, ku): the largest distance below and above the diagonal of a non-zero of A."""
    C = A.tocoo()
    off = C.col.astype(np.int64) - C.row.astype(np.int64)
    nz = C.data != 0
    kl = int(max(0, -off[nz].min())) if nz.any() else 0
    ku = int(max(0, off[nz].max())) if nz.any() else 0
    return kl, ku


def banded_lu(A):
    """Factor A by Gaussian elimination with partial pivoting, using the band.

    Returns (LU, ipiv, kl, ku): at step k, rows k and ipiv[k] (k <= ipiv[k] <=
    k + kl) were interchanged in the columns k and beyond, and the multipliers
    of column k were stored below the diagonal; they stay where they were put
    (later interchanges do not move them), so column k of L has its non-zeros
    in rows k+1 .. k+kl. U is on and above the diagonal, within kl + ku of it."""
    n = A.shape[0]
    kl, ku = bandwidths(A)
    LU = np.array(A.todense(), dtype=np.float64)
    ipiv = np.arange(n)
    for k in range(n):
        last = min(n, k + kl + 1)                 # rows that can hold a non-zero in column k
        piv = k + int(np.argmax(np.abs(LU[k:last, k])))
        if LU[piv, k] == 0.0:
            raise np.linalg.LinAlgError("singular matrix")
        ipiv[k] = piv
        if piv != k:
            LU[[k, piv], k:] = LU[[piv, k], k:]
        right = min(n, k + kl + ku + 1)           # U's band after interchanges
        LU[k + 1:last, k] /= LU[k, k]
        LU[k + 1:last, k + 1:right] -= np.outer(LU[k + 1:last, k], LU[k, k + 1:right])
    return LU, ipiv, kl, ku


def banded_solve(factors, b):
    """Solve A x = b with the factors of banded_lu: the interchanges and the
    multipliers of each step in turn, then back substitution with U."""
    LU, ipiv, kl, ku = factors
    n = LU.shape[0]
    y = np.array(b, dtype=np.float64)
    for k in range(n):
        if ipiv[k] != k:
            y[[k, ipiv[k]]] = y[[ipiv[k], k]]
        last = min(n, k + kl + 1)
        y[k + 1:last] -= LU[k + 1:last, k] * y[k]
    x = y
    for k in range(n - 1, -1, -1):
        right = min(n, k + kl + ku + 1)
        x[k] = (x[k] - LU[k, k + 1:right] @ x[k + 1:right]) / LU[k, k]
    return x
