"""Pins of the oracle's adjoint quantities against the mathematics.

The oracle's Algorithm 1 on the transposed pencil (W_t^T in place of W_t) must
give P^{-T} r: checked against SuperLU on the directly assembled P^T, for both
parities of n_t - 1 (with and without the zero eigenvalue of the Remark in
Sec. 4.5)."""
import numpy as np
import pytest
import scipy.sparse.linalg as spla

from oracle import assemble, fd as ofd, matrices as omat
from paper_1909_07309_gb300 import inputs


@pytest.mark.parametrize("d,p,n_el", [(1, 2, 6), (1, 3, 6), (2, 2, 4), (2, 3, 3)])
def test_transposed_fd_is_inverse_of_PT(d, p, n_el):
    sm = [omat.space_matrices(p, n_el) for _ in range(d)]
    Wt, Mt = omat.time_matrices(p, n_el, 1.0)
    K, M = [k for k, _ in sm], [m for _, m in sm]
    fac_t = ofd.setup(K, M, Wt.T.copy(), Mt)
    A = assemble.assemble_space_time(d, p, n_el, p, n_el)
    r = inputs.standard_normal(A.shape[0], seed=3)
    s, _ = ofd.apply(fac_t, r)
    ref = spla.spsolve(A.T.tocsc(), r)
    assert np.linalg.norm(s - ref) <= 1e-12 * np.linalg.norm(ref)
    # and it is not P^{-1}
    s_fwd, _ = ofd.apply(ofd.setup(K, M, Wt, Mt), r)
    assert np.linalg.norm(s_fwd - s) > 1e-6 * np.linalg.norm(s)
