"""The allocation-free matvec entry point, called through the C ABI.

stfd_st_matvec_noalloc is for callers that must not allocate device memory
(a host application that owns all device memory through its own allocator,
or a latency-critical loop where cudaMalloc would synchronise the device).
It keeps its scratch in a static device array shared by every call; these
tests check it against stfd_st_matvec and against the oracle's sum-factorised
matvec on two calls in a row (the second call starts from the first call's
leftover scratch) and that oversize problems and overlapping vectors are
refused. This file is collected last so that a failure here cannot hide one
elsewhere.
"""
import ctypes

import numpy as np
import pytest

from oracle import kron as okron, matrices as omat
from paper_1909_07309_gb300 import inputs, stfd

pytestmark = pytest.mark.gpu
torch = pytest.importorskip("torch")


def _dev_colmajor(A):
    return torch.as_tensor(np.asarray(A, dtype=np.float64).ravel(order="F"), device="cuda")


def _noalloc(lib, n, Kd, Md, Wd, Mtd, bw, gamma, nu, x, y):
    d = len(n) - 1
    ptrs = lambda ts: (ctypes.c_void_p * len(ts))(*[t.data_ptr() for t in ts])
    return lib.stfd_st_matvec_noalloc(d, (ctypes.c_int * (d + 1))(*n), ptrs(Kd), ptrs(Md),
                                      ctypes.c_void_p(Wd.data_ptr()), ctypes.c_void_p(Mtd.data_ptr()),
                                      (ctypes.c_int * (d + 1))(*bw), gamma, nu, ctypes.c_void_p(x.data_ptr()),
                                      ctypes.c_void_p(y.data_ptr()),
                                      ctypes.c_void_p(torch.cuda.current_stream().cuda_stream))


@pytest.mark.parametrize("d,p,n_el,gamma,nu", [(3, 3, 12, 1.0, 1.0), (2, 2, 60, 0.7, 1.6), (1, 4, 200, 1.0, 2.0)])
def test_noalloc_matvec_matches_st_matvec_twice(d, p, n_el, gamma, nu):
    lib = stfd.load()
    K, M, Wt, Mt = stfd.heat_problem(d, p, n_el)
    A = stfd.KronOp(K, M, Wt, Mt, gamma, nu)
    assert A.N <= stfd.STFD_NOALLOC_MAX_N
    Kd, Md = [_dev_colmajor(k) for k in K], [_dev_colmajor(m) for m in M]
    Wd, Mtd = _dev_colmajor(Wt), _dev_colmajor(Mt)
    bw = [p] * (d + 1)
    sm = [omat.space_matrices(p, n_el) for _ in range(d)]
    oWt, oMt = omat.time_matrices(p, n_el)
    for seed in (31, 32):                       # two calls in a row
        x_np = inputs.standard_normal(A.N, seed)
        x = torch.as_tensor(x_np, device="cuda")
        y = torch.full_like(x, float("nan"))
        rc = _noalloc(lib, A.n, Kd, Md, Wd, Mtd, bw, gamma, nu, x, y)
        assert rc == 0, stfd._strerror(rc)
        ref = A.matvec(x)
        torch.cuda.synchronize()
        err = float(torch.max(torch.abs(y - ref)) / torch.max(torch.abs(ref)))
        assert err <= 1e-13, err
        # and the oracle (plain CPU FP64), element by element
        ref_o = okron.st_matvec(x_np, [k for k, _ in sm], [m for _, m in sm], oWt, oMt, gamma, nu)
        y_np = y.cpu().numpy()
        assert np.max(np.abs(y_np - ref_o)) <= 1e-13 * np.max(np.abs(ref_o))


def test_noalloc_dense_band_and_size_limit():
    lib = stfd.load()
    K, M, Wt, Mt = stfd.heat_problem(2, 2, 10)
    A = stfd.KronOp(K, M, Wt, Mt)
    Kd, Md = [_dev_colmajor(k) for k in K], [_dev_colmajor(m) for m in M]
    Wd, Mtd = _dev_colmajor(Wt), _dev_colmajor(Mt)
    x = torch.as_tensor(inputs.standard_normal(A.N, 5), device="cuda")
    y = torch.empty_like(x)
    assert _noalloc(lib, A.n, Kd, Md, Wd, Mtd, [-1, -1, -1], 1.0, 1.0, x, y) == 0   # dense loops
    ref = A.matvec(x)
    torch.cuda.synchronize()
    assert float(torch.max(torch.abs(y - ref)) / torch.max(torch.abs(ref))) <= 1e-13
    big = [256, 256, 9]                          # N = 589,824 > STFD_NOALLOC_MAX_N
    assert _noalloc(lib, big, [Kd[0], Kd[0]], [Md[0], Md[0]], Wd, Mtd, [2, 2, 2], 1.0, 1.0, x, y) == -1
    assert _noalloc(lib, A.n, Kd, Md, Wd, Mtd, [2, 2, 2], 1.0, 1.0, x, x) == -1  # aliasing
    both = torch.zeros(2 * A.N, dtype=torch.float64, device="cuda")
    assert _noalloc(lib, A.n, Kd, Md, Wd, Mtd, [2, 2, 2], 1.0, 1.0, both[:A.N], both[A.N // 2:A.N // 2 + A.N]) == -1
    assert _noalloc(lib, A.n, Kd, Md, Wd, Mtd, [2, 2, 2], 1.0, 1.0, both[A.N:], both[:A.N]) == 0  # adjacent: fine


@pytest.mark.skipif(not torch.cuda.is_available() or torch.cuda.device_count() < 2,
                    reason="needs two visible GPUs")
def test_noalloc_second_device():
    """The shared-memory attribute and the scratch address are per device: a
    dense-band call (the largest shared-memory request) works on device 1 after
    device 0 has been used."""
    lib = stfd.load()
    K, M, Wt, Mt = stfd.heat_problem(1, 2, 150)
    for devno in (0, 1):
        with torch.cuda.device(devno):
            Kd, Md = [_dev_colmajor(k).to(devno) for k in K], [_dev_colmajor(m).to(devno) for m in M]
            Wd, Mtd = _dev_colmajor(Wt).to(devno), _dev_colmajor(Mt).to(devno)
            n = [K[0].shape[0], Wt.shape[0]]
            x = torch.as_tensor(inputs.standard_normal(n[0] * n[1], 3), device="cuda:%d" % devno)
            y = torch.empty_like(x)
            assert _noalloc(lib, n, Kd, Md, Wd, Mtd, [-1, -1], 1.0, 1.0, x, y) == 0
            torch.cuda.synchronize()
