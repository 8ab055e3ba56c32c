"""Failure detection on the GPU without faulting it: a bounded device wait that
is never satisfied gives up, raises the status flag and returns, and the host
reads it as STFD_ERR_TIMEOUT (the same path the tensor-core kernels use when
their pipeline stalls)."""
import pytest

from paper_1909_07309_gb300 import stfd

pytestmark = pytest.mark.gpu
torch = pytest.importorskip("torch")


def test_bounded_wait_times_out_and_reports():
    lib = stfd.load()
    assert lib.stfd_device_status() == 0                     # clean start
    assert lib.stfd_probe_bounded_wait(2000, None) == 0      # the kernel returns by itself
    assert lib.stfd_device_status() == -7                    # STFD_ERR_TIMEOUT
    assert lib.stfd_device_status() == 0                     # reading cleared it
    assert lib.stfd_probe_bounded_wait(0, None) == -1        # argument check


def test_context_usable_after_timeout():
    lib = stfd.load()
    lib.stfd_probe_bounded_wait(100, None)
    assert lib.stfd_device_status() == -7
    K, M, Wt, Mt = stfd.heat_problem(2, 2, 6)
    P = stfd.FD(K, M, Wt, Mt, precision=stfd.STFD_FP64TC)
    r = torch.ones(P.N, dtype=torch.float64, device="cuda")
    s = P.apply(r)
    torch.cuda.synchronize()
    assert bool(torch.isfinite(s).all())
    assert lib.stfd_device_status() == 0


@pytest.mark.parametrize("prec", [stfd.STFD_FP64TC, stfd.STFD_FP64TC7, stfd.STFD_TF32])
def test_solve_reports_timeout_of_its_preconditioner(prec):
    """With the wait limit at 0 every tensor-core wait gives up at once: the
    kernels let their own work in flight finish, skip the rest and return, and
    the solve (which reads the status word after each iteration) returns
    STFD_ERR_TIMEOUT. With the limit restored the same solve is clean."""
    lib = stfd.load()
    assert lib.stfd_device_status() == 0
    K, M, Wt, Mt = stfd.heat_problem(3, 3, 10)
    A = stfd.KronOp(K, M, Wt, Mt)
    P = stfd.FD(K, M, Wt, Mt, precision=prec)
    f = torch.ones(A.N, dtype=torch.float64, device="cuda")
    old = lib.stfd_get_wait_limit()
    assert lib.stfd_set_wait_limit(0) == 0
    try:
        with pytest.raises(stfd.StfdError) as e:
            A.gmres(P, f)
        assert e.value.code == -7
    finally:
        assert lib.stfd_set_wait_limit(old) == 0
    assert lib.stfd_device_status() == 0
    u, info = A.gmres(P, f)
    assert info["converged"] and info["rel_res_true"] <= 1e-8
    assert lib.stfd_set_wait_limit(-1) == -1


def test_fd_apply_reports_earlier_timeout_on_entry():
    """stfd_fd_apply is asynchronous: a timeout inside its kernels is reported
    by the next entry point that reads the status word (here the next apply)."""
    lib = stfd.load()
    assert lib.stfd_device_status() == 0
    K, M, Wt, Mt = stfd.heat_problem(2, 3, 12)
    P = stfd.FD(K, M, Wt, Mt, precision=stfd.STFD_FP64TC)
    r = torch.ones(P.N, dtype=torch.float64, device="cuda")
    s = torch.empty_like(r)
    old = lib.stfd_get_wait_limit()
    lib.stfd_set_wait_limit(0)
    try:
        P.apply(r, s)
        torch.cuda.synchronize()
    finally:
        lib.stfd_set_wait_limit(old)
    with pytest.raises(stfd.StfdError) as e:
        P.apply(r, s)
    assert e.value.code == -7
    P.apply(r, s)                      # cleared: the next apply is clean
    torch.cuda.synchronize()
    assert bool(torch.isfinite(s).all()) and lib.stfd_device_status() == 0
