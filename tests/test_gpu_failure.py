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
