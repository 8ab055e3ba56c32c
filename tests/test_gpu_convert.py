"""FP64 <-> double-float conversions of the double-float and tensor-core
kernels, assembled from the IEEE 754 bit fields with integer and FP32
instructions, against numpy's own FP32/FP64 rounding on the host.

Reference values: h + l must equal x to 2^-47 relative and |l| <= 2^-24 |h|
(a normalised pair); converting back gives the exact FP64 sum h + l; FP64 ->
FP32 is round-to-nearest (numpy's float32 cast) up to a rare double rounding
of exact ties (at most 1 ulp, in a negligible fraction of the entries); FP32 ->
FP64 is exact. Inputs cover every exponent of the fast path, both signs,
floats that a double holds exactly, zeros, subnormal doubles and magnitudes
that take the FP64 instructions."""
import numpy as np
import pytest

from paper_1909_07309_gb300 import stfd

pytestmark = pytest.mark.gpu
torch = pytest.importorskip("torch")


def _inputs():
    g = np.random.default_rng(11)
    n = 200_000
    mant = g.uniform(1.0, 2.0, n)
    expo = g.integers(-70, 127, n)
    x = np.ldexp(mant, expo) * np.where(g.random(n) < 0.5, -1.0, 1.0)
    as_float = g.standard_normal(5000).astype(np.float32).astype(np.float64)   # l must be 0
    special = np.array([0.0, -0.0, 5e-324, -2.2e-308, 1.0, -1.0, 2.0 ** -70, 2.0 ** 126 * 1.999999,
                        2.0 ** -80 * 1.3, -(2.0 ** -100) * 1.7, 2.0 ** 127 * 1.5, 1.0 + 2.0 ** -52,
                        1.0 - 2.0 ** -53, np.pi, -np.e, 1e-30, 3.0e38])
    ties = np.ldexp(1.0 + (2 * g.integers(0, 2 ** 22, 2000) + 1) * 2.0 ** -24, g.integers(-60, 100, 2000))
    return np.concatenate([x, as_float, special, ties])


def test_double_float_conversions_match_ieee():
    x = _inputs()
    n = x.size
    xd = torch.from_numpy(x).cuda()
    pairs = torch.empty(2 * n, dtype=torch.float32, device="cuda")
    back = torch.empty(n, dtype=torch.float64, device="cuda")
    f = torch.empty(n, dtype=torch.float32, device="cuda")
    fback = torch.empty(n, dtype=torch.float64, device="cuda")
    rc = stfd.load().stfd_probe_convert(xd.data_ptr(), n, pairs.data_ptr(), back.data_ptr(), f.data_ptr(),
                                        fback.data_ptr(), None)
    assert rc == 0
    torch.cuda.synchronize()
    pr = pairs.cpu().numpy().reshape(n, 2)
    h, l = pr[:, 0].astype(np.float64), pr[:, 1].astype(np.float64)
    back, f, fback = back.cpu().numpy(), f.cpu().numpy(), fback.cpu().numpy()

    finite32 = np.abs(x) < float(np.finfo(np.float32).max)
    fast = (np.abs(x) >= 2.0 ** -70) & (np.abs(x) < 2.0 ** 127)
    # the pair represents x to 2^-47 and is normalised
    assert np.all(np.abs(h[fast] + l[fast] - x[fast]) <= 2.0 ** -47 * np.abs(x[fast]))
    assert np.all(np.abs(l[fast]) <= 2.0 ** -24 * np.abs(h[fast]))
    # outside the fast path: the rounded FP32 value and its rounded remainder
    slow = finite32 & ~fast & (np.abs(x) >= 2.0 ** -1022)
    x32 = x.astype(np.float32).astype(np.float64)
    assert np.array_equal(h[slow], x32[slow])
    assert np.array_equal(l[slow], (x[slow] - x32[slow]).astype(np.float32).astype(np.float64))
    # zeros and subnormal doubles map to zero
    tiny = np.abs(x) < 2.0 ** -1022
    assert np.all(h[tiny] == 0) and np.all(l[tiny] == 0) and np.all(back[tiny] == 0)
    # floats held exactly: no low part, exact round trip
    exact = finite32 & (x32 == x) & fast
    assert np.all(l[exact] == 0) and np.array_equal(back[exact], x[exact])
    # back to FP64: the exact sum h + l
    sel = finite32 & ~tiny
    assert np.array_equal(back[sel], h[sel] + l[sel])
    # FP64 -> FP32 rounds to nearest (double rounding only at exact ties)
    ulp32 = np.spacing(np.abs(x32[fast]).astype(np.float32)).astype(np.float64)
    diff = np.abs(f[fast].astype(np.float64) - x32[fast])
    assert np.all(diff <= ulp32)
    assert np.count_nonzero(diff) <= 1e-4 * diff.size
    # FP32 -> FP64 is exact
    assert np.array_equal(fback[finite32], f[finite32].astype(np.float64))
