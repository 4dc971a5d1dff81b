"""mfs_dot_noalloc, the allocation-free dot product, against mfs_dot.

mfs_dot_noalloc serves callers that may not call cudaMalloc while they run
(a framework's caching allocator already owns the device memory, a latency
loop cannot take cudaMalloc's device-wide synchronisation, a plug-in may only
allocate at initialisation): its partial sums live in a device array compiled
into the library instead of a handle's scratch.  Two calls in a row, on
different vectors, must agree with the handle-based mfs_dot within the
tolerance of the other dot-product tests (1e-13 of the bound on the sum);
both use the same reduction kernels, so they normally agree exactly.  Named to
be collected last.  Needs a GB300.
"""
import numpy as np
import pytest

torch = pytest.importorskip("torch")

from paper_1605_01522_gb300 import inputs, mfs

pytestmark = pytest.mark.gpu


def test_noalloc_dot_matches_handle_dot_on_two_calls():
    s = inputs.coupled_box_3d(ne=13, nfields=2)
    rng = np.random.default_rng(21)
    with mfs.Solver(s, max_levels=3, coarse_max=100) as lib:
        for _ in range(2):
            xh, yh = rng.standard_normal(s.ndofs), rng.standard_normal(s.ndofs)
            x, y = torch.from_numpy(xh).cuda(), torch.from_numpy(yh).cuda()
            ref = lib.dot(x, y)
            got = mfs.dot_noalloc(x, y)
            bound = np.abs(xh).max() * np.abs(yh).max() * s.ndofs ** 0.5
            assert abs(got - ref) <= 1e-13 * bound
            assert abs(got - float(np.dot(xh, yh))) <= 1e-13 * bound


def test_noalloc_dot_rejects_bad_arguments():
    x = torch.zeros(8, dtype=torch.float64, device="cuda")
    with pytest.raises(mfs.MfsError) as e:
        mfs.dot_noalloc(x, x, n=mfs.DOT_NOALLOC_MAX_N + 1)
    assert e.value.code == mfs.ERR_INVALID and "MAX_N" in str(e.value)
    with pytest.raises(mfs.MfsError):
        mfs.dot_noalloc(np.zeros(8), np.zeros(8), n=8)
    assert mfs.dot_noalloc(x, x, n=0) == 0.0
