"""mfs_dot_noalloc, the allocation-free dot product, against mfs_dot.

mfs_dot_noalloc serves callers that may not call cudaMalloc while they run
(a framework's caching allocator already owns the device memory, a latency
loop cannot take cudaMalloc's device-wide synchronisation, a plug-in may only
allocate at initialisation): its partial sums live in a device array compiled
into the library instead of a handle's scratch.  Calls in a row, on
different vectors, must agree with the handle-based mfs_dot within the
tolerance of the other dot-product tests (1e-13 of the bound on the sum);
both use the same reduction kernels, so they normally agree exactly.  The
sizes cover a few reduction blocks, the full block count of the array (n of
the 64^3 box, not a multiple of the 2048-entry chunk) and a smaller call
after that larger one.  Named to be collected last.  Needs a GB300.
"""
import numpy as np
import pytest

torch = pytest.importorskip("torch")

from paper_1605_01522_gb300 import inputs, mfs

pytestmark = pytest.mark.gpu


def _check(lib, n, rng):
    xh, yh = rng.standard_normal(n), rng.standard_normal(n)
    x, y = torch.from_numpy(xh).cuda(), torch.from_numpy(yh).cuda()
    ref = lib.dot(x[:lib.n], y[:lib.n]) if n == lib.n else None
    got = mfs.dot_noalloc(x, y)
    bound = np.abs(xh).max() * np.abs(yh).max() * n ** 0.5
    if ref is not None:
        assert abs(got - ref) <= 1e-13 * bound
    assert abs(got - float(np.dot(xh, yh))) <= 1e-13 * bound
    return got


def test_noalloc_dot_matches_handle_dot_on_two_calls():
    s = inputs.coupled_box_3d(ne=13, nfields=2)
    rng = np.random.default_rng(21)
    with mfs.Solver(s, max_levels=3, coarse_max=100) as lib:
        for _ in range(2):
            _check(lib, s.ndofs, rng)


def test_noalloc_dot_full_partial_count_then_smaller_call():
    """n = 1,373,125 fills all 608 reduction blocks (n >= 608 * 2048) and is
    not a multiple of the chunk; a call on a much smaller vector afterwards
    reads only the partials it wrote itself."""
    rng = np.random.default_rng(5)
    n_big = 1_373_125
    assert n_big >= 608 * 2048 and n_big % 2048
    for n in (n_big, n_big, 5_000 + 37, 777):
        xh, yh = rng.standard_normal(n), rng.standard_normal(n)
        x, y = torch.from_numpy(xh).cuda(), torch.from_numpy(yh).cuda()
        got = mfs.dot_noalloc(x, y)
        bound = np.abs(xh).max() * np.abs(yh).max() * n ** 0.5
        assert abs(got - float(np.dot(xh, yh))) <= 1e-13 * bound, n


def test_noalloc_dot_matches_handle_dot_at_full_size():
    """Same sums as mfs_dot on a handle of the 1.37 M-dof 64^3 box."""
    s = inputs.coupled_box_3d(ne=64, nfields=3, seed=1)
    rng = np.random.default_rng(9)
    with mfs.Solver(s, max_levels=5, coarse_max=1000) as lib:
        xh, yh = rng.standard_normal(s.ndofs), rng.standard_normal(s.ndofs)
        x, y = torch.from_numpy(xh).cuda(), torch.from_numpy(yh).cuda()
        for _ in range(2):
            assert mfs.dot_noalloc(x, y) == lib.dot(x, y)


def test_noalloc_dot_rejects_bad_arguments():
    import ctypes as C
    lib = mfs.load()
    x = torch.zeros(8, dtype=torch.float64, device="cuda")
    out = C.c_double()
    # the C entry point itself: n beyond the limit, host vectors, NULL
    rc = lib.mfs_dot_noalloc(C.c_void_p(x.data_ptr()), C.c_void_p(x.data_ptr()), mfs.DOT_NOALLOC_MAX_N + 1,
                             C.byref(out), None)
    assert rc == mfs.ERR_INVALID and b"MAX_N" in lib.mfs_last_error()
    h = np.zeros(8)
    rc = lib.mfs_dot_noalloc(C.c_void_p(h.ctypes.data), C.c_void_p(h.ctypes.data), 8, C.byref(out), None)
    assert rc == mfs.ERR_INVALID and b"device" in lib.mfs_last_error()
    assert lib.mfs_dot_noalloc(None, None, 8, C.byref(out), None) == mfs.ERR_INVALID
    # the binding: a length beyond the vectors, float32, host arrays
    with pytest.raises(ValueError):
        mfs.dot_noalloc(x, x, n=9)
    with pytest.raises(TypeError):
        mfs.dot_noalloc(x.float(), x.float())
    with pytest.raises(mfs.MfsError):
        mfs.dot_noalloc(np.zeros(8), np.zeros(8), n=8)
    assert mfs.dot_noalloc(x, x, n=0) == 0.0


def test_noalloc_dot_refused_on_a_capturing_stream():
    """The call synchronises its stream, so under stream capture it returns
    MFS_ERR_INVALID before launching anything (the capture stays valid)."""
    import ctypes as C
    lib = mfs.load()
    x = torch.ones(4096, dtype=torch.float64, device="cuda")
    assert mfs.dot_noalloc(x, x) == 4096.0  # first call on the device outside capture
    s = torch.cuda.Stream()
    g = torch.cuda.CUDAGraph()
    out = C.c_double()
    with torch.cuda.graph(g, stream=s, capture_error_mode="relaxed"):
        y = x * 2.0
        rc = lib.mfs_dot_noalloc(C.c_void_p(x.data_ptr()), C.c_void_p(x.data_ptr()), 4096, C.byref(out),
                                 C.c_void_p(s.cuda_stream))
    assert rc == mfs.ERR_INVALID and b"captur" in lib.mfs_last_error()
    g.replay()
    torch.cuda.synchronize()
    assert float(y.sum()) == 8192.0
