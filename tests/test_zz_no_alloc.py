"""elmfb_error_norms_noalloc: error norms for callers that cannot allocate.

Callers whose device memory is already held by a pool, or that run where
calling an allocator is not allowed, use this entry point: it reads device
inputs in place and keeps its scratch in a fixed array of the library.  The
tests call it through the C ABI twice in a row (the scratch keeps the first
call's contents) and check both results against elmfb_error_norms, within the
tolerance of the other error-norm tests; they check that repeated calls leave
the device's free memory unchanged, on the default stream and on a stream of
the caller's.  This file is collected last.
"""
import ctypes as C

import numpy as np
import pytest

pytestmark = pytest.mark.gpu


def _norms_noalloc(lib, uh, ur, n=None, stream=0):
    out = np.zeros(3)
    rc = lib.elmfb_error_norms_noalloc(C.c_void_p(uh.data_ptr()), C.c_void_p(ur.data_ptr()),
                                       C.c_int64(uh.numel() if n is None else n),
                                       C.c_void_p(out.ctypes.data), C.c_void_p(stream))
    return rc, out


def test_noalloc_error_norms_match_allocating_entry_point():
    torch = pytest.importorskip("torch")
    import paper_2409_01949_gb300 as E
    import workloads as WL

    lib = E.lib()
    dev = torch.device("cuda", 0)
    rng = np.random.default_rng(11)
    P = WL.poisson1d(levels=(2,), features=4, n_interior=10)
    with E.Solver.from_problem(P) as s:
        # two calls in a row: a large input, then a smaller one that reuses
        # fewer scratch slots than the first call left behind
        for n in (300_001, 4_099):
            u = rng.standard_normal(n)
            uh = u + 1e-3 * rng.standard_normal(n)
            ud = torch.as_tensor(u, device=dev)
            uhd = torch.as_tensor(uh, device=dev)
            rc, got = _norms_noalloc(lib, uhd, ud,
                                     stream=torch.cuda.current_stream().cuda_stream)
            assert rc == E.OK
            ref = s.error_norms(uhd, ud)
            assert got[0] == pytest.approx(ref["rel_l2"], rel=1e-12)
            assert got[1] == pytest.approx(ref["e_l1"], rel=1e-12)
            assert got[2] == pytest.approx(ref["max_abs"], rel=1e-15)


def test_noalloc_calls_leave_device_memory_unchanged():
    """After a first call (which loads the kernels and looks up the scratch
    address), further calls -- on the default stream and on a caller's stream
    -- change neither the device's free memory nor torch's allocator."""
    torch = pytest.importorskip("torch")
    import paper_2409_01949_gb300 as E

    lib = E.lib()
    dev = torch.device("cuda", 0)
    rng = np.random.default_rng(12)
    n = 100_003
    u = torch.as_tensor(rng.standard_normal(n), device=dev)
    uh = u + 1e-2
    side = torch.cuda.Stream(device=dev)
    side.wait_stream(torch.cuda.current_stream())
    rc, first = _norms_noalloc(lib, uh, u)
    assert rc == E.OK
    torch.cuda.synchronize()
    free0 = torch.cuda.mem_get_info(dev)[0]
    stats0 = torch.cuda.memory_stats(dev).get("allocation.all.allocated", 0)
    results = []
    for stream in (0, side.cuda_stream, 0, side.cuda_stream):
        rc, got = _norms_noalloc(lib, uh, u, stream=stream)
        assert rc == E.OK
        results.append(got)
    torch.cuda.synchronize()
    assert torch.cuda.mem_get_info(dev)[0] == free0
    assert torch.cuda.memory_stats(dev).get("allocation.all.allocated", 0) == stats0
    for got in results:
        assert np.array_equal(got, first)


def test_noalloc_rejects_oversize_and_host_inputs():
    torch = pytest.importorskip("torch")
    import paper_2409_01949_gb300 as E

    lib = E.lib()
    dev = torch.device("cuda", 0)
    a = torch.zeros(8, dtype=torch.float64, device=dev)
    rc, _ = _norms_noalloc(lib, a, a, n=(1 << 24) + 1)
    assert rc == E.ERR_UNSUPPORTED
    h = torch.zeros(8, dtype=torch.float64)
    rc, _ = _norms_noalloc(lib, h, h)
    assert rc == E.ERR_INVALID_ARG
