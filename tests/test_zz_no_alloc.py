"""mr_react_radau5_noalloc: reacting a plain array of cells without allocating.

Callers that cannot allocate device memory (another component owns the
device's memory, or the allocator must not be called) integrate their cells
through this entry point; its scratch is a static device array.  Here it is
called through the C-ABI on a copy of a context's leaf values and must give
the same result as react_radau5 on the context, on two calls in a row (the
second call starts from what the shared scratch kept from the first).  This
file is collected last so that a run stopping at the first failure has run
every other test already.
"""
import ctypes as C

import numpy as np
import pytest

pytestmark = pytest.mark.gpu


def _entry(mr):
    f = mr.lib().mr_react_radau5_noalloc
    f.argtypes = [C.c_int, C.POINTER(C.c_double), C.c_int, C.c_void_p, C.c_int64, C.c_int64,
                  C.c_double, C.c_double, C.c_double, C.c_void_p, C.c_void_p]
    f.restype = C.c_int
    return f


def test_noalloc_reaction_matches_react_radau5_on_two_calls():
    import torch

    import __graft_entry__ as g
    g.build()
    from paper_1506_04651_gb300 import inputs as I
    from paper_1506_04651_gb300 import mr

    f = _entry(mr)
    J, dt = 8, 5e-4
    ctx = mr.Context(mr.problem(2, J))
    ctx.build(I.bz_cross_2d(J, 2), 1e-3)
    _, u0 = ctx.leaves()
    n = u0.shape[1]
    ld = n + 37  # a row stride larger than n
    host = np.zeros((3, ld))
    host[:, :n] = u0
    dev = torch.from_numpy(host).cuda()
    cx = torch.zeros(n, dtype=torch.int32, device="cuda")
    params = (C.c_double * 4)(1e-2, 1e-5, 1.6, 2e-3)
    for call in range(2):
        ctx.react(dt, 1e-6, 1e-6)
        rc = f(1, params, 4, dev.data_ptr(), n, ld, dt, 1e-6, 1e-6, cx.data_ptr(), None)
        assert rc == 0, (call, rc)
        torch.cuda.synchronize()
        _, want = ctx.leaves()
        got = dev.cpu().numpy()[:, :n]
        rel = max(np.max(np.abs(got[i] - want[i])) / np.max(np.abs(want[i])) for i in range(3))
        assert rel <= 1e-9, (call, rel)
        assert np.array_equal(cx.cpu().numpy(), ctx.complexity())
        assert np.all(dev.cpu().numpy()[:, n:] == 0.0)  # padding past n untouched
    ctx.close()


def test_noalloc_rejects_sizes_beyond_the_maximum():
    import torch

    from paper_1506_04651_gb300 import mr

    f = _entry(mr)
    params = (C.c_double * 4)(1e-2, 1e-5, 1.6, 2e-3)
    buf = torch.zeros(3, 4, dtype=torch.float64, device="cuda")
    too_many = mr.NOALLOC_MAX_CELLS + 1
    assert f(1, params, 4, buf.data_ptr(), too_many, too_many, 5e-4, 1e-6, 1e-6, None, None) == -1
    assert f(1, params, 4, buf.data_ptr(), 4, 3, 5e-4, 1e-6, 1e-6, None, None) == -1  # ld < n
    assert f(7, params, 4, buf.data_ptr(), 4, 4, 5e-4, 1e-6, 1e-6, None, None) == -1  # unknown model
    assert f(1, params, 4, buf.data_ptr(), 0, 0, 5e-4, 1e-6, 1e-6, None, None) == 0  # nothing to do
