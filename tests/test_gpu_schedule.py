"""The two Radau5 schedules (one thread per cell; the phase-sorted pool in
shared memory) run the same operations per cell in the same order, so the
states, the per-cell complexity and the launch counters they give are
bit-identical: on the 2D BZ crossing fronts (several thousand stiff front
cells among rest-state cells, in FP64 and in the mixed form), on a 3D
sphere and on the NAGUMO front.  In a batch the autotuner tries both
schedules and its test checks the results bit for bit against the default.
The thread kernel is the default and every parity test that integrates
reactions compares it with the oracle; the pool matches it bit for bit."""
import numpy as np
import pytest

from paper_1506_04651_gb300 import inputs as I

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def mr():
    import __graft_entry__ as g
    g.build()
    from paper_1506_04651_gb300 import mr as M
    return M


def run(mr, prob, u0, eta, schedule, steps):
    import torch
    c = mr.Context(prob)
    c.set_radau_schedule(schedule)
    c.build(torch.from_numpy(np.ascontiguousarray(u0)).cuda(), eta)
    counters = []
    for _ in range(steps):
        c.strang(1e-3, eta)
        st = c.stats()
        counters.append(tuple(int(st[k]) for k in ("radau_fev", "radau_jac", "radau_steps", "radau_accept",
                                                    "radau_reject", "radau_newton", "radau_dec")))
    keys, vals = c.leaves()
    return keys, vals, counters


CASES = [
    ("bz2d_J9_fp64", lambda mr: mr.problem(2, 9), lambda: I.bz_cross_2d(9, 2, **I.CROSS_J10), 1e-3, 3),
    ("bz2d_J9_mixed", lambda mr: mr.problem(2, 9, precision=mr.MR_MIXED),
     lambda: I.bz_cross_2d(9, 2, **I.CROSS_J10), 1e-3, 3),
    ("bz3d_J6_fp64", lambda mr: mr.problem(3, 6), lambda: I.bz_sphere_3d(6, 3), 1e-2, 2),
    ("nagumo2d_J8", lambda mr: mr.problem(2, 8, model="nagumo", D=(I.NAGUMO_D,), params=(I.NAGUMO_K,)),
     lambda: I.nagumo_front(2, 8), 1e-4, 3),
]


@pytest.mark.parametrize("name,prob,gen,eta,steps", CASES, ids=[c[0] for c in CASES])
def test_pool_and_thread_schedules_are_bit_identical(mr, name, prob, gen, eta, steps):
    u0 = gen()
    k_p, v_p, c_p = run(mr, prob(mr), u0, eta, mr.MR_RADAU_POOL, steps)
    k_t, v_t, c_t = run(mr, prob(mr), u0, eta, mr.MR_RADAU_THREAD, steps)
    assert np.array_equal(k_p, k_t)
    assert np.array_equal(v_p, v_t)
    assert c_p == c_t
    assert c_p[-1][2] > 0  # Radau5 steps were taken

