"""The threaded form of the oracle (timed CPU baseline only) computes exactly
what the serial loops compute: leaves of a reaction sub-step and rows of an
operator application are independent, and counters and first errors are
combined in a fixed order."""
import numpy as np

from oracle import oracle as O
from paper_1506_04651_gb300 import inputs as I


def run(threads):
    O.set_threads(threads)
    try:
        T = O.Tree(2, 7, 3, jmin=2)
        T.set_full(I.bz_cross_2d(7, 2, w=0.01, amp=0.1))
        assert T.adapt(1e-3) == 0
        md = O.make_model("bz")
        rc, st, cx = T.react(md, 5e-4, want_complexity=True)
        assert rc == 0
        rc, rs = T.diffuse(I.BZ_D, 1e-3)
        assert rc == 0
        assert T.strang(md, I.BZ_D, 1e-3, 1e-3) == 0
        return T.leaves(), st, cx, rs
    finally:
        O.set_threads(1)


def test_threads_match_serial_bit_for_bit():
    (k1, v1), s1, c1, r1 = run(1)
    (k4, v4), s4, c4, r4 = run(4)
    assert np.array_equal(k1, k4) and np.array_equal(v1, v4)
    assert s1 == s4 and r1 == r4
    assert np.array_equal(c1, c4)


def test_operator_rows_threaded_match_serial():
    """Operator rows built by the parallel-for (chunks concatenated in leaf
    order) equal the serial loop's, in 2D and 3D adaptive trees."""
    for d, J, eta in ((2, 7, 1e-3), (3, 5, 1e-2)):
        u0 = I.bz_cross_2d(J, 2, w=0.01, amp=0.1) if d == 2 else I.bz_sphere_3d(J, 3)
        T = O.Tree(d, J, 3, jmin=2)
        T.set_full(u0)
        assert T.adapt(eta) == 0
        out = []
        for th in (1, 3):
            O.set_threads(th)
            try:
                out.append(T.operator())
            finally:
                O.set_threads(1)
        (rp1, c1, w1, r1), (rp3, c3, w3, r3) = out
        assert np.array_equal(rp1, rp3) and np.array_equal(c1, c3) and np.array_equal(w1, w3)
        assert r1 == r3
        assert len(rp1) == T.num_leaves() + 1 and rp1[-1] == len(c1)
