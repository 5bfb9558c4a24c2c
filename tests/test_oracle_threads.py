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
