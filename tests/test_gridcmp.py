"""The finest-grid injection used by the GPU parity tests, checked against
the oracle's own key decoding on adaptive trees (2D and 3D)."""
import numpy as np
import pytest

from oracle import oracle as O
from paper_1506_04651_gb300 import inputs as I
from tests import gridcmp as G


def slow_finest(keys, vals, d, J):
    n = 1 << J
    out = np.zeros((vals.shape[0],) + (n,) * d)
    for r, key in enumerate(keys):
        j, k = O.key_decode(d, int(key))
        b = 1 << (J - j)
        sl = tuple(slice(k[a] * b, (k[a] + 1) * b) for a in reversed(range(d)))
        for i in range(vals.shape[0]):
            out[(i,) + sl] = vals[i, r]
    return out.reshape(vals.shape[0], -1)


@pytest.mark.parametrize("d,J,eta", [(2, 7, 1e-3), (3, 5, 1e-2)])
def test_finest_injection_matches_key_decoding(d, J, eta):
    u0 = I.bz_cross_2d(J, 2) if d == 2 else I.bz_sphere_3d(J, 3)
    T = O.Tree(d, J, 3, jmin=2)
    T.set_full(u0)
    assert T.adapt(eta) == 0
    keys, vals = T.leaves()
    assert len(np.unique(G.key_levels(keys))) > 1  # a real adaptive tree
    fast = G.finest(keys, vals, d, J)
    assert np.array_equal(fast, slow_finest(keys, vals, d, J))
    # injection keeps the integral: finest mean = volume-weighted leaf sum
    vol = np.ldexp(1.0, -d * G.key_levels(keys))
    np.testing.assert_allclose(fast.mean(axis=1), vals @ vol, rtol=1e-13)
    assert G.rel_l1_finest(keys, vals, keys, vals, d, J) == 0.0
