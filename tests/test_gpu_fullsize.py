"""Parity at the benchmark's full sizes: the initial grid and one Strang step
of the J = 10 2D workload (1024^2 finest, ~10% leaves) and of the J = 7 3D
workload (128^3 finest), through the C-ABI in the configuration bench.py
times, against the oracle on every leaf.  Grids must be identical and values
agree to 1e-9 relative L-infinity per species."""
import numpy as np
import pytest

from oracle import oracle as O
from paper_1506_04651_gb300 import inputs as I

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def mr():
    import __graft_entry__ as g
    g.build()
    from paper_1506_04651_gb300 import mr as M
    return M


def rel_linf(a, b):
    return max(np.max(np.abs(a[i] - b[i])) / np.max(np.abs(b[i])) for i in range(len(b)))


@pytest.mark.parametrize("d,J,eta,gen", [
    (2, 10, 1e-3, lambda J: I.bz_cross_2d(J, 2, **I.CROSS_J10)),
    (3, 7, 1e-2, lambda J: I.bz_sphere_3d(J, 3)),
])
def test_full_size_build_and_step(mr, d, J, eta, gen):
    import torch
    md = O.make_model("bz")
    u0 = gen(J)
    T = O.Tree(d, J, 3, jmin=2)
    T.set_full(u0)
    assert T.adapt(eta) == 0
    ctx = mr.Context(mr.problem(d, J), stream=torch.cuda.current_stream())
    ctx.build(torch.from_numpy(u0).cuda(), eta)
    k_o, v_o = T.leaves()
    k_g, v_g = ctx.leaves()
    assert np.array_equal(k_o, k_g) and np.array_equal(v_o, v_g)
    assert T.strang(md, I.BZ_D, 1e-3, eta) == 0
    ctx.strang(1e-3, eta)
    k_o, v_o = T.leaves()
    k_g, v_g = ctx.leaves()
    assert np.array_equal(k_o, k_g)
    assert rel_linf(v_g, v_o) <= 1e-9
    st = ctx.stats()
    assert st["leaves"] == len(k_o) and st["irregular_rows"] > 0
    np.testing.assert_allclose(ctx.mass(), T.mass(), rtol=1e-11)
