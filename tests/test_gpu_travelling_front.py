"""The GPU path against a closed form: the NAGUMO model's exact travelling
front U(z) = 1 / (1 + exp(lambda z)), lambda^2 = k / (2D), c = sqrt(k D / 2)
(Sec. 1 item I; derivation in tests/test_oracle_travelling_front.py).  The
domain integral of u grows by c t while the front's tails stay away from the
walls: 100 Strang steps of the 2D J = 9 adaptive grid, within 1% of c t, in
the FP64 and the mixed form, with u in [0, 1] up to rounding."""
import numpy as np
import pytest

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def mr():
    import __graft_entry__ as g
    g.build()
    from paper_1506_04651_gb300 import mr as M
    return M


@pytest.mark.parametrize("precision", [0, 1])
def test_front_speed(mr, precision):
    J, k, D = 9, 20.0, 2e-3
    lam, c = np.sqrt(k / (2 * D)), np.sqrt(k * D / 2)
    n = 1 << J
    x = (np.arange(n) + 0.5) / n
    u0 = np.tile(1.0 / (1.0 + np.exp(lam * (x - 0.35))), (n, 1)).reshape(1, -1)
    ctx = mr.Context(mr.problem(2, J, model="nagumo", params=(k,), D=(D,), precision=precision))
    ctx.build(u0, 1e-4)
    m0 = ctx.mass()[0]
    dt, steps = 2e-3, 100
    for _ in range(steps):
        ctx.strang(dt, 1e-4)
    grown = ctx.mass()[0] - m0
    assert abs(grown - c * dt * steps) <= 0.01 * c * dt * steps
    _, v = ctx.leaves()
    assert v.min() >= -1e-6 and v.max() <= 1.0 + 1e-6
