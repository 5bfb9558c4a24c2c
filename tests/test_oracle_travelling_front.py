"""A pin of the oracle's whole multi-step Strang trajectory (adaptation,
Radau5, ROCK4 on adaptive grids, splitting) against a closed form.

The NAGUMO reaction f(u) = k u^2 (1 - u) (Sec. 1 item I) with diffusion D
has the exact travelling front u = U(x - c t), U(z) = 1 / (1 + exp(lambda z)):
with U' = -lambda U (1 - U) and U'' = lambda^2 U (1 - U) (1 - 2U), the
equation -c U' = D U'' + f(U) reduces to c lambda = D lambda^2 (1 - 2U) + k U
for every U, so lambda^2 = k / (2D) and c = D lambda = sqrt(k D / 2).  Along
the front the integral of f(U) is c, while diffusion keeps the integral of u
(homogeneous Neumann), so the domain integral of u grows by exactly c t as
long as the front's tails stay far from the walls.

Here k = 20, D = 2e-3 (lambda = 70.7, c = 0.1414), a front along y at
x0 = 0.35 on the 2D J = 9 grid (lambda h = 0.14), eta = 1e-4, dt = 2e-3,
100 Strang steps: the integral must grow by c t within 1% (discretisation
errors in space, time and splitting, measured: 0.013%), and u must stay in
[0, 1] up to rounding (no overshoot of the stabilised diffusion at the
level jumps)."""
import numpy as np

from oracle import oracle as O


def test_nagumo_front_moves_at_the_exact_speed():
    J, k, D = 9, 20.0, 2e-3
    lam, c = np.sqrt(k / (2 * D)), np.sqrt(k * D / 2)
    n = 1 << J
    x = (np.arange(n) + 0.5) / n
    x0 = 0.35
    u0 = np.tile(1.0 / (1.0 + np.exp(lam * (x - x0))), (n, 1)).reshape(1, -1)
    T = O.Tree(2, J, 1, jmin=2)
    T.set_full(u0)
    assert T.adapt(1e-4) == 0
    md = O.make_model("nagumo", params=(k,))
    m0 = T.mass()[0]
    dt, steps = 2e-3, 100
    for _ in range(steps):
        assert T.strang(md, (D,), dt, 1e-4) == 0
    grown = T.mass()[0] - m0
    assert abs(grown - c * dt * steps) <= 0.01 * c * dt * steps
    _, v = T.leaves()
    assert v.min() >= -1e-9 and v.max() <= 1.0 + 1e-9


def test_one_dimensional_trees_are_refused():
    import pytest
    with pytest.raises(ValueError):
        O.Tree(1, 8, 1, jmin=2)
