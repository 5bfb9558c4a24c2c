"""GPU parity of the synthetic 21-species membrane model (the STROKE-case
stand-in: warp-per-cell team Radau5 with a forward-difference Jacobian, and
ROCK4 in species windows of 16), through the C-ABI, against the oracle on
identical seeded inputs.

Tolerance.  Both sides form the Jacobian by forward differences with
increments delta ~ 1e-8 |y|; the CUDA and host libraries' log and exp (and
the GPU's fused multiply-adds) differ in the last bit, and the difference
quotient magnifies that by 1 / delta, so the two Jacobians agree to about
1e-8 relative, not 1e-15.  The Jacobian only steers the simplified Newton
iteration, whose stopping rule accepts an iterate once its estimated error
is below fnewt (atol_t + rtol_t |y|) per component (rtol = atol = 1e-6:
rtol_t = atol_t = 0.1 rtol^(2/3) = 1e-5, fnewt = sqrt(rtol_t) = 3.2e-3).  Two
correct implementations whose Jacobians differ may stop on iterates that
differ by up to that amount, 3.2e-8 (1 + |y|) per component and step, and
the tests bound the per-component difference of one reaction half step by
four times that, 1.3e-7 (1 + |y|), in every cell whose work (right-hand
sides, Jacobians counted as 21 each) equals the oracle's.  Where a stopping
or step-size decision fell the other way (measured: 3 to 7 cells of
thousands, work differing by a few right-hand sides) the two step sequences
differ and the bound is the step tolerance itself, atol + rtol |y|; such
cells must stay under 1%.  Adaptations are bit-identical; species with D = 0 are untouched
by the diffusion; a diffusing species in the second window (species 16..20)
is diffused as the oracle does; the mixed form stays within 1e-5 relative L1
of the FP64 oracle; the bench's full-size 2D J = 9 step agrees on every leaf."""
import numpy as np
import pytest

from oracle import oracle as O
from paper_1506_04651_gb300 import inputs as I
from tests import gridcmp as G

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def mr():
    import __graft_entry__ as g
    g.build()
    from paper_1506_04651_gb300 import mr as M
    return M


def rel_linf(a, b):
    return max(np.max(np.abs(a[i] - b[i])) / max(np.max(np.abs(b[i])), 1e-300) for i in range(len(b)))


def within_newton_bound(a, b, steps=1):
    """|a - b| <= 4 fnewt rtol_t (1 + |b|) per component and step (see above)."""
    return bool(np.all(np.abs(a - b) <= steps * 4 * 3.2e-8 * (1.0 + np.abs(b))))


def rel_l1(a, b):
    return max(np.sum(np.abs(a[i] - b[i])) / max(np.sum(np.abs(b[i])), 1e-300) for i in range(len(b)))


def pair(mr, d, J, eta, D=I.IONIC_D, precision=0, r0=0.2, w=0.03):
    u0 = I.ionic_core(d, J, r0=r0, w=w)
    T = O.Tree(d, J, 21, jmin=2)
    T.set_full(u0)
    assert T.adapt(eta) == 0
    c = mr.Context(mr.problem(d, J, model="ionic", D=D, precision=precision))
    c.build(u0, eta)
    k_o, v_o = T.leaves()
    k_g, v_g = c.leaves()
    assert np.array_equal(k_o, k_g) and np.array_equal(v_o, v_g)
    return T, c


@pytest.mark.parametrize("d,J", [(2, 6), (3, 4)])
def test_react_matches_oracle(mr, d, J):
    T, c = pair(mr, d, J, 1e-3)
    rc, st, cx_o = T.react(O.make_model("ionic"), 5e-4, want_complexity=True)
    assert rc == 0
    c.react(5e-4)
    s = c.stats()
    assert s["radau_jac"] > 0 and s["radau_newton"] > 0
    _, v_o = T.leaves()
    _, v_g = c.leaves()
    cx_g = c.complexity()
    assert cx_g.min() >= 1 + 21  # at least f(y0) and one numerical Jacobian
    same = cx_g == cx_o
    assert np.mean(same) >= 0.99
    assert within_newton_bound(v_g[:, same], v_o[:, same])
    assert np.all(np.abs(v_g - v_o) <= 1e-6 * (1.0 + np.abs(v_o)))


def test_diffusion_windows(mr):
    """Species 16..20 have D = 0 in the model, so the second window is
    skipped; giving S (species 20) a coefficient runs it, against the
    oracle's diffusion."""
    D = list(I.IONIC_D)
    D[20] = 5e-3
    T, c = pair(mr, 2, 6, 1e-3, D=D)
    before = c.leaves()[1]
    assert T.diffuse(D, 1e-3)[0] == 0
    c.diffuse(1e-3)
    _, v_o = T.leaves()
    _, v_g = c.leaves()
    assert rel_linf(v_g, v_o) <= 1e-9
    for i in range(21):
        if D[i] == 0.0:
            assert np.array_equal(v_g[i], before[i])
    assert c.stats()["rock_kernel_launches"] >= 2


@pytest.mark.parametrize("d,J,steps", [(2, 6, 3), (3, 4, 2)])
def test_strang_matches_oracle(mr, d, J, steps):
    T, c = pair(mr, d, J, 1e-3)
    md = O.make_model("ionic")
    for q in range(steps):
        assert T.strang(md, I.IONIC_D, 1e-3, 1e-3) == 0
        c.strang(1e-3, 1e-3)
        k_o, v_o = T.leaves()
        k_g, v_g = c.leaves()
        assert np.array_equal(k_o, k_g)
        assert within_newton_bound(v_g, v_o, steps=2 * (q + 1))  # two reaction half steps per step


def test_mixed_form(mr):
    d, J = 2, 6
    T, c = pair(mr, d, J, 1e-3, precision=mr.MR_MIXED)
    md = O.make_model("ionic")
    for _ in range(3):
        assert T.strang(md, I.IONIC_D, 1e-3, 1e-3) == 0
        c.strang(1e-3, 1e-3)
    k_o, v_o = T.leaves()
    k_g, v_g = c.leaves()
    # compared on the finest grid by injection (the mixed form may adapt
    # differently where a detail lies within FP32 noise of its threshold);
    # every species with a non-zero integral
    A, B = G.finest(k_g, v_g, d, J), G.finest(k_o, v_o, d, J)
    checked = 0
    for i in range(21):
        den = np.sum(np.abs(B[i]))
        if den > 0:
            assert np.sum(np.abs(A[i] - B[i])) / den <= 1e-5, i
            checked += 1
    assert checked >= 20


def test_full_size_step(mr):
    """The bench's 2D J = 9 workload: the initial grid and one Strang step
    against the oracle on every leaf.  Grids identical; every component
    within the step tolerance atol + rtol |y| of each half step, and 99% of
    the leaves within the Newton bound (see above) of the two half steps;
    the five linear invariants' domain integrals as the oracle's to 1e-10."""
    import os
    import torch
    J, eta = 9, 1e-3
    u0 = I.ionic_core(2, J, 7)
    T = O.Tree(2, J, 21, jmin=2)
    T.set_full(u0)
    assert T.adapt(eta) == 0
    c = mr.Context(mr.problem(2, J, model="ionic", D=I.IONIC_D), stream=torch.cuda.current_stream())
    c.build(torch.from_numpy(u0).cuda(), eta)
    k_o, v_o = T.leaves()
    k_g, v_g = c.leaves()
    assert np.array_equal(k_o, k_g) and np.array_equal(v_o, v_g)
    O.set_threads(os.cpu_count() or 1)
    try:
        assert T.strang(O.make_model("ionic"), I.IONIC_D, 1e-3, eta) == 0
    finally:
        O.set_threads(1)
    c.strang(1e-3, eta)
    k_o, v_o = T.leaves()
    k_g, v_g = c.leaves()
    assert np.array_equal(k_o, k_g)
    diff = np.abs(v_g - v_o)
    assert np.all(diff <= 2 * 1e-6 * (1.0 + np.abs(v_o)))
    ok = np.all(diff <= 2 * 4 * 3.2e-8 * (1.0 + np.abs(v_o)), axis=0)
    assert np.mean(ok) >= 0.99
    np.testing.assert_allclose(c.mass(), T.mass(), rtol=1e-10, atol=1e-14)
