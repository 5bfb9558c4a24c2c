"""Pins of the oracle's synthetic 21-species membrane model (IONIC, the
stand-in for the paper's STROKE case: 21 equations, steep sigmoid gates, log
Nernst potentials, Jacobian eigenvalues down to about -1e8 near rest, and a
numerical Jacobian), of its forward-difference Jacobian, and of Radau5 and
the Strang step on it.

* conservation: the reaction keeps c_k + e_k / beta (k = 0..2),
  c_3 + e_3 / beta + Bt B and Cm V - sum_k z_k c_k - 2 Bt B (a dropped or
  mis-signed term of the pump, the transmitter current, the buffer or a
  valence breaks one of them), pointwise and along a Radau5 trajectory;
* Nernst equilibrium: with every ion at its Nernst potential (e_k = c_k
  exp(z_k V)), no pump (E = 0) and no transmitter, every current vanishes;
* the Jacobian's columns against central differences of f along random
  directions (a transposed or misplaced column fails);
* the stiffness the paper reports for its model: at rest the most negative
  eigenvalue lies near -1e8 and none is positive beyond rounding;
* bistability (the front mechanism): a small transmitter pulse decays, a
  larger one switches the cell to the depolarised state;
* Radau5 at rtol = atol = 1e-6 against a run at 1e-10;
* one Strang step of a small tree keeps the domain integrals of the five
  invariants (diffusion keeps each species' integral)."""
import numpy as np
import pytest

from oracle import oracle as O
from paper_1506_04651_gb300 import inputs as I

BETA, CM, BT = 4.0, 3e-9, 0.05
Z = (1.0, 1.0, -1.0, 2.0)


def model():
    return O.make_model("ionic")


def invariants():
    W = []
    for k in range(3):
        w = np.zeros(21)
        w[5 + k] = 1.0
        w[k] = 1.0 / BETA
        W.append(w)
    w = np.zeros(21)
    w[8], w[3], w[19] = 1.0, 1.0 / BETA, BT
    W.append(w)
    w = np.zeros(21)
    w[9] = CM
    w[5:9] = [-z for z in Z]
    w[19] = -2.0 * BT
    W.append(w)
    return np.array(W)


def random_state(rng):
    y = np.empty(21)
    y[0:4] = rng.uniform(0.1, 20.0, 4)
    y[4] = rng.uniform(0.0, 2.0)
    y[5:9] = rng.uniform(1e-5, 20.0, 4)
    y[9] = rng.uniform(-5.0, 1.0)
    y[10:18] = rng.uniform(0.0, 1.0, 8)
    y[18:21] = rng.uniform(0.0, 1.0, 3)
    return y


def test_reaction_keeps_the_invariants():
    md = model()
    rng = np.random.default_rng(3)
    W = invariants()
    for _ in range(50):
        y = random_state(rng)
        f = O.model_f(md, y)
        terms = np.abs(W * f[None, :]).sum(axis=1)
        assert np.all(np.abs(W @ f) <= 1e-12 * np.maximum(terms, 1e-300))


def test_no_current_at_nernst_equilibrium():
    md = model()
    rng = np.random.default_rng(4)
    for _ in range(20):
        y = random_state(rng)
        V = y[9]
        for k in range(4):
            y[k] = y[5 + k] * np.exp(Z[k] * V)
        y[4] = 0.0   # no transmitter
        y[18] = 0.0  # no energy: no pump
        f = O.model_f(md, y)
        # V' = -(sum of currents) / Cm: each current is G (V - E_k) with
        # V - E_k at rounding level
        assert abs(f[9]) <= 1e-6
        assert np.all(np.abs(f[0:3]) <= 1e-12) and np.all(np.abs(f[5:8]) <= 1e-12)
        assert abs(f[3]) <= 1e-12


def test_jacobian_columns_against_central_differences():
    md = model()
    rng = np.random.default_rng(5)
    for y in (np.asarray(I.IONIC_REST), np.asarray(I.IONIC_DEP), random_state(rng)):
        J = O.model_jac(md, y).reshape(21, 21)
        for _ in range(5):
            v = rng.standard_normal(21) * np.maximum(np.abs(y), 1e-3)
            eps = 1e-7
            fd = (O.model_f(md, y + eps * v) - O.model_f(md, y - eps * v)) / (2 * eps)
            scale = np.abs(J).dot(np.abs(v))
            assert np.all(np.abs(J @ v - fd) <= 1e-4 * scale + 1e-9 * scale.max())


def test_stiffness_at_rest():
    md = model()
    J = O.model_jac(md, np.asarray(I.IONIC_REST)).reshape(21, 21)
    ev = np.linalg.eigvals(J)
    assert -2e8 <= ev.real.min() <= -5e7
    assert ev.real.max() <= 1e-3


def test_rest_state_is_at_rest():
    md = model()
    y, rc, st = O.radau5(md, np.asarray(I.IONIC_REST), 1e-3)
    assert rc == 0 and st["nstep"] == 1 and st["nnewton"] <= 2
    assert np.all(np.abs(y - np.asarray(I.IONIC_REST)) <= 1e-6 * np.maximum(np.abs(y), 1.0))


@pytest.mark.parametrize("g0,flips", [(0.05, False), (0.5, True)])
def test_bistable_switch(g0, flips):
    md = model()
    y = np.array(I.IONIC_REST)
    y[4] = g0
    y, rc, _ = O.radau5(md, y, 1.0)
    assert rc == 0
    assert (y[9] > -1.0) == flips  # depolarised near -0.5, rest near -4.55


def test_radau_keeps_invariants_and_matches_tight_run():
    md = model()
    y0 = np.array(I.IONIC_REST)
    y0[4] = 0.5  # switching: the stiff transient of a front cell
    W = invariants()
    y, rc, st = O.radau5(md, y0, 0.01, 1e-6, 1e-6)
    assert rc == 0 and st["nstep"] > 5 and st["njac"] >= 1
    w0, w1 = W @ y0, W @ y
    assert np.all(np.abs(w1 - w0) <= 1e-8 * np.abs(W).dot(np.abs(y0)))
    yt, rc, _ = O.radau5(md, y0, 0.01, 1e-10, 1e-10)
    assert rc == 0
    assert np.all(np.abs(y - yt) <= 1e-4 * np.maximum(np.abs(yt), 1e-2))


def test_strang_keeps_domain_integrals():
    d, J = 2, 4
    u0 = I.ionic_core(d, J, r0=0.25, w=0.05)
    T = O.Tree(d, J, 21, jmin=2)
    T.set_full(u0)
    assert T.adapt(1e-3) == 0
    W = invariants()
    before = W @ T.mass()
    assert T.strang(model(), I.IONIC_D, 1e-3, 1e-3) == 0
    after = W @ T.mass()
    assert np.all(np.abs(after - before) <= 1e-8 * np.abs(W).dot(np.abs(T.mass())))
