"""Pins of the oracle's reaction models and Radau5 (no GPU).

Each check compares the oracle with something other than itself: the paper's
printed right-hand side, closed forms (Pade stability function, matrix
exponentials), finite differences, convergence orders, fixed points.
"""
import json
import os

import numpy as np
import pytest
import scipy.linalg as sla

from oracle import oracle as O
from paper_1506_04651_gb300 import inputs as I

GOLD = json.load(open(os.path.join(os.path.dirname(__file__), "golden", "paper_values.json")))


def test_bz_rhs_matches_printed_form():
    """Sec. 1 item II prints f with q = 0.02, 1/mu = 1e5, 1/eps = 1e2, f = 1.6."""
    g = GOLD["bz_constants"]
    md = O.make_model("bz", params=(1 / g["inv_eps"], 1 / g["inv_mu"], g["f"], g["q_printed"]))
    rng = np.random.default_rng(3)
    for _ in range(20):
        u1, u2, u3 = rng.uniform(0, 1, 3)
        want = [1e5 * (-0.02 * u1 - u2 * u1 + 1.6 * u3),
                1e2 * (u2 - u2 ** 2 - u1 * (u2 - 0.02)),
                u2 - u3]
        np.testing.assert_allclose(O.model_f(md, [u1, u2, u3]), want, rtol=1e-13, atol=1e-9)


@pytest.mark.parametrize("kind", ["bz", "nagumo"])
def test_jacobian_matches_finite_differences(kind):
    md = O.make_model(kind)
    rng = np.random.default_rng(4)
    for _ in range(10):
        y = rng.uniform(0.05, 0.9, md.m)
        J = O.model_jac(md, y)
        Jfd = np.zeros_like(J)
        for j in range(md.m):
            e = np.zeros(md.m)
            e[j] = 1e-6 * max(1.0, abs(y[j]))
            Jfd[:, j] = (O.model_f(md, y + e) - O.model_f(md, y - e)) / (2 * e[j])
        np.testing.assert_allclose(J, Jfd, rtol=1e-7, atol=1e-6 * np.abs(J).max())


def test_bz_rest_state_is_fixed_point_and_stays_fixed():
    md = O.make_model("bz")
    b = I.bz_rest_state(1.6, 2e-3)
    y0 = np.array([1.6 * b / (2e-3 + b), b, b])
    assert np.max(np.abs(O.model_f(md, y0))) < 1e-9
    y, rc, st = O.radau5(md, y0, 5e-4)
    assert rc == 0
    np.testing.assert_allclose(y, y0, rtol=1e-12)
    # App. A: one sub-step, one Newton iteration, Jacobian = 3 evaluations -> 7
    assert st["nfev"] + 3 * st["njac"] == GOLD["radau5_min_complexity"]["value"]


def test_radau_iia_tableau_from_collocation_conditions():
    """A from sum_j a_ij c_j^(k-1) = c_i^k / k (k = 1..3), nodes = zeros of the Radau
    polynomial; eigen-structure of A^{-1} and the T-transformation."""
    rc = O.radau_constants()
    c = np.roots([10.0, -8.0, 1.0])  # (4 -+ sqrt 6)/10: zeros of 10 x^2 - 8 x + 1
    c = np.sort(np.append(c, 1.0))
    np.testing.assert_allclose(rc["c"], c, rtol=1e-15)
    V = np.array([[cj ** k for cj in c] for k in range(3)])
    A = np.array([np.linalg.solve(V, [ci ** (k + 1) / (k + 1) for k in range(3)]) for ci in c])
    np.testing.assert_allclose(rc["A"], A, rtol=1e-13, atol=1e-15)
    ev = np.linalg.eigvals(np.linalg.inv(A))
    real = ev[np.abs(ev.imag) < 1e-12].real[0]
    cplx = ev[ev.imag > 1e-12][0]
    np.testing.assert_allclose(rc["gam"], real, rtol=1e-13)
    np.testing.assert_allclose(rc["alp"], cplx.real, rtol=1e-13)
    np.testing.assert_allclose(rc["bet"], cplx.imag, rtol=1e-13)
    Lam = rc["Tinv"] @ np.linalg.inv(A) @ rc["T"]
    want = np.array([[real, 0, 0], [0, cplx.real, -cplx.imag], [0, cplx.imag, cplx.real]])
    np.testing.assert_allclose(Lam, want, atol=1e-12)
    # embedded weights: order-3 quadrature on (0, c1, c2, c3) with weight 1/gam at 0
    nodes = np.append(0.0, c)
    wts = np.append(1.0 / real, rc["bhat"])
    for k in range(3):
        assert abs(wts @ nodes ** k - 1.0 / (k + 1)) < 1e-14


@pytest.mark.parametrize("hl", [-0.3, -3.0, -266.7, -1e4, 0.5])
def test_fixed_step_equals_pade_23(hl):
    """Radau IIA (s=3): R(z) = (1 + 2z/5 + z^2/20)/(1 - 3z/5 + 3z^2/20 - z^3/60)."""
    md = O.make_model("linear", K=[[hl]])
    z = hl
    R = (1 + 2 * z / 5 + z * z / 20) / (1 - 3 * z / 5 + 3 * z * z / 20 - z ** 3 / 60)
    y, rc, _ = O.radau5(md, [1.0], 1.0, 1e-10, 1e-10, hfix=1.0)
    assert rc == 0
    assert abs(y[0] - R) <= 1e-14 * max(1.0, abs(R))


def test_fixed_step_order_five():
    """u' = u^2 (1 - u), u(0) = 1/2 (NAGUMO with k = 1).  Its exact solution satisfies
    G(u) = ln(u/(1-u)) - 1/u = G(1/2) + t; halving h divides the error by ~2^5."""
    md = O.make_model("nagumo", params=(1.0,))
    G = lambda u: np.log(u / (1 - u)) - 1 / u
    target = G(0.5) + 1.0
    u = 0.6
    for _ in range(60):
        u -= (G(u) - target) / (1 / u + 1 / (1 - u) + 1 / u ** 2)
    e = []
    for n in (4, 8, 16):
        y, rc, _ = O.radau5(md, [0.5], 1.0, 1e-10, 1e-10, hfix=1.0 / n)
        assert rc == 0
        e.append(abs(y[0] - u))
    assert e[0] / e[1] > 24 and e[1] / e[2] > 24


@pytest.mark.parametrize("lam", [-1.0, -100.0])
def test_adaptive_matches_exponential(lam):
    md = O.make_model("linear", K=[[lam]])
    y, rc, st = O.radau5(md, [1.0], 0.05, 1e-6, 1e-6)
    assert rc == 0
    assert abs(y[0] - np.exp(lam * 0.05)) < 1e-6


def test_adaptive_very_stiff_decays():
    md = O.make_model("linear", K=[[-1e5]])
    y, rc, st = O.radau5(md, [1.0], 1.0, 1e-6, 1e-6)
    assert rc == 0 and abs(y[0]) < 1e-8
    assert st["nstep"] < 60  # L-stability: no step-size collapse after the transient


def test_stiff_linear_system_vs_expm():
    rng = np.random.default_rng(7)
    m = 5
    lam = -np.array([1.0, 10.0, 1e3, 1e5, 1e6])
    V = rng.standard_normal((m, m)) + 3 * np.eye(m)
    K = V @ np.diag(lam) @ np.linalg.inv(V)
    y0 = rng.uniform(0.5, 1.5, m)
    md = O.make_model("linear", K=K)
    for tol in (1e-6, 1e-9):
        y, rc, _ = O.radau5(md, y0, 5e-4, tol, tol)
        exact = sla.expm(K * 5e-4) @ y0
        assert rc == 0
        assert np.max(np.abs(y - exact)) < 50 * tol * max(1.0, np.abs(exact).max())


def test_bz_tolerance_proportionality():
    """Error against a rtol=1e-13 run shrinks with the tolerance (BZ, dt/2 = 5e-4).
    Cells whose first step covers dt/2 at loose tolerances keep one step, so the
    bound is checked per tolerance decade rather than as strict proportionality."""
    md = O.make_model("bz")
    u = I.bz_cross_2d(5, 2)
    rng = np.random.default_rng(1)
    cells = rng.choice(u.shape[1], 40, replace=False)
    worst = np.zeros(4)
    for cidx in cells:
        y0 = u[:, cidx]
        ref, rc, _ = O.radau5(md, y0, 5e-4, 1e-13, 1e-13)
        assert rc == 0
        for q, tol in enumerate((1e-5, 1e-7, 1e-9, 1e-11)):
            y, rc, _ = O.radau5(md, y0, 5e-4, tol, tol)
            assert rc == 0
            worst[q] = max(worst[q], np.max(np.abs(y - ref) / (1e-3 + np.abs(ref))))
    assert np.all(worst < np.array([1e-3, 1e-4, 1e-6, 1e-8]))
    assert worst[3] < worst[0] / 100


def test_bz_jacobian_eigenvalues_reach_order_1e5():
    """Sec. 1 footnote: along the BZ limit cycle Jacobian eigenvalues reach ~1e5."""
    md = O.make_model("bz")
    y = np.array([0.01, 0.8, 0.8])
    big = 0.0
    for _ in range(200):
        big = max(big, np.max(np.abs(np.linalg.eigvals(O.model_jac(md, y)))))
        y, rc, _ = O.radau5(md, y, 5e-3, 1e-8, 1e-8)
        assert rc == 0
    order = GOLD["bz_jacobian_eigenvalue_order"]["order"]
    assert order / 10 <= big <= order * 10


def test_singular_newton_matrix_halves_the_step_and_recovers():
    """y' = k y with k = gam / tend: on the first attempt (h = tend) the
    filtering matrix gam/h - k of the error estimate is exactly zero, so the
    factorisation fails; the step is halved and the integration goes on to
    the exact solution e^(k tend) within its tolerance."""
    gam = O.radau_constants()["gam"]
    tend = 1.0
    k = gam / tend
    md = O.make_model("linear", K=[[k]])
    y, rc, st = O.radau5(md, [1.0], tend, rtol=1e-8, atol=1e-8)
    assert rc == 0
    assert abs(y[0] - np.exp(k * tend)) <= 1e-5 * np.exp(k * tend)
    assert st["status"] == 0 and st["naccept"] > 0


def test_six_singular_matrices_in_a_row_are_reported():
    """K = diag(gam/tend * 2^q), q = 0..5: every halving of h makes the next
    diagonal entry of gam/h - K exactly zero, so the sixth consecutive
    singular factorisation ends the integration with MR_ERADAU_SINGULAR."""
    gam = O.radau_constants()["gam"]
    tend = 1.0
    K = np.diag([(gam / tend) * 2.0 ** q for q in range(6)])
    md = O.make_model("linear", K=K)
    _, rc, st = O.radau5(md, np.ones(6), tend)
    assert rc == -12
    assert st["ndec"] == 6 and st["nstep"] == 0
