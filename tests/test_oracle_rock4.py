"""Pins of the oracle's ROCK4-type diffusion integrator (no GPU).

The polynomials are checked against the properties that define them
(Abdulle's construction, cited by the paper for ROCK4): order conditions,
stability on [-l_s, 0], orthogonality for the weight w^2/sqrt(1-x^2), the
embedded estimate being O(z^4); the integrator against the exact decay of a
cosine mode of the Neumann heat equation and its fourth-order convergence.
"""
import json
import math
import os

import numpy as np
import pytest

from oracle import oracle as O

GOLD = json.load(open(os.path.join(os.path.dirname(__file__), "golden", "paper_values.json")))
S_LIST = list(range(5, 31)) + [40, 60, 100, 152]


def _stages_taylor(c, K=6):
    """Taylor coefficients (z^0..z^K) of P_n and R = w P_n from the recurrence."""
    n = len(c["mu"]) - 1
    P_prev, P = np.zeros(K + 1), np.zeros(K + 1)
    P[0] = 1.0
    for j in range(1, n + 1):
        zP = np.concatenate([[0.0], P[:-1]])
        P_new = c["mu"][j] * P + c["kap"][j] * zP + (c["nu"][j] * P_prev if j > 1 else 0.0)
        P_prev, P = P, P_new
    R = np.convolve(np.concatenate([c["w"], np.zeros(K + 1)]), P)[: K + 1]
    return P, R


def _eval_R(c, z):
    n = len(c["mu"]) - 1
    p_prev, p = np.zeros_like(z), np.ones_like(z)
    pmax = 1.0
    for j in range(1, n + 1):
        p_new = c["mu"][j] * p + c["kap"][j] * z * p + (c["nu"][j] * p_prev if j > 1 else 0.0)
        p_prev, p = p, p_new
        pmax = max(pmax, np.max(np.abs(p)))
    w = c["w"]
    return (w[0] + z * (w[1] + z * (w[2] + z * (w[3] + z * w[4])))) * p, p, pmax


@pytest.mark.parametrize("s", S_LIST)
def test_order_conditions(s):
    c = O.rock4_coeffs(s)
    _, R = _stages_taylor(c)
    for k in range(5):
        assert abs(R[k] - 1.0 / math.factorial(k)) < 1e-10 / math.factorial(k), (s, k, R[k])
    assert abs(R[5] - 1.0 / 120) > 1e-6  # order exactly four


@pytest.mark.parametrize("s", S_LIST)
def test_stability_on_interval_and_internal_stages(s):
    c = O.rock4_coeffs(s)
    ell = c["ell"]
    assert abs(ell - (0.336 * s * s - 2.7)) < 1e-12
    z = -ell * (1 - np.cos(np.linspace(0, np.pi, 40001))) / 2
    R, P, pmax = _eval_R(c, z)
    assert np.max(np.abs(R)) <= 1.0 + 1e-12
    assert np.max(np.abs(R[z < -2.0])) < 0.8  # damped away from the origin
    assert pmax <= 1.0 + 1e-10  # every recurrence stage stays bounded


@pytest.mark.parametrize("s", [5, 9, 20, 60])
def test_orthogonality_for_the_weight(s):
    """P_j orthogonal on [-1,1] w.r.t. w(x)^2/sqrt(1-x^2), x = 1 + 2 z / l_s."""
    c = O.rock4_coeffs(s)
    n, ell = len(c["mu"]) - 1, c["ell"]
    M = 3 * n + 50
    x = np.cos((2 * np.arange(M) + 1) * np.pi / (2 * M))
    z = ell * (x - 1) / 2
    w = np.polyval(c["xc"][::-1], x - 1)
    assert np.all(w > 0)  # the quartic has no real zero on [-1,1]
    Ps = [np.ones(M)]
    p_prev, p = np.zeros(M), np.ones(M)
    for j in range(1, n + 1):
        p_new = c["mu"][j] * p + c["kap"][j] * z * p + (c["nu"][j] * p_prev if j > 1 else 0.0)
        p_prev, p = p, p_new
        Ps.append(p)
    G = np.array([[np.sum(w * w * a * b) for b in Ps] for a in Ps])
    off = G - np.diag(np.diag(G))
    assert np.max(np.abs(off)) < 1e-11 * np.max(np.abs(np.diag(G)))
    # finishing quartic in z agrees with the quartic in x - 1
    np.testing.assert_allclose(c["w"], c["xc"] * (2 / ell) ** np.arange(5), rtol=1e-14)


@pytest.mark.parametrize("s", [5, 8, 20, 100])
def test_embedded_estimate_is_order_four(s):
    c = O.rock4_coeffs(s)
    w = c["w"]
    a, b1, b2, d = c["errc"]
    h1 = np.array([w[1], w[2], w[3], w[4], 0, 0])
    h2 = np.array([w[2], w[3], w[4], 0, 0, 0])
    ww = np.array([*w, 0])
    zw = np.array([0, *w])
    E = a * np.eye(6)[0] + b1 * h1 + b2 * h2 + ww + d * zw
    assert np.max(np.abs(E[:4])) < 1e-13
    assert abs(E[4]) > 1e-5


def test_stage_count_choice():
    for rd in (0.1, 5.7, 5.71, 30.0, 400.0):
        s, ell, over = O.rock4_choose(rd)
        assert ell >= rd and not over
        if s > 5:
            assert O.rock4_ell(s - 1) < rd
    s, ell, over = O.rock4_choose(1e5)
    assert over and s == 152


def _uniform_tree(J, m=1, d=2):
    T = O.Tree(d, J, m, jmin=1)
    T.set_full(np.zeros((m, 1 << (d * J))))
    return T


def _mode(J, kx, ky):
    n = 1 << J
    x = (np.arange(n) + 0.5) / n
    X, Y = np.meshgrid(x, x, indexing="xy")
    return (np.cos(np.pi * kx * X) * np.cos(np.pi * ky * Y)).ravel()


def _leaf_order(T, J):
    keys, _ = T.leaves()
    idx = []
    for k in keys:
        j, kk = O.key_decode(2, int(k))
        idx.append(kk[0] + (kk[1] << J))
    return np.array(idx)


def test_heat_cosine_mode_semidiscrete_and_pde_decay():
    J, kx, ky, D, t = 5, 2, 1, 1e-2, 0.05
    T = _uniform_tree(J)
    u0 = _mode(J, kx, ky)
    T.set_full(u0[None, :])
    rc, st = T.diffuse([D], t, tol=1e-9)
    assert rc == 0
    keys, vals = T.leaves()
    u = np.zeros_like(u0)
    u[_leaf_order(T, J)] = vals[0]
    h = 1.0 / (1 << J)
    lam_h = -4 / h ** 2 * (np.sin(np.pi * kx * h / 2) ** 2 + np.sin(np.pi * ky * h / 2) ** 2)
    assert np.max(np.abs(u - np.exp(D * lam_h * t) * u0)) < 1e-7
    lam = -np.pi ** 2 * (kx ** 2 + ky ** 2)
    assert np.max(np.abs(u - np.exp(D * lam * t) * u0)) < 2e-3  # O(h^2) space error


def test_fixed_step_fourth_order():
    J, D = 4, 1e-2
    T = _uniform_tree(J)
    rp, col, val, rho = T.operator()
    u0 = _mode(J, 1, 1)[_leaf_order(T, J)]
    h = 1.0 / (1 << J)
    lam_h = -4 / h ** 2 * 2 * np.sin(np.pi * h / 2) ** 2
    exact = np.exp(D * lam_h * 1.0) * u0
    errs = []
    for n in (4, 8, 16):
        assert O.rock4_choose(D * rho / n)[0] == 5
        y, rc, st = O.rock4_linear(rp, col, val, D, rho, u0, 1.0, hfix=1.0 / n)
        assert rc == 0
        errs.append(np.max(np.abs(y - exact)))
    assert 13 < errs[0] / errs[1] < 19 and 13 < errs[1] / errs[2] < 19


def test_gershgorin_matches_paper_eigenvalue_scale():
    """Sec. 1 footnote: at h = 1/1024 the largest negative diffusion eigenvalues are
    about -2e4 (BZ, D = 2.5e-3)."""
    g = GOLD["bz_diffusion_eigenvalue_h1024"]
    T = _uniform_tree(10)
    _, _, _, rho = T.operator()
    D = GOLD["bz_constants"]["D"][0]
    assert abs(-D * rho - g["value"]) <= g["rel_tol"] * abs(g["value"])
