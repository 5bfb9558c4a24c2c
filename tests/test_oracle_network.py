"""Pins of the oracle's synthetic stiff mass-action network (the 16-species
workload; reversible reactions u_a + u_b <-> u_c + u_d with mass-action rates).

* f is pinned by a one-reaction network, whose extent x(t) obeys a Riccati
  equation with a closed-form solution, integrated by the oracle's Radau5;
* the analytic Jacobian against central finite differences;
* conservation: sum_i f_i = 0 (two molecules in, two out) and y^T f = 0 for
  every vector y of the left null space of the stoichiometric matrix
  (conserved moieties), also after a Radau5 integration (Runge-Kutta methods
  keep linear invariants);
* the seeded generator: four distinct species per reaction, rates and
  diffusion coefficients in their stated ranges."""
import numpy as np
import pytest

from oracle import oracle as O
from paper_1506_04651_gb300 import inputs as I


def net16():
    sp, kf, kb, D = I.network_instance(5)
    return O.make_model("network", m=16, params=(sp, kf, kb)), sp, kf, kb, D


def stoich(sp, m):
    S = np.zeros((m, len(sp)))
    for r, (a, b, c, d) in enumerate(sp):
        S[a, r] -= 1
        S[b, r] -= 1
        S[c, r] += 1
        S[d, r] += 1
    return S


def test_generator_ranges():
    sp, kf, kb, D = I.network_instance(5)
    assert sp.shape == (32, 4) and all(len(set(row)) == 4 for row in sp)
    assert sp.min() >= 0 and sp.max() <= 15
    for v in (kf, kb):
        assert v.min() >= 1e-2 and v.max() <= 1e6
        assert np.log10(v).std() > 1.5  # spread over the decades
    assert D.min() >= 1e-4 and D.max() <= 1e-2
    u = I.network_bumps(2, 5, 5)
    assert u.shape == (16, 1024) and u.min() >= 0.1 and u.max() < 0.1 + 4.0


def test_rhs_against_the_rate_law():
    md, sp, kf, kb, _ = net16()
    rng = np.random.default_rng(0)
    y = rng.uniform(0.05, 1.5, 16)
    w = kf * y[sp[:, 0]] * y[sp[:, 1]] - kb * y[sp[:, 2]] * y[sp[:, 3]]
    f = stoich(sp, 16) @ w
    np.testing.assert_allclose(O.model_f(md, y), f, rtol=1e-12, atol=1e-9)


def test_jacobian_against_finite_differences():
    md, *_ = net16()
    rng = np.random.default_rng(1)
    y = rng.uniform(0.05, 1.5, 16)
    J = O.model_jac(md, y)
    h = 1e-6
    Jfd = np.zeros((16, 16))
    for j in range(16):
        e = np.zeros(16)
        e[j] = h
        Jfd[:, j] = (O.model_f(md, y + e) - O.model_f(md, y - e)) / (2 * h)
    scale = np.abs(J).max()
    assert np.abs(J - Jfd).max() <= 1e-7 * scale


def test_conserved_moieties_of_f_and_of_radau5():
    md, sp, *_ = net16()
    S = stoich(sp, 16)
    # left null space: y^T S = 0
    U, sv, Vt = np.linalg.svd(S.T)
    rank = int((sv > 1e-10).sum())
    Y = Vt[rank:]
    assert Y.shape[0] >= 1
    ones = np.ones(16) / 4.0
    assert np.abs(ones @ S).max() < 1e-14  # total amount is one of them
    rng = np.random.default_rng(2)
    y0 = rng.uniform(0.1, 1.0, 16)
    f = O.model_f(md, y0)
    scale = np.abs(f).max()
    assert abs(f.sum()) <= 1e-12 * scale * 16
    assert np.abs(Y @ f).max() <= 1e-12 * scale * 16
    y1, rc, st = O.radau5(md, y0, 5e-4, 1e-6, 1e-6)
    assert rc == 0 and st["naccept"] >= 1
    np.testing.assert_allclose(Y @ y1, Y @ y0, rtol=0, atol=1e-12)
    assert abs(y1.sum() - y0.sum()) <= 1e-12 * y0.sum()


@pytest.mark.parametrize("kf,kb,y0", [
    (3.0, 1.0, (1.0, 0.5, 0.2, 0.1)),
    (50.0, 200.0, (0.3, 0.9, 0.6, 0.4)),
    (1e3, 1e3, (0.2, 0.3, 0.9, 0.7)),    # equal rates: the extent is linear-fractional
])
def test_one_reaction_closed_form(kf, kb, y0):
    """A + B <-> C + D: with the extent x, a = a0 - x, b = b0 - x,
    c = c0 + x, d = d0 + x and x' = kf (a0 - x)(b0 - x) - kb (c0 + x)(d0 + x)
    = al x^2 + be x + ga, solved through the roots x1, x2 of the quadratic:
    (x - x1)/(x - x2) = (x0 - x1)/(x0 - x2) exp(al (x1 - x2) t)  (al != 0),
    x(t) = (ga/be)(exp(be t) - 1)  (al = 0, be != 0)."""
    md = O.make_model("network", m=4, params=(np.array([[0, 1, 2, 3]]), [kf], [kb]))
    a0, b0, c0, d0 = y0
    al = kf - kb
    be = -kf * (a0 + b0) - kb * (c0 + d0)
    ga = kf * a0 * b0 - kb * c0 * d0
    t = 2e-2
    if al != 0.0:
        disc = np.sqrt(be * be - 4 * al * ga)
        x1, x2 = (-be - disc) / (2 * al), (-be + disc) / (2 * al)
        q = (0 - x1) / (0 - x2) * np.exp(al * (x1 - x2) * t)
        x = (x1 - q * x2) / (1 - q)
    else:
        x = (ga / be) * (np.exp(be * t) - 1.0)
    exact = np.array([a0 - x, b0 - x, c0 + x, d0 + x])
    y, rc, _ = O.radau5(md, np.array(y0), t, 1e-11, 1e-11)
    assert rc == 0
    np.testing.assert_allclose(y, exact, rtol=1e-8, atol=1e-10)


def test_strang_steps_conserve_every_moiety_integral():
    """Adaptation (projection based), reaction (pointwise linear invariants)
    and diffusion (each species' integral) all conserve y^T (integral of u)
    for every conserved moiety y; checked over two Strang steps on an
    adaptive 2D tree."""
    md, sp, kf, kb, D = net16()
    S = stoich(sp, 16)
    _, sv, Vt = np.linalg.svd(S.T)
    Y = Vt[int((sv > 1e-10).sum()):]
    Y = np.vstack([Y, np.ones(16)])
    J = 5
    T = O.Tree(2, J, 16, jmin=2)
    T.set_full(I.network_bumps(2, J, 5))
    assert T.adapt(1e-3) == 0
    m0 = Y @ T.mass()
    for _ in range(2):
        assert T.strang(md, D, 1e-3, 1e-3) == 0
    m1 = Y @ T.mass()
    np.testing.assert_allclose(m1, m0, rtol=0, atol=1e-11 * np.abs(m0).max())
