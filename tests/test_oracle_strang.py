"""Pins of the oracle's Strang step (Sec. 2.1) and whole-step invariants (no GPU)."""
import numpy as np
import scipy.linalg as sla

from oracle import oracle as O
from paper_1506_04651_gb300 import inputs as I


def _mode_tree(J, amps, kx=1, ky=1):
    m = len(amps)
    n = 1 << J
    x = (np.arange(n) + 0.5) / n
    X, Y = np.meshgrid(x, x, indexing="xy")
    phi = (np.cos(np.pi * kx * X) * np.cos(np.pi * ky * Y)).ravel()
    T = O.Tree(2, J, m, jmin=1)
    T.set_full(np.outer(amps, phi))
    return T, phi


def test_strang_second_order_on_linear_reaction():
    """f = K u with K not commuting with diag(D): per cosine mode the exact
    semi-discrete solution is expm((lam_h diag(D) + K) t) a.  Strang's error
    under dt halving must fall by ~4."""
    J = 4
    K = np.array([[-2.0, 3.0], [1.0, -4.0]])
    D = np.array([5e-3, 3e-2])
    a0 = np.array([1.0, 0.5])
    md = O.make_model("linear", K=K)
    h = 1.0 / (1 << J)
    lam_h = -4 / h ** 2 * 2 * np.sin(np.pi * h / 2) ** 2
    tend = 0.4
    exact = sla.expm((lam_h * np.diag(D) + K) * tend) @ a0
    errs = []
    for nsteps in (4, 8, 16):
        T, phi = _mode_tree(J, a0)
        dt = tend / nsteps
        for _ in range(nsteps):
            assert T.strang(md, D, dt, 0.0, 1e-11, 1e-11, 1e-11) == 0
        keys, vals = T.leaves()
        # the solution stays in the mode: read its amplitude from any cell
        r = int(np.argmax(np.abs(phi)))
        j, k = O.key_decode(2, int(keys[0]))
        amp = np.array([T.value(J, [0, 0], i) for i in range(2)]) / phi[0]
        errs.append(np.max(np.abs(amp - exact)))
        del r, j, k
    assert 3.4 < errs[0] / errs[1] < 4.6 and 3.4 < errs[1] / errs[2] < 4.6


def test_diffusion_conserves_mass_on_adaptive_tree():
    for d, J in ((2, 7), (3, 5)):
        T = O.Tree(d, J, 3, jmin=2)
        T.set_full(I.bz_cross_2d(J, 2) if d == 2 else I.bz_sphere_3d(J, 3))
        assert T.adapt(1e-3) == 0
        m0 = T.mass()
        rc, st = T.diffuse(I.BZ_D, 1e-3, 1e-6)
        assert rc == 0 and st["naccept"] >= 3
        np.testing.assert_allclose(T.mass(), m0, rtol=1e-13)


def test_bz_strang_steps_keep_invariants():
    # J = 8 resolves the w = 0.02 front; on coarser grids the linear (non-monotone)
    # third-order prediction overshoots the steep profile and values can change sign
    J = 8
    md = O.make_model("bz")
    T = O.Tree(2, J, 3, jmin=2)
    T.set_full(I.bz_cross_2d(J, 2))
    assert T.adapt(1e-3) == 0
    for _ in range(3):
        assert T.strang(md, I.BZ_D, 1e-3, 1e-3) == 0
        assert T.is_graded()
        keys, vals = T.leaves()
        assert np.all(np.isfinite(vals)) and np.all(vals > -1e-6)
    rc, st, cx = T.react(md, 5e-4, want_complexity=True)
    assert rc == 0 and cx.min() == 7  # App. A minimum complexity
