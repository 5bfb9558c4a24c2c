"""GPU parity of the 16-species stiff mass-action network (team Radau5 kernel,
16-species ROCK4), through the C-ABI, against the oracle on identical seeded
inputs.

Tolerances as for BZ: one reaction / diffusion / Strang step agrees to 1e-9
relative L-infinity per species (relative to the species' largest value);
adaptations are bit-identical (same detail arithmetic); conserved moieties of
the network (left null space of the stoichiometric matrix, and the total
amount) keep their integrals to rounding; the mixed form (FP32 Newton
factorisations) stays within 1e-5 relative L1 of the FP64 oracle.  At the
full 3D J = 8 size, sampled cells are integrated one by one by the oracle's
Radau5 and compared with the GPU's result for the same cells."""
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


NET = I.network_instance(5)


def rel_linf(a, b):
    return max(np.max(np.abs(a[i] - b[i])) / max(np.max(np.abs(b[i])), 1e-300) for i in range(len(b)))


def rel_l1(a, b):
    return max(np.sum(np.abs(a[i] - b[i])) / max(np.sum(np.abs(b[i])), 1e-300) for i in range(len(b)))


def model():
    sp, kf, kb, _ = NET
    return O.make_model("network", m=16, params=(sp, kf, kb))


def context(mr, d, J, precision=0):
    sp, kf, kb, D = NET
    c = mr.Context(mr.problem(d, J, model="network", D=D, precision=precision))
    c.set_network(sp, kf, kb)
    return c


def pair(mr, d, J, eta, precision=0):
    u0 = I.network_bumps(d, J, 5)
    T = O.Tree(d, J, 16, jmin=2)
    T.set_full(u0)
    assert T.adapt(eta) == 0
    c = context(mr, d, J, precision)
    c.build(u0, eta)
    k_o, v_o = T.leaves()
    k_g, v_g = c.leaves()
    assert np.array_equal(k_o, k_g) and np.array_equal(v_o, v_g)
    return T, c


@pytest.mark.parametrize("d,J", [(2, 6), (3, 4)])
def test_react_matches_oracle(mr, d, J):
    T, c = pair(mr, d, J, 1e-3)
    rc, st = T.react(model(), 5e-4)
    assert rc == 0
    c.react(5e-4)
    s = c.stats()
    assert s["radau_fev"] > 0 and s["radau_newton"] > 0
    _, v_o = T.leaves()
    _, v_g = c.leaves()
    assert rel_linf(v_g, v_o) <= 1e-9


@pytest.mark.parametrize("d,J", [(2, 6), (3, 4)])
def test_diffuse_matches_oracle_and_conserves_mass(mr, d, J):
    T, c = pair(mr, d, J, 1e-3)
    m0 = c.mass()
    rc, _ = T.diffuse(NET[3], 1e-3)
    assert rc == 0
    c.diffuse(1e-3)
    _, v_o = T.leaves()
    _, v_g = c.leaves()
    assert rel_linf(v_g, v_o) <= 1e-9
    np.testing.assert_allclose(c.mass(), m0, rtol=1e-12)


def test_strang_steps_match_oracle_and_keep_moieties(mr):
    sp = NET[0]
    S = np.zeros((16, len(sp)))
    for r, (a, b, cc, dd) in enumerate(sp):
        S[a, r] -= 1
        S[b, r] -= 1
        S[cc, r] += 1
        S[dd, r] += 1
    _, sv, Vt = np.linalg.svd(S.T)
    Y = np.vstack([Vt[int((sv > 1e-10).sum()):], np.ones(16)])
    T, c = pair(mr, 2, 6, 1e-3)
    m0 = Y @ c.mass()
    md = model()
    for step in range(3):
        assert T.strang(md, NET[3], 1e-3, 1e-3) == 0
        c.strang(1e-3, 1e-3)
        k_o, v_o = T.leaves()
        k_g, v_g = c.leaves()
        assert np.array_equal(k_o, k_g), step  # FP64: the adapted grids are identical
        assert rel_linf(v_g, v_o) <= 1e-8 * (step + 1)
    np.testing.assert_allclose(Y @ c.mass(), m0, rtol=0, atol=1e-11 * np.abs(m0).max())


def test_mixed_form_within_1e5_of_fp64_oracle(mr):
    T, c = pair(mr, 2, 6, 1e-3, precision=1)
    md = model()
    for _ in range(3):
        assert T.strang(md, NET[3], 1e-3, 1e-3) == 0
        c.strang(1e-3, 1e-3)
    k_o, v_o = T.leaves()
    k_g, v_g = c.leaves()
    assert np.array_equal(k_o, k_g)
    assert rel_l1(v_g, v_o) <= 1e-5


def test_invalid_networks_rejected(mr):
    sp, kf, kb, D = NET
    c = mr.Context(mr.problem(2, 5, model="network", D=D))
    bad = sp.copy()
    bad[0, 1] = bad[0, 0]  # repeated species
    for args in ((bad, kf, kb), (np.full_like(sp, 16), kf, kb), (sp, -kf, kb)):
        with pytest.raises(mr.MRError) as e:
            c.set_network(*args)
        assert e.value.code == -1
    c.build(I.network_bumps(2, 5, 5), 1e-3)
    with pytest.raises(mr.MRError) as e:  # no reactions set yet
        c.react(1e-4)
    assert e.value.code == -4
    bz = mr.Context(mr.problem(2, 5))
    with pytest.raises(mr.MRError):
        bz.set_network(sp, kf, kb)


def test_full_size_3d_J8_sampled_cells(mr):
    """The 3D J = 8 network configuration (256^3 finest, eta = 1e-3): the GPU
    builds the grid and integrates one reaction half step; sampled leaves
    are integrated from the same values by the oracle's Radau5, cell by cell."""
    import torch
    d, J, eta = 3, 8, 1e-3
    sp, kf, kb, D = NET
    u0 = I.network_bumps(d, J, 5)
    c = mr.Context(mr.problem(d, J, model="network", D=D), stream=torch.cuda.current_stream())
    c.set_network(sp, kf, kb)
    c.build(torch.from_numpy(u0).cuda(), eta)
    del u0
    keys, before = c.leaves()
    n = len(keys)
    assert 0 < n < (1 << (d * J))
    c.react(5e-4)
    _, after = c.leaves()
    rng = np.random.default_rng(7)
    md = model()
    for r in rng.choice(n, 48, replace=False):
        y, rc, _ = O.radau5(md, before[:, r], 5e-4)
        assert rc == 0
        assert np.max(np.abs(after[:, r] - y)) <= 1e-9 * np.max(np.abs(y))


def test_3d_trajectory_fp64_and_mixed_against_oracle(mr):
    """Ten Strang steps of the 3D J = 4 network workload (48x48 Newton
    systems, rates up to 1e6): in FP64 the grids equal the oracle's after
    every step and the values stay within 1e-8 per step; the conserved
    moieties hold to 1e-11; the mixed form ends within 1e-5 (relative L1 on
    the finest grid) of the FP64 oracle."""
    from tests import gridcmp as G
    sp = NET[0]
    S = np.zeros((16, len(sp)))
    for r, (a, b, cc, dd) in enumerate(sp):
        S[a, r] -= 1
        S[b, r] -= 1
        S[cc, r] += 1
        S[dd, r] += 1
    _, sv, Vt = np.linalg.svd(S.T)
    Y = np.vstack([Vt[int((sv > 1e-10).sum()):], np.ones(16)])
    T, c = pair(mr, 3, 4, 1e-3)
    _, cm = pair(mr, 3, 4, 1e-3, precision=mr.MR_MIXED)
    m0 = Y @ c.mass()
    md = model()
    import os
    O.set_threads(len(os.sched_getaffinity(0)))  # the threaded oracle equals its serial loops
    try:
        for step in range(10):
            assert T.strang(md, NET[3], 1e-3, 1e-3) == 0
            c.strang(1e-3, 1e-3)
            cm.strang(1e-3, 1e-3)
            k_o, v_o = T.leaves()
            k_g, v_g = c.leaves()
            assert np.array_equal(k_o, k_g), step
            assert rel_linf(v_g, v_o) <= 1e-8 * (step + 1), step
    finally:
        O.set_threads(1)
    np.testing.assert_allclose(Y @ c.mass(), m0, rtol=0, atol=1e-11 * np.abs(m0).max())
    k_m, v_m = cm.leaves()
    assert G.rel_l1_finest(k_m, v_m, k_o, v_o, 3, 4) <= 1e-5
