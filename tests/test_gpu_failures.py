"""Failure statuses reach the caller.  Every failure is made on the host (a
leaf value set to NaN through mr_set_leaves); no kernel is made to fault.

* adaptation: a non-finite detail makes mr_adapt / strang_step return
  MR_ESTATE;
* reaction: a cell whose state is not finite is reported as MR_ENONFINITE at
  once (the other cells are integrated exactly as without it);
* diffusion: a non-finite error norm gives MR_ENONFINITE;
* the 16-lane team kernel (network model) reports MR_ENONFINITE likewise."""
import numpy as np
import pytest

from paper_1506_04651_gb300 import inputs as I

pytestmark = pytest.mark.gpu

ESTATE, ENONFINITE = -4, -30


@pytest.fixture(scope="module")
def mr():
    import __graft_entry__ as g
    g.build()
    from paper_1506_04651_gb300 import mr as M
    return M


def poisoned(mr, J=7, which=1234, species=1, model="bz"):
    if model == "network":
        sp, kf, kb, D = I.network_instance(5)
        c = mr.Context(mr.problem(2, 5, model="network", D=D))
        c.set_network(sp, kf, kb)
        c.build(I.network_bumps(2, 5, 5), 1e-3)
    else:
        c = mr.Context(mr.problem(2, J))
        c.build(I.bz_cross_2d(J, 2, w=0.01, amp=0.1), 1e-3)
    keys, vals = c.leaves()
    clean = vals.copy()
    which = which % len(keys)
    vals[species, which] = np.nan
    c.set_leaves(keys, np.ascontiguousarray(vals))
    return c, keys, clean, which


def test_nan_leaf_makes_the_step_report_estate(mr):
    c, _, _, _ = poisoned(mr)
    with pytest.raises(mr.MRError) as e:
        c.strang(1e-3, 1e-3)
    assert e.value.code == ESTATE
    c2, _, _, _ = poisoned(mr)
    with pytest.raises(mr.MRError) as e:
        c2.adapt(1e-3)
    assert e.value.code == ESTATE


def test_nan_leaf_reaction_reports_nonfinite_and_spares_the_rest(mr):
    c, keys, clean, which = poisoned(mr)
    with pytest.raises(mr.MRError) as e:
        c.react(5e-4)
    assert e.value.code == ENONFINITE
    _, got = c.leaves()
    assert c.complexity()[which] == 1  # stopped before any Newton work
    ref = mr.Context(mr.problem(2, 7))
    ref.set_leaves(keys, np.ascontiguousarray(clean))
    ref.react(5e-4)
    _, want = ref.leaves()
    ok = np.ones(len(keys), dtype=bool)
    ok[which] = False
    assert np.array_equal(got[:, ok], want[:, ok])  # cells are independent
    assert np.isnan(got[1, which])


def test_nan_leaf_diffusion_reports_nonfinite(mr):
    c, _, _, _ = poisoned(mr)
    with pytest.raises(mr.MRError) as e:
        c.diffuse(1e-3)
    assert e.value.code == ENONFINITE


def test_nan_leaf_team_kernel_reports_nonfinite(mr):
    c, _, _, which = poisoned(mr, which=17, species=5, model="network")
    with pytest.raises(mr.MRError) as e:
        c.react(5e-4)
    assert e.value.code == ENONFINITE
    _, got = c.leaves()
    assert np.isnan(got[5, which])
    assert np.all(np.isfinite(np.delete(got, which, axis=1)))
