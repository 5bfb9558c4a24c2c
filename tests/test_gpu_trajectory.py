"""Whole trajectories against the oracle at the configured step counts.

* 2D BZ, finest level J = 10 (1024^2), eta = 1e-3, two crossing fronts (the
  default bench workload): 100 Strang steps, dt = 1e-3.
* 3D BZ, J = 7 (128^3), eta = 1e-2, spherical front: 50 Strang steps, in the
  FP64 and the mixed form side by side.

FP64 form: the adapted grid equals the oracle's after every step (details
are summed in the oracle's order, so equal values give equal grids); the
relative L-inf error is at most 1e-9 after the first step and the relative L1
error over the finest grid at most 1e-6 at the final time.

Mixed form: relative L1 over the finest grid at most 1e-5 against the FP64
oracle at the final time (its grids may differ from the oracle's where a
detail lies within FP32 noise of its threshold, so the comparison injects
both leaf sets onto the finest grid).

The oracle runs its threaded form on every host core (bit-identical to its
serial loops: tests/test_oracle_threads.py).
"""
import os

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


def host_cores():
    try:
        return len(os.sched_getaffinity(0))
    except AttributeError:
        return os.cpu_count() or 1


def trajectory(mr, d, J, eta, u0, nsteps, precisions):
    """Steps the oracle and one GPU context per precision in lockstep; returns
    per-precision records of the grids and errors."""
    import torch
    md = O.make_model("bz")
    T = O.Tree(d, J, 3, jmin=2)
    T.set_full(u0)
    assert T.adapt(eta) == 0
    ctxs = {}
    for p in precisions:
        c = mr.Context(mr.problem(d, J, precision=p), stream=torch.cuda.current_stream())
        c.build(torch.from_numpy(u0).cuda(), eta)
        ctxs[p] = c
    rec = {p: {"grid_diff_steps": [], "err_step1": None} for p in precisions}
    O.set_threads(host_cores())
    try:
        for s in range(nsteps):
            assert T.strang(md, I.BZ_D, 1e-3, eta) == 0, s
            for p, c in ctxs.items():
                c.strang(1e-3, eta)
            k_o, v_o = T.leaves()
            for p, c in ctxs.items():
                k_g, v_g = c.leaves()
                same = np.array_equal(k_o, k_g)
                if not same:
                    rec[p]["grid_diff_steps"].append(s)
                if s == 0 and same:
                    rec[p]["err_step1"] = G.rel_linf(v_g, v_o)
                if s == nsteps - 1:
                    rec[p]["rel_l1_final"] = G.rel_l1_finest(k_g, v_g, k_o, v_o, d, J)
                    rec[p]["leaves"] = (len(k_g), len(k_o))
    finally:
        O.set_threads(1)
        for c in ctxs.values():
            c.close()
    return rec


def test_2d_J10_headline_workload_100_steps(mr):
    J, eta = 10, 1e-3
    u0 = I.bz_cross_2d(J, 2, **I.CROSS_J10)
    rec = trajectory(mr, 2, J, eta, u0, 100, [mr.MR_FP64])[mr.MR_FP64]
    assert rec["grid_diff_steps"] == [], rec
    assert rec["err_step1"] <= 1e-9, rec
    assert rec["rel_l1_final"] <= 1e-6, rec


def test_3d_J7_sphere_50_steps_fp64_and_mixed(mr):
    J, eta = 7, 1e-2
    u0 = I.bz_sphere_3d(J, 3)
    rec = trajectory(mr, 3, J, eta, u0, 50, [mr.MR_FP64, mr.MR_MIXED])
    f64, mix = rec[mr.MR_FP64], rec[mr.MR_MIXED]
    assert f64["grid_diff_steps"] == [], f64
    assert f64["err_step1"] <= 1e-9, f64
    assert f64["rel_l1_final"] <= 1e-6, f64
    assert mix["rel_l1_final"] <= 1e-5, mix
