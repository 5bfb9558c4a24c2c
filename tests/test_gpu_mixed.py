"""Mixed-precision form (MR_MIXED): Radau5 factorises and solves its Newton
systems in FP32 while residuals, error estimates, step control and the state
stay FP64.  Its result is compared with the FP64 oracle at the final time,
relative L1 over the finest grid <= 1e-5 (the bound the benchmark metric
states); the grids are compared through piecewise-constant injection so that a
leaf whose refinement decision flipped at the threshold still counts."""
import numpy as np
import pytest

from oracle import oracle as O
from paper_1506_04651_gb300 import inputs as I

pytestmark = pytest.mark.gpu


def finest(keys, vals, d, J):
    n = 1 << J
    out = np.zeros((vals.shape[0],) + (n,) * d)
    for r, key in enumerate(keys):
        j, k = O.key_decode(d, int(key))
        b = 1 << (J - j)
        sl = tuple(slice(k[a] * b, (k[a] + 1) * b) for a in reversed(range(d)))
        for i in range(vals.shape[0]):
            out[(i,) + sl] = vals[i, r]
    return out.reshape(vals.shape[0], -1)


def rel_l1(a, b):
    return max(np.sum(np.abs(a[i] - b[i])) / np.sum(np.abs(b[i])) for i in range(len(b)))


@pytest.fixture(scope="module")
def mr():
    import __graft_entry__ as g
    g.build()
    from paper_1506_04651_gb300 import mr as M
    return M


def test_mixed_react_against_fp64_oracle(mr):
    md = O.make_model("bz")
    J = 9
    T = O.Tree(2, J, 3, jmin=2)
    T.set_full(I.bz_cross_2d(J, 2))
    T.adapt(1e-3)
    keys, vals = T.leaves()
    ctx = mr.Context(mr.problem(2, J, precision=mr.MR_MIXED))
    ctx.set_leaves(keys, np.ascontiguousarray(vals))
    assert T.react(md, 5e-4)[0] == 0
    ctx.react(5e-4)
    _, v_o = T.leaves()
    _, v_g = ctx.leaves()
    assert rel_l1(v_g, v_o) <= 1e-7
    assert np.max(np.abs(v_g - v_o) / (1e-6 + np.abs(v_o))) < 1e-4


def test_mixed_strang_steps_against_fp64_oracle(mr):
    md = O.make_model("bz")
    J, eta, nsteps = 8, 1e-3, 10
    u0 = I.bz_cross_2d(J, 2)
    T = O.Tree(2, J, 3, jmin=2)
    T.set_full(u0)
    T.adapt(eta)
    ctx = mr.Context(mr.problem(2, J, precision=mr.MR_MIXED))
    ctx.build(u0, eta)
    for _ in range(nsteps):
        assert T.strang(md, I.BZ_D, 1e-3, eta) == 0
        ctx.strang(1e-3, eta)
    k_o, v_o = T.leaves()
    k_g, v_g = ctx.leaves()
    err = rel_l1(finest(k_g, v_g, 2, J), finest(k_o, v_o, 2, J))
    assert err <= 1e-5, err


def test_fp32_details_option_against_fp64_oracle(mr):
    """The mixed form with FP32 MR details (MR_MIXED_F32_DETAILS): ten steps of
    the 2D J = 8 crossing fronts stay within 1e-5 (relative L1 over the
    finest grid) of the FP64 oracle, and its adapted grid differs from the
    FP64 path's in few leaves (only details within FP32 rounding of their
    threshold can be tagged differently)."""
    md = O.make_model("bz")
    J, eta, nsteps = 8, 1e-3, 10
    u0 = I.bz_cross_2d(J, 2)
    T = O.Tree(2, J, 3, jmin=2)
    T.set_full(u0)
    T.adapt(eta)
    c32 = mr.Context(mr.problem(2, J, precision=mr.MR_MIXED_F32_DETAILS))
    c64 = mr.Context(mr.problem(2, J, precision=mr.MR_FP64))
    c32.build(u0, eta)
    c64.build(u0, eta)
    for _ in range(nsteps):
        assert T.strang(md, I.BZ_D, 1e-3, eta) == 0
        c32.strang(1e-3, eta)
        c64.strang(1e-3, eta)
    k_o, v_o = T.leaves()
    k_g, v_g = c32.leaves()
    k_f, _ = c64.leaves()
    assert np.array_equal(k_f, k_o)
    err = rel_l1(finest(k_g, v_g, 2, J), finest(k_o, v_o, 2, J))
    assert err <= 1e-5, err
    assert len(np.setxor1d(k_g, k_o)) <= 0.01 * len(k_o)
