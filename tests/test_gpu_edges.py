"""Degenerate and boundary cases of the method on the GPU, each against the
oracle on the same inputs: constant data (every detail zero: the grid
coarsens to jmin), a threshold above every detail, no diffusion (D = 0: the
diffusion sub-step is the identity), the smallest trees (J = jmin), the
NAGUMO model in the mixed form, and step arguments that must be rejected."""
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


def both(mr, d, J, u0, eta, D=I.BZ_D, jmin=2, precision=0):
    T = O.Tree(d, J, 3, jmin=jmin)
    T.set_full(u0)
    assert T.adapt(eta) == 0
    c = mr.Context(mr.problem(d, J, D=D, jmin=jmin, precision=precision))
    c.build(u0, eta)
    k_o, v_o = T.leaves()
    k_g, v_g = c.leaves()
    assert np.array_equal(k_o, k_g) and np.array_equal(v_o, v_g)
    return T, c


def step_and_compare(T, c, D, dt=1e-3, eta=1e-3, tol=1e-9):
    md = O.make_model("bz")
    assert T.strang(md, D, dt, eta) == 0
    c.strang(dt, eta)
    k_o, v_o = T.leaves()
    k_g, v_g = c.leaves()
    assert np.array_equal(k_o, k_g)
    assert rel_linf(v_g, v_o) <= tol


@pytest.mark.parametrize("d,J", [(2, 8), (3, 5)])
def test_constant_data_coarsens_to_jmin(mr, d, J):
    u0 = np.stack([np.full(1 << (d * J), v) for v in (0.4, 0.3, 0.2)])
    T, c = both(mr, d, J, u0, 1e-3)
    keys, _ = c.leaves()
    assert len(keys) == 1 << (d * 2)  # every leaf at jmin = 2
    assert np.all((keys >> np.uint64(48)) == 2)
    step_and_compare(T, c, I.BZ_D)


def test_threshold_above_every_detail(mr):
    u0 = I.bz_cross_2d(8, 2, w=0.01, amp=0.1)
    T, c = both(mr, 2, 8, u0, 1e12)
    assert c.num_leaves() == 16
    step_and_compare(T, c, I.BZ_D, eta=1e12)


def test_no_diffusion_is_two_reactions(mr):
    u0 = I.bz_cross_2d(8, 2, w=0.01, amp=0.1)
    D0 = (0.0, 0.0, 0.0)
    T, c = both(mr, 2, 8, u0, 1e-3, D=D0)
    before = c.leaves()[1]
    c.diffuse(1e-3)
    assert np.array_equal(c.leaves()[1], before)  # D = 0: the identity
    step_and_compare(T, c, D0)


@pytest.mark.parametrize("d", [2, 3])
def test_smallest_trees(mr, d):
    J = 2
    u0 = I.bz_sphere_3d(J, 3) if d == 3 else I.bz_front_2d(J, 1)
    T, c = both(mr, d, J, u0, 1e-3, jmin=2)
    assert c.num_leaves() == 1 << (d * J)
    for _ in range(2):
        step_and_compare(T, c, I.BZ_D)


def test_nagumo_mixed_form(mr):
    J, eta = 8, 1e-3
    x = (np.arange(1 << J) + 0.5) / (1 << J)
    u0 = (0.5 * (1 - np.tanh((np.add.outer(0 * x, x) - 0.4) / 0.03))).reshape(1, -1)
    md = O.make_model("nagumo")
    T = O.Tree(2, J, 1, jmin=2)
    T.set_full(u0)
    assert T.adapt(eta) == 0
    c = mr.Context(mr.problem(2, J, model="nagumo", precision=mr.MR_MIXED))
    c.build(u0, eta)
    for _ in range(5):
        assert T.strang(md, (0.1,), 1e-2, eta) == 0
        c.strang(1e-2, eta)
    k_o, v_o = T.leaves()
    k_g, v_g = c.leaves()
    # the mixed form may round a detail to the other side of its threshold,
    # so the two grids are compared on the finest grid by injection
    assert G.rel_l1_finest(k_g, v_g, k_o, v_o, 2, J) <= 1e-5


def test_step_arguments_rejected(mr):
    c = mr.Context(mr.problem(2, 6))
    c.build(I.bz_front_2d(6, 1), 1e-3)
    for args in ((0.0, 1e-3), (-1e-3, 1e-3), (1e-3, -1.0), (float("nan"), 1e-3)):
        with pytest.raises(mr.MRError) as e:
            c.strang(*args)
        assert e.value.code == -1
    with pytest.raises(mr.MRError) as e:
        c.strang(1e-3, 1e-3, rtol=0.0)
    assert e.value.code == -1


def test_capacities_and_empty_inputs_are_reported(mr):
    """Capacity and size errors reach the caller before any data is written:
    a leaf capacity below the finest grid makes mr_build report MR_ENOMEM, a
    short output buffer makes mr_get_leaves report MR_ENOMEM with the count
    it needs, and an empty or non-tiling leaf set is MR_EINVAL."""
    import ctypes as C
    small = mr.Context(mr.problem(2, 6, max_leaves=100))
    with pytest.raises(mr.MRError) as e:
        small.build(I.bz_front_2d(6, 1), 1e-3)
    assert e.value.code == -2
    c = mr.Context(mr.problem(2, 6))
    c.build(I.bz_front_2d(6, 1), 1e-3)
    n = c.num_leaves()
    keys = np.zeros(n, dtype=np.uint64)
    vals = np.zeros((3, n))
    got = C.c_int64()
    rc = mr.lib().mr_get_leaves(c.h, C.c_void_p(keys.ctypes.data), C.c_void_p(vals.ctypes.data), n - 1,
                                C.byref(got), 0)
    assert rc == -2 and got.value == n
    assert not keys.any() and not vals.any()  # nothing written
    with pytest.raises(mr.MRError) as e:
        c.set_leaves(np.zeros(0, dtype=np.uint64), np.zeros((3, 0)))
    assert e.value.code == -1
    k, v = c.leaves()
    with pytest.raises(mr.MRError) as e:  # one leaf missing: the leaves no longer tile the domain
        c.set_leaves(k[:-1].copy(), np.ascontiguousarray(v[:, :-1]))
    assert e.value.code == -1
