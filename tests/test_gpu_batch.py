"""Batched serving (mr_batch_*): instances stepped together give the results
of stepping each instance alone (the joint Radau5 launch integrates every
cell with the same arithmetic: exactly; the joint ROCK4 launch keeps each
instance's step control but sums its error norm in another order: to
rounding), the counters add up, models that cannot share a launch fall back
to per-instance launches, and one instance is checked against the oracle."""
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


def instances(n):
    out = []
    for inst in I.batch_instances(n, master_seed=77):
        inst = dict(inst, J=min(inst["J"], 8))
        u0 = I.bz_front_smooth_2d(inst["J"], inst["seed"] & 0xFFFFFFFF, x0=inst["x0"], f=inst["f"])
        out.append((inst, u0))
    return out


def problem(mr, inst):
    return mr.problem(2, inst["J"], params=(1e-2, 1e-5, inst["f"], 2e-3))


def test_batch_equals_separate_contexts(mr):
    insts = instances(6)
    b = mr.Batch([problem(mr, i) for i, _ in insts], threads=4)
    singles = []
    for k, (inst, u0) in enumerate(insts):
        b[k].build(u0, inst["eta"])
        c = mr.Context(problem(mr, inst))
        c.build(u0, inst["eta"])
        singles.append(c)
    eta = [i["eta"] for i, _ in insts]
    b.run(3, 1e-3, eta)
    st = b.stats()
    assert st["joint_reaction"] == 1 and st["steps"] == 3 and st["react_launches"] == 6
    assert st["joint_diffusion"] == 1 and st["diffuse_launches"] == 3 and st["ms_diffuse_kernel"] > 0
    assert st["radau_fev"] > 0 and st["radau_newton"] > 0 and st["ms_device"] > 0
    updates = 0
    for _ in range(3):
        for c, (inst, _) in zip(singles, insts):
            c.strang(1e-3, inst["eta"])
            updates += c.num_leaves()
    assert st["leaf_updates"] == updates
    for k, c in enumerate(singles):
        kb, vb = b[k].leaves()
        ks, vs = c.leaves()
        assert np.array_equal(kb, ks)
        # error norms summed in another order: the same steps, states equal
        # to a few units of rounding of the stage recurrence
        assert b[k].stats()["rock_steps"] == c.stats()["rock_steps"]
        for i in range(3):
            assert np.max(np.abs(vb[i] - vs[i])) <= 1e-12 * np.max(np.abs(vs[i]))
    b.close()


def test_joint_diffusion_alone(mr):
    """The joint ROCK4 launch on its own (no reaction): each instance's
    diffusion sub-step against the same instance's one-context ROCK4 driver,
    in the FP64 and in the mixed form."""
    for precision, tol in ((0, 1e-12), (mr.MR_MIXED, 1e-12)):
        insts = instances(5)
        probs = [mr.problem(2, i["J"], params=(1e-2, 1e-5, i["f"], 2e-3), precision=precision) for i, _ in insts]
        b = mr.Batch(probs, threads=4)
        singles = []
        for k, (inst, u0) in enumerate(insts):
            b[k].build(u0, inst["eta"])
            c = mr.Context(probs[k])
            c.build(u0, inst["eta"])
            singles.append(c)
        b.diffuse(2e-3)
        st = b.stats()
        assert st["joint_diffusion"] == 1 and st["diffuse_launches"] == 1
        for k, c in enumerate(singles):
            c.diffuse(2e-3)
            assert b[k].stats()["rock_steps"] == c.stats()["rock_steps"]
            kb, vb = b[k].leaves()
            ks, vs = c.leaves()
            assert np.array_equal(kb, ks)
            for i in range(3):
                assert np.max(np.abs(vb[i] - vs[i])) <= tol * np.max(np.abs(vs[i]))
        b.close()


def test_batch_instance_matches_oracle(mr):
    inst, u0 = instances(1)[0]
    b = mr.Batch([problem(mr, inst)])
    b[0].build(u0, inst["eta"])
    T = O.Tree(2, inst["J"], 3, jmin=2)
    T.set_full(u0)
    assert T.adapt(inst["eta"]) == 0
    md = O.make_model("bz", params=(1e-2, 1e-5, inst["f"], 2e-3))
    b.run(1, 1e-3, [inst["eta"]])
    assert T.strang(md, I.BZ_D, 1e-3, inst["eta"]) == 0
    k_o, v_o = T.leaves()
    k_g, v_g = b[0].leaves()
    assert np.array_equal(k_o, k_g)
    for i in range(3):
        assert np.max(np.abs(v_g[i] - v_o[i])) <= 1e-9 * np.max(np.abs(v_o[i]))


def test_mixed_models_fall_back_per_instance(mr):
    inst, u0 = instances(1)[0]
    pn = mr.problem(2, 6, model="nagumo")
    b = mr.Batch([problem(mr, inst), pn])
    b[0].build(u0, inst["eta"])
    x = (np.arange(64) + 0.5) / 64
    un = (0.5 * (1 - np.tanh((np.add.outer(x * 0, x) - 0.5) / 0.05))).reshape(1, -1)
    b[1].build(un, 1e-3)
    cn = mr.Context(pn)
    cn.build(un, 1e-3)
    b.run(2, 1e-3, [inst["eta"], 1e-3])
    assert b.stats()["joint_reaction"] == 0 and b.stats()["joint_diffusion"] == 0
    for _ in range(2):
        cn.strang(1e-3, 1e-3)
    kb, vb = b[1].leaves()
    ks, vs = cn.leaves()
    assert np.array_equal(kb, ks) and np.array_equal(vb, vs)


def test_batch_rejects_bad_arguments(mr):
    inst, u0 = instances(1)[0]
    b = mr.Batch([problem(mr, inst)])
    b[0].build(u0, inst["eta"])
    with pytest.raises(mr.MRError) as e:
        b.run(1, 1e-3, [-1.0])
    assert e.value.code == -1
    with pytest.raises(mr.MRError) as e:
        b.run(1, -1e-3, [1e-3])
    assert e.value.code == -1
    for bad in ((0.0, 1e-6), (float("inf"), 1e-6), (1e-3, 0.0)):
        with pytest.raises(mr.MRError) as e:
            b.diffuse(*bad)
        assert e.value.code == -1


def test_full_batch_config_one_step(mr):
    """The full batched configuration (64 instances, J in {7..10}, seeded f,
    eta, front position): one batched step, the smallest, a median and the
    largest instance checked against the oracle."""
    import torch
    insts = I.batch_instances(64)
    b = mr.Batch([mr.problem(2, i["J"], params=(1e-2, 1e-5, i["f"], 2e-3)) for i in insts])
    u0s = {}
    for k, inst in enumerate(insts):
        u0s[k] = I.bz_front_smooth_2d(inst["J"], inst["seed"] & 0xFFFFFFFF, x0=inst["x0"], f=inst["f"])
        b[k].build(torch.from_numpy(u0s[k]).cuda(), inst["eta"])
    b.run(1, 1e-3, [i["eta"] for i in insts])
    assert b.stats()["joint_reaction"] == 1
    order = sorted(range(64), key=lambda k: (insts[k]["J"], k))
    for k in (order[0], order[32], order[-1]):
        inst = insts[k]
        T = O.Tree(2, inst["J"], 3, jmin=2)
        T.set_full(u0s[k])
        assert T.adapt(inst["eta"]) == 0
        md = O.make_model("bz", params=(1e-2, 1e-5, inst["f"], 2e-3))
        assert T.strang(md, I.BZ_D, 1e-3, inst["eta"]) == 0
        k_o, v_o = T.leaves()
        k_g, v_g = b[k].leaves()
        assert np.array_equal(k_o, k_g)
        for i in range(3):
            assert np.max(np.abs(v_g[i] - v_o[i])) <= 1e-9 * np.max(np.abs(v_o[i]))
    b.close()


def test_autotuner_changes_no_result(mr):
    """The batch's autotuner tries its candidate launch shapes on the first
    launches (joint Radau5: the thread schedule with 128 or 64 threads per
    block, or the pooled schedule, each with the finest levels first or in leaf
    order; joint ROCK4: 2 or 1 blocks per SM).  None of them changes
    a result: after six steps every instance equals, bit for bit, the same
    batch run with the default shapes fixed.  The trial table lists every
    candidate, each tried twice, and one shape chosen per phase."""
    insts = instances(6)
    eta = [i["eta"] for i, _ in insts]
    runs = []
    for tuned in (True, False):
        b = mr.Batch([problem(mr, i) for i, _ in insts], threads=4)
        if not tuned:
            b.set_autotune(False)
        for k, (inst, u0) in enumerate(insts):
            b[k].build(u0, inst["eta"])
        b.run(6, 1e-3, eta)
        runs.append(([b[k].leaves() for k in range(b.n)], b.tuning()))
        b.close()
    (tuned, table), (fixed, table_fixed) = runs
    for (k1, v1), (k2, v2) in zip(tuned, fixed):
        assert np.array_equal(k1, k2) and np.array_equal(v1, v2)
    react = [e for e in table if e["phase"] == "reaction"]
    diff = [e for e in table if e["phase"] == "diffusion"]
    assert len(react) == 6 and len(diff) == 2
    assert all(e["launches"] >= 2 and e["rate"] > 0 for e in react + diff)
    assert sum(e["chosen"] for e in react) == 1 and sum(e["chosen"] for e in diff) == 1
    assert {(e["schedule"], e["block"], e["order"]) for e in react} == {
        ("pool", 128, 1), ("pool", 128, 0), ("thread", 128, 1), ("thread", 64, 1), ("thread", 128, 0),
        ("thread", 64, 0)}
    assert {e["per_sm"] for e in diff} == {1, 2}
    # with the tuner off only the default shapes run
    assert [e["launches"] > 0 for e in table_fixed] == [True] + [False] * 5 + [True, False]
