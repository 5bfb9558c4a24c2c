"""Pins of the oracle's multiresolution tree and finite-volume operator (no GPU).

Checks against the paper's printed formulas (key layout, Eq. inter_1d,
threshold law), closed forms (polynomial reproduction, exact averages,
quadratic Laplacian), invariants (grading, conservation, eta = 0 uniform),
and a brute-force re-implementation of one adaptation on tiny trees written
with Python sets in a different formulation (refined-node sets swept by
level) than the oracle's literal tag/refine/coarsen passes.
"""
import itertools
import json
import os

import numpy as np
import pytest

from oracle import oracle as O
from paper_1506_04651_gb300 import inputs as I

GOLD = json.load(open(os.path.join(os.path.dirname(__file__), "golden", "paper_values.json")))


# ---------------------------------------------------------------- keys

def test_key_layout_golden():
    g = GOLD["key_layout"]
    assert O.key(g["d"], g["level"], g["k"]) == int(g["key_hex"], 16)


def test_key_roundtrip_and_order():
    rng = np.random.default_rng(0)
    for d in (2, 3):
        for _ in range(200):
            j = int(rng.integers(0, 16 if d == 2 else 10))
            k = rng.integers(0, 1 << j, d) if j else np.zeros(d, dtype=int)
            key = O.key(d, j, k)
            assert key >> 48 == j
            jj, kk = O.key_decode(d, key)
            assert jj == j and list(kk) == list(k)
    # x digit is the most significant digit of each pair (Fig. 2 text)
    assert O.key(2, 1, [1, 0]) & 3 == 2 and O.key(2, 1, [0, 1]) & 3 == 1


# ---------------------------------------------------------------- helpers

def level_keys(d, j):
    return [O.key(d, j, k[::-1]) for k in itertools.product(range(1 << j), repeat=d)]


def cell_avg_poly(d, J, coef):
    """exact cell averages at level J of sum c_(a) x^a0 y^a1 (z^a2), a_i <= 2"""
    n = 1 << J
    edges = np.arange(n + 1) / n

    def avg1(p):
        lo, hi = edges[:-1], edges[1:]
        return (hi ** (p + 1) - lo ** (p + 1)) / ((p + 1) * (hi - lo))

    out = np.zeros([n] * d)
    for powers, c in coef.items():
        term = np.ones([n] * d)
        for a, p in enumerate(powers):
            shape = [1] * d
            shape[d - 1 - a] = n  # axis order: last axis is x (x fastest in ravel)
            term = term * avg1(p).reshape(shape)
        out += c * term
    return out.ravel()


# ---------------------------------------------------------------- prediction, projection

def test_prediction_golden_1d_example():
    g = GOLD["prediction_1d_example"]
    # coarse level 2 leaves depending on x only; ask for absent level-3 values
    T = O.Tree(2, 3, 1, jmin=2)
    keys = level_keys(2, 2)
    vals = []
    for key in keys:
        _, k = O.key_decode(2, key)
        vals.append({0: 0.5, 1: g["coarse"][0], 2: g["coarse"][1], 3: g["coarse"][2]}[k[0]])
    assert T.set_leaves(np.array(keys, dtype=np.uint64), np.array(vals)) == 0
    # coarse cell kx = 2 has neighbours kx = 1, 3 -> values (1, 2, 4)
    assert abs(T.value(3, [4, 1], 0) - g["fine_even"]) < 1e-15
    assert abs(T.value(3, [5, 1], 0) - g["fine_odd"]) < 1e-15


def test_projection_is_exact_block_average():
    J = 5
    rng = np.random.default_rng(2)
    u = rng.standard_normal((2, 1 << (2 * J)))
    T = O.Tree(2, J, 2, jmin=1)
    T.set_full(u)
    for j in (0, 2, 4):
        b = 1 << (J - j)
        blocks = u.reshape(2, 1 << j, b, 1 << j, b).mean(axis=(2, 4))
        for (ky, kx) in [(0, 0), ((1 << j) - 1, 0), (0, (1 << j) // 2)]:
            for i in range(2):
                assert abs(T.value(j, [kx, ky], i) - blocks[i, ky, kx]) < 1e-14


def _parent_stencil_in_range(d, j, k):
    return all(1 <= (kk >> 1) <= (1 << (j - 1)) - 2 for kk in k)


def test_details_vanish_for_quadratics_interior():
    J = 6
    u = cell_avg_poly(2, J, {(0, 0): 1.0, (1, 0): 0.3, (0, 1): -2.0, (2, 0): 3.0,
                             (1, 1): -1.0, (0, 2): 0.5})
    T = O.Tree(2, J, 1, jmin=1)
    T.set_full(u[None, :])
    keys, delta = T.details()
    n_in = 0
    for key, dl in zip(keys, delta):
        j, k = O.key_decode(2, int(key))
        if j >= 2 and _parent_stencil_in_range(2, j, k):
            assert dl < 1e-13
            n_in += 1
    assert n_in > 1000
    assert np.max(delta) > 1e-6  # boundary nodes of a non-even quadratic do see details


def test_details_vanish_for_even_quadratic_at_mirror_faces():
    J = 6
    u = cell_avg_poly(2, J, {(2, 0): 1.0, (0, 2): 2.0, (0, 0): 1.0})  # even about x=0, y=0
    T = O.Tree(2, J, 1, jmin=1)
    T.set_full(u[None, :])
    keys, delta = T.details()
    for key, dl in zip(keys, delta):
        j, k = O.key_decode(2, int(key))
        if j >= 2 and all((kk >> 1) <= (1 << (j - 1)) - 2 for kk in k):
            assert dl < 1e-13


def test_constant_data_coarsens_to_jmin():
    for d, J in ((2, 5), (3, 3)):
        T = O.Tree(d, J, 2, jmin=2)
        T.set_full(np.full((2, 1 << (d * J)), 0.7))
        assert T.adapt(1e-3) == 0
        keys, vals = T.leaves()
        assert all(int(k) >> 48 == 2 for k in keys) and len(keys) == 1 << (2 * d)
        assert np.allclose(vals, 0.7)


def test_threshold_law_golden():
    g = GOLD["threshold_law"]
    assert abs(g["eps"] * 2.0 ** (g["d"] / 2 * (g["j"] - g["J"])) - g["eps_j"]) < 1e-18


def test_eta_zero_gives_uniform_finest_grid():
    J = 5
    u = I.bz_cross_2d(J, 3)
    T = O.Tree(2, J, 3, jmin=2)
    T.set_full(u)
    assert T.adapt(0.0) == 0
    assert T.num_leaves() == 1 << (2 * J)
    # from the coarsest admissible tree, eta = 0 refines one level per adaptation
    T2 = O.Tree(2, J, 3, jmin=2)
    keys = np.array(level_keys(2, 2), dtype=np.uint64)
    T2.set_leaves(keys, np.ones((3, len(keys))))
    for step in range(J - 2):
        assert T2.adapt(0.0) == 0
        lv = np.array([int(k) >> 48 for k in T2.leaves()[0]])
        assert np.all(lv == 3 + step)


# ---------------------------------------------------------------- brute-force adaptation

def _brute_adapt(d, J, jmin, leaves, eta):
    """Independent restatement of one adaptation with sets of refined nodes."""
    nst = list(itertools.product((-1, 0, 1), repeat=d))
    kids = list(itertools.product((0, 1), repeat=d))
    R_old = set()
    for (j, k) in leaves:
        while j > 0:
            j, k = j - 1, tuple(c >> 1 for c in k)
            R_old.add((j, k))
    m = len(next(iter(leaves.values())))
    val = {}
    for (j, k), v in leaves.items():
        val[(j, k)] = np.array(v, dtype=float)
    for j in range(J - 1, -1, -1):
        for (jj, k) in [n for n in R_old if n[0] == j]:
            val[(jj, k)] = np.mean([val[(j + 1, tuple(2 * c + a for c, a in zip(k, t)))] for t in kids], axis=0)

    def mir(c, j):
        return -1 - c if c < 0 else (2 * (1 << j) - 1 - c if c >= (1 << j) else c)

    def v(j, k):
        k = tuple(mir(c, j) for c in k)
        if (j, k) in val:
            return val[(j, k)]
        par = tuple(c >> 1 for c in k)
        s = np.zeros(m)
        for o in nst:
            wgt = 1.0
            for c, oo in zip(k, o):
                wgt *= 1.0 if oo == 0 else (0.125 if (oo == -1) == (c % 2 == 0) else -0.125)
            s = s + wgt * v(j - 1, tuple(p + oo for p, oo in zip(par, o)))
        return s

    scale = np.maximum(np.max(np.abs(np.array(list(leaves.values()))), axis=0), 1e-30)
    tag = {}
    for node in val:
        j, k = node
        if j == 0:
            continue
        par = tuple(c >> 1 for c in k)
        pred = np.zeros(m)
        for o in nst:
            wgt = 1.0
            for c, oo in zip(k, o):
                wgt *= 1.0 if oo == 0 else (0.125 if (oo == -1) == (c % 2 == 0) else -0.125)
            pred = pred + wgt * v(j - 1, tuple(p + oo for p, oo in zip(par, o)))
        tag[node] = np.max(np.abs(val[node] - pred) / scale) >= eta * 2.0 ** (0.5 * d * (j - J))
    # refined set: old internal nodes + tagged leaves, closed under the grading rule
    R = set(R_old) | {n for n in leaves if tag.get(n, False) and n[0] < J}
    for i in range(J - 1, 0, -1):
        for (j, p) in [n for n in R if n[0] == i]:
            for o in nst:
                q = tuple(c + oo for c, oo in zip(p, o))
                if all(0 <= c < (1 << i) for c in q):
                    R.add((i - 1, tuple(c >> 1 for c in q)))
    # coarsening: remove untagged old refined nodes not forced from one level finer
    for i in range(J - 1, jmin - 1, -1):
        forced = set()
        for (j, p) in [n for n in R if n[0] == i + 1]:
            for o in nst:
                q = tuple(c + oo for c, oo in zip(p, o))
                if all(0 <= c < (1 << (i + 1)) for c in q):
                    forced.add((i, tuple(c >> 1 for c in q)))
        for n in [n for n in R if n[0] == i]:
            if n in R_old and not tag.get(n, False) and n not in forced:
                R.discard(n)
    nodes = {(0, (0,) * d)} | {(j + 1, tuple(2 * c + a for c, a in zip(k, t))) for (j, k) in R for t in kids}
    return {n: v(*n) for n in nodes - R}


@pytest.mark.parametrize("case", range(8))
def test_adapt_matches_bruteforce_on_tiny_trees(case):
    rng = np.random.default_rng(100 + case)
    d, J, jmin = 2, 5, 1 + case % 2
    # random graded starting tree from a random field + a random threshold
    u = rng.standard_normal((2, 1 << (d * J))) * np.exp(-rng.uniform(0, 6, 1 << (d * J)))
    T = O.Tree(d, J, 2, jmin=jmin)
    T.set_full(u)
    assert T.adapt(10 ** rng.uniform(-2.5, -0.5)) == 0
    keys0, vals0 = T.leaves()
    # perturb values so the next adaptation both refines and coarsens
    vals0 = vals0 * (1 + 0.5 * rng.standard_normal(vals0.shape) * (rng.uniform(size=len(keys0)) < 0.3))
    T.set_leaves(keys0, vals0)
    eta = 10 ** rng.uniform(-2.0, -0.7)
    leaves = {}
    for key, col in zip(keys0, vals0.T):
        j, k = O.key_decode(d, int(key))
        leaves[(j, tuple(int(c) for c in k))] = col
    want = _brute_adapt(d, J, jmin, leaves, eta)
    assert T.adapt(eta) == 0
    keys1, vals1 = T.leaves()
    got = {}
    for key, col in zip(keys1, vals1.T):
        j, k = O.key_decode(d, int(key))
        got[(j, tuple(int(c) for c in k))] = col
    assert set(got) == set(want)
    # every case both refines and coarsens somewhere
    assert set(got) - set(leaves) and set(leaves) - set(got)
    for n in got:
        np.testing.assert_allclose(got[n], want[n], rtol=1e-12, atol=1e-12)


def test_bz_adapt_is_graded_with_level_jump_at_most_one():
    J = 7
    T = O.Tree(2, J, 3, jmin=2)
    T.set_full(I.bz_cross_2d(J, 2))
    assert T.adapt(1e-3) == 0 and T.is_graded()
    keys, _ = T.leaves()
    n = 1 << J
    lev = np.full((n, n), -1)
    for key in keys:
        j, k = O.key_decode(2, int(key))
        b = 1 << (J - j)
        lev[k[1] * b:(k[1] + 1) * b, k[0] * b:(k[0] + 1) * b] = j
    assert lev.min() >= 2
    assert np.max(np.abs(np.diff(lev, axis=0))) <= 1 and np.max(np.abs(np.diff(lev, axis=1))) <= 1


def test_compression_ratio_golden():
    g = GOLD["compression_ratio"]
    assert abs((1 - g["N"] / 2 ** (g["d"] * g["J"])) * 100 - g["CR"]) < 1e-9


# ---------------------------------------------------------------- finite-volume operator

def _adaptive_tree(J, seed=2, m=1, d=2, eta=3e-3):
    T = O.Tree(d, J, m, jmin=2)
    if d == 2:
        u = I.bz_cross_2d(J, seed)
    else:
        u = I.bz_sphere_3d(J, seed)
    T.set_full(u[:m] if m <= 3 else np.tile(u, (m, 1))[:m])
    assert T.adapt(eta) == 0
    return T


def test_operator_eta_zero_is_five_point_neumann_laplacian():
    J = 4
    n = 1 << J
    T = O.Tree(2, J, 1, jmin=1)
    T.set_full(np.zeros((1, n * n)))
    rp, col, val, rho = T.operator()
    keys, _ = T.leaves()
    order = [O.key_decode(2, int(k))[1] for k in keys]
    where = {(int(k[0]), int(k[1])): r for r, k in enumerate(order)}
    h2 = float(n * n)
    A = np.zeros((n * n, n * n))
    for (x, y), r in where.items():
        for dx, dy in ((1, 0), (-1, 0), (0, 1), (0, -1)):
            if 0 <= x + dx < n and 0 <= y + dy < n:
                A[r, where[(x + dx, y + dy)]] += h2
                A[r, r] -= h2
    B = np.zeros_like(A)
    for r in range(n * n):
        B[r, col[rp[r]:rp[r + 1]]] = val[rp[r]:rp[r + 1]]
    np.testing.assert_array_equal(A, B)
    assert rho == 8 * h2


@pytest.mark.parametrize("d,J", [(2, 7), (3, 5)])
def test_operator_conserves_mass_and_matches_literal(d, J):
    T = _adaptive_tree(J, d=d, m=2)
    rp, col, val, rho = T.operator()
    keys, _ = T.leaves()
    N = len(keys)
    lev = np.array([int(k) >> 48 for k in keys])
    assert lev.max() > lev.min()  # genuinely adaptive
    vol = 2.0 ** (-d * lev)
    rng = np.random.default_rng(5)
    u = rng.standard_normal((2, N))
    Lu = np.stack([np.add.reduceat(val * u[i][col], rp[:-1]) for i in range(2)])
    scale = np.abs(val).max() * np.abs(u).max()
    assert np.all(np.abs(Lu @ vol) < 1e-12 * scale * np.sum(vol))
    np.testing.assert_allclose(T.apply_literal(u), Lu, atol=1e-12 * scale)
    assert np.allclose(np.add.reduceat(val, rp[:-1]), 0.0, atol=1e-9 * np.abs(val).max())


def test_operator_exact_for_even_quadratic_away_from_far_faces():
    """Prediction reproduces quadratics (Sec. 2.2, l = 1) and the flux rule is
    conservative, so L applied to cell averages of x^2 + y^2 gives exactly 4
    wherever no mirrored stencil crosses the faces x = 1 or y = 1."""
    J = 7
    T = _adaptive_tree(J)
    rp, col, val, rho = T.operator()
    keys, _ = T.leaves()
    n = 1 << J
    ufine = cell_avg_poly(2, J, {(2, 0): 1.0, (0, 2): 1.0})
    u = np.zeros(len(keys))
    inner = np.zeros(len(keys), dtype=bool)
    for r, key in enumerate(keys):
        j, k = O.key_decode(2, int(key))
        b = 1 << (J - j)
        blk = ufine.reshape(n, n)[k[1] * b:(k[1] + 1) * b, k[0] * b:(k[0] + 1) * b]
        u[r] = blk.mean()
        inner[r] = all((kk + 3) * b <= n - 2 * b for kk in k)
    Lu = np.add.reduceat(val * u[col], rp[:-1])
    assert inner.sum() > 100
    np.testing.assert_allclose(Lu[inner], 4.0, rtol=1e-9)
