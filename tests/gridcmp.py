"""Comparisons of two leaf sets (keys as in include/mr.h: Morton abscissa in
bits 0-47, level in bits 48-51) used by the GPU parity tests.

When two runs adapt differently (the mixed form rounds a detail to the other
side of its threshold), their leaves are compared on the finest grid: every
leaf value is injected piecewise constant onto the level-J cells it covers.
"""
import numpy as np


def key_levels(keys):
    return (np.asarray(keys, dtype=np.uint64) >> np.uint64(48)).astype(np.int64)


def finest(keys, vals, d, J):
    """Leaf values on the 2^(dJ) finest cells, lexicographic with x fastest."""
    keys = np.asarray(keys, dtype=np.uint64)
    vals = np.asarray(vals).reshape(-1, len(keys))
    lev = key_levels(keys)
    code = (keys & np.uint64((1 << 48) - 1)).astype(np.int64)
    n = 1 << J
    out = np.zeros((vals.shape[0],) + (n,) * d)
    for j in np.unique(lev):
        sel = np.nonzero(lev == j)[0]
        c = code[sel]
        k = np.zeros((d, len(sel)), dtype=np.int64)
        for b in range(j):  # digit b of every coordinate; x is the more significant bit of a group
            for a in range(d):
                k[a] |= ((c >> (d * b + (d - 1 - a))) & 1) << b
        bsz = 1 << (J - j)
        # every leaf covers a bsz^d block of finest cells; idx[a] runs over
        # coordinate a of the block, shaped to broadcast over the block
        offs = np.arange(bsz)
        idx = []
        for a in range(d):
            shape = [len(sel)] + [1] * d
            shape[1 + (d - 1 - a)] = bsz
            idx.append(((k[a] * bsz)[:, None] + offs[None, :]).reshape(shape))
        # out is indexed [species, z, y, x] (x fastest), so coordinate a is axis d - a
        for i in range(vals.shape[0]):
            v = vals[i, sel].reshape([len(sel)] + [1] * d)
            out[(i,) + tuple(idx[a] for a in reversed(range(d)))] = v
    return out.reshape(vals.shape[0], -1)


def rel_l1_finest(k_a, v_a, k_b, v_b, d, J):
    """max over species of |a - b|_1 / |b|_1 on the finest grid (b the reference)."""
    A, B = finest(k_a, v_a, d, J), finest(k_b, v_b, d, J)
    return max(float(np.sum(np.abs(A[i] - B[i])) / max(np.sum(np.abs(B[i])), 1e-300)) for i in range(len(B)))


def rel_l1_leaves(keys, v_a, v_b, d):
    """The same norm when both live on one leaf set: leaves weighted by their volume."""
    vol = np.ldexp(1.0, -d * key_levels(keys))
    return max(float(np.sum(vol * np.abs(v_a[i] - v_b[i])) / max(np.sum(vol * np.abs(v_b[i])), 1e-300))
               for i in range(len(v_b)))


def rel_linf(a, b):
    return max(float(np.max(np.abs(a[i] - b[i])) / max(np.max(np.abs(b[i])), 1e-300)) for i in range(len(b)))
