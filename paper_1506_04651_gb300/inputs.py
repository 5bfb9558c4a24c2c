"""Seeded synthetic inputs for the BZ front-propagation workloads.

This module only generates input data (initial states on the finest grid and
random instance parameters).  It holds none of the method's arithmetic and is
the one piece of code that both the GPU path's callers and the oracle's tests
use.  The paper prints no initial data (Sec. 4 shows BZ fronts, Fig. 3), so
these recipes are readings of its figures and of the workload descriptions:

* a tanh front of width w in b = u2 between the rest state b_r and an excited
  value b_e, c = u3 = b, and a = u1 slaved to the fast manifold a = f c/(q + b);
* "1% seeded noise": a multiplicative factor (1 + 0.01 xi), xi ~ U[-1, 1];
* "smooth seeded noise": the front position is perturbed by 8 seeded Fourier
  modes of amplitude 0.01 (so the details stay small away from the front).

Random numbers come from splitmix64(seed XOR index) mapped to [0, 1).
Cell values are point values at cell centres of the finest level J, laid out
as an array of shape (m, 2^(d J)) with x fastest (lexicographic).
"""
from __future__ import annotations

import numpy as np

BZ_DEFAULT = dict(eps=1e-2, mu=1e-5, f=1.6, q=2e-3)
BZ_D = (2.5e-3, 2.5e-3, 1.5e-3)
# front width and position-noise amplitude of the adaptive 2D J = 10 workload
# (two crossing fronts, eta = 1e-3): sharper and more convoluted fronts than
# the 3D sphere's, so that 10-20% of the finest cells are leaves
CROSS_J10 = dict(w=0.01, amp=0.3)
_M64 = np.uint64(0xFFFFFFFFFFFFFFFF)


def splitmix64(x: np.ndarray) -> np.ndarray:
    """splitmix64 finaliser applied elementwise to uint64 inputs (Steele et al.)."""
    with np.errstate(over="ignore"):
        z = (np.asarray(x, dtype=np.uint64) + np.uint64(0x9E3779B97F4A7C15)) & _M64
        z = ((z ^ (z >> np.uint64(30))) * np.uint64(0xBF58476D1CE4E5B9)) & _M64
        z = ((z ^ (z >> np.uint64(27))) * np.uint64(0x94D049BB133111EB)) & _M64
        return z ^ (z >> np.uint64(31))


def uniform(seed: int, index: np.ndarray) -> np.ndarray:
    """U[0,1) doubles from splitmix64(seed ^ index), 53 significant bits."""
    z = splitmix64(np.uint64(seed) ^ np.asarray(index, dtype=np.uint64))
    return (z >> np.uint64(11)).astype(np.float64) * (1.0 / 9007199254740992.0)


def bz_rest_state(f: float, q: float) -> float:
    """Positive root b of b^2 + (q + f - 1) b - q (1 + f) = 0 (the BZ fixed point)."""
    bq = q + f - 1.0
    return 0.5 * (-bq + np.sqrt(bq * bq + 4.0 * q * (1.0 + f)))


def cell_centres(d: int, J: int):
    n = 1 << J
    x = (np.arange(n) + 0.5) / n
    grids = np.meshgrid(*([x] * d), indexing="ij")
    # lexicographic with x fastest: coordinate a varies with stride n^a
    return [g.transpose(tuple(range(d))[::-1]).ravel() for g in grids]


def _profile(s, w):
    return 0.5 * (1.0 - np.tanh(s / w))


def _fourier(seed: int, t: np.ndarray, nmodes: int = 8, amp: float = 0.01) -> np.ndarray:
    r = uniform(seed, np.arange(2 * nmodes, dtype=np.uint64))
    out = np.zeros_like(t)
    for k in range(nmodes):
        out += np.sin(2.0 * np.pi * (k + 1) * t + 2.0 * np.pi * r[2 * k]) * (r[2 * k + 1] - 0.5)
    return amp * out / (0.5 * nmodes ** 0.5)


def bz_state(b: np.ndarray, c: np.ndarray, f: float, q: float) -> np.ndarray:
    a = f * c / (q + b)
    return np.stack([a, b, c])


def bz_front_2d(J: int, seed: int, x0: float = 0.5, w: float = 0.02, noise: float = 0.01,
                f: float = BZ_DEFAULT["f"], q: float = BZ_DEFAULT["q"], be: float = 0.8):
    """2D front in x at x0 with multiplicative white noise (uniform 128x128 workload)."""
    x, y = cell_centres(2, J)
    br = bz_rest_state(f, q)
    b = br + (be - br) * _profile(x - x0, w)
    u = bz_state(b, b.copy(), f, q)
    if noise:
        idx = np.arange(u.size, dtype=np.uint64)
        xi = 2.0 * uniform(seed, idx) - 1.0
        u = u * (1.0 + noise * xi.reshape(u.shape))
    return u


def bz_cross_2d(J: int, seed: int, w: float = 0.02, f: float = BZ_DEFAULT["f"],
                q: float = BZ_DEFAULT["q"], be: float = 0.8, x0: float = 0.5, y0: float = 0.5,
                amp: float = 0.01):
    """Two crossing fronts: b from a front along x = x0(y), c from a front along y = y0(x),
    both positions perturbed by smooth seeded Fourier noise of amplitude amp."""
    x, y = cell_centres(2, J)
    br = bz_rest_state(f, q)
    px = x0 + _fourier(seed, y, amp=amp)
    py = y0 + _fourier(seed + 1, x, amp=amp)
    b = br + (be - br) * _profile(x - px, w)
    c = br + (be - br) * _profile(y - py, w)
    return bz_state(b, c, f, q)


def bz_front_smooth_2d(J: int, seed: int, x0: float = 0.5, f: float = BZ_DEFAULT["f"],
                       q: float = BZ_DEFAULT["q"], w: float = 0.02, amp: float = 0.02, be: float = 0.8):
    """One front along x = x0(y) (smooth seeded position noise), rest state of the
    instance's f: the per-instance initial state of the batched workload."""
    x, y = cell_centres(2, J)
    br = bz_rest_state(f, q)
    b = br + (be - br) * _profile(x - (x0 + _fourier(seed, y, amp=amp)), w)
    return bz_state(b, b.copy(), f, q)


def bz_sphere_3d(J: int, seed: int, r0: float = 0.3, w: float = 0.02,
                 f: float = BZ_DEFAULT["f"], q: float = BZ_DEFAULT["q"], be: float = 0.8):
    """Spherical front of radius r0 about the centre, radius perturbed smoothly."""
    x, y, z = cell_centres(3, J)
    br = bz_rest_state(f, q)
    dx, dy, dz = x - 0.5, y - 0.5, z - 0.5
    r = np.sqrt(dx * dx + dy * dy + dz * dz)
    th = np.arctan2(dy, dx) / (2.0 * np.pi)
    ph = np.arccos(np.clip(dz / np.maximum(r, 1e-300), -1.0, 1.0)) / np.pi
    rr = r0 + 0.5 * (_fourier(seed, th) + _fourier(seed + 1, ph))
    b = br + (be - br) * _profile(r - rr, w)
    return bz_state(b, b.copy(), f, q)


NAGUMO_K, NAGUMO_D = 10.0, 0.1  # Sec. 1 item I: k = 10, diffusion 0.1


def nagumo_front(d: int, J: int, r0: float = 0.3, k: float = NAGUMO_K, D: float = NAGUMO_D):
    """A circular (2D) or spherical (3D) NAGUMO front of radius r0 about the
    domain centre with the travelling-front profile 1 / (1 + exp(lam (r - r0))),
    lam = sqrt(k / (2 D)); values in [0, 1].  Shape (1, 2^(dJ))."""
    xs = cell_centres(d, J)
    r = np.sqrt(sum((x - 0.5) ** 2 for x in xs))
    lam = np.sqrt(k / (2.0 * D))
    return (1.0 / (1.0 + np.exp(lam * (r - r0)))).reshape(1, -1)


def batch_instances(n: int, master_seed: int = 2026):
    """Per-instance parameters of the batched workload: J ~ U{7..10}, f ~ U[0.9, 2.0],
    eta log-uniform in [1e-4, 1e-2], front position ~ U[0.2, 0.8]."""
    out = []
    for i in range(n):
        s = int(splitmix64(np.uint64(master_seed) ^ np.uint64(i)))
        r = uniform(s, np.arange(4, dtype=np.uint64))
        out.append(dict(seed=s, J=7 + int(r[0] * 4), f=0.9 + 1.1 * r[1],
                        eta=10.0 ** (-4.0 + 2.0 * r[2]), x0=0.2 + 0.6 * r[3]))
    return out


def network_instance(seed: int = 5, m: int = 16, nr: int = 32):
    """Synthetic stiff mass-action network: nr reversible reactions
    u_a + u_b <-> u_c + u_d, the four species of each reaction distinct and
    drawn uniformly, forward / backward rates log-uniform in [1e-2, 1e6],
    diffusion coefficients log-uniform in [1e-4, 1e-2].  Returns
    (species (nr x 4 int32), kf (nr), kb (nr), D (m))."""
    r = uniform(seed, np.arange(4 * nr + 2 * nr + m + 64 * nr, dtype=np.uint64))
    sp = np.zeros((nr, 4), dtype=np.int32)
    pos = 0
    for q in range(nr):
        pool = list(range(m))
        for t in range(4):
            # draw without replacement: index into the remaining species
            k = int(r[pos] * len(pool))
            pos += 1
            sp[q, t] = pool.pop(min(k, len(pool) - 1))
    kf = 10.0 ** (-2.0 + 8.0 * r[pos:pos + nr])
    pos += nr
    kb = 10.0 ** (-2.0 + 8.0 * r[pos:pos + nr])
    pos += nr
    D = 10.0 ** (-4.0 + 2.0 * r[pos:pos + m])
    return sp, kf, kb, D


def network_bumps(d: int, J: int, seed: int = 5, m: int = 16, nbumps: int = 4):
    """Positive initial state of the network workload: per species
    u_i = 0.1 + sum_b A_ib exp(-|x - c_ib|^2 / (2 sigma_ib^2)), A ~ U[0.2, 1],
    sigma ~ U[0.05, 0.15], centres ~ U[0.2, 0.8]^d; shape (m, 2^(dJ))."""
    n = 1 << J
    x = (np.arange(n) + 0.5) / n
    r = uniform(seed ^ 0x5EED, np.arange(m * nbumps * (2 + d), dtype=np.uint64)).reshape(m, nbumps, 2 + d)
    u = np.empty((m,) + (n,) * d)
    for i in range(m):
        acc = u[i]
        acc.fill(0.1)
        for b in range(nbumps):
            amp = 0.2 + 0.8 * r[i, b, 0]
            sig = 0.05 + 0.10 * r[i, b, 1]
            # the Gaussian is the product of one factor per axis; array axes
            # are (z, y, x) / (y, x) so that x varies fastest
            g = [np.exp(-((x - (0.2 + 0.6 * r[i, b, 2 + a])) ** 2) / (2.0 * sig * sig)) for a in range(d)]
            prod = amp * g[d - 1]
            for a in range(d - 2, -1, -1):
                prod = np.multiply.outer(prod, g[a])
            acc += prod
    return u.reshape(m, -1)


# ---- the synthetic 21-species membrane model (stand-in for the paper's STROKE case)
# Species order: e_0..e_3, g, c_0..c_3, V, a_0..a_3, b_0..b_3, E, B, S (the
# first five diffuse).  IONIC_REST is the model's resting state with energy
# supply S = 1 and IONIC_DEP its depolarised state (transmitter released,
# ion 1 released to the extracellular space), both found once by integrating
# a single cell to rest; they are initial data, not expected values.
IONIC_M = 21
IONIC_D = (2e-3, 2e-3, 2e-3, 1e-3, 1e-2) + (0.0,) * 16
IONIC_REST = (14.22728634, 0.1269996353, 12.00428593, 0.15, 8.033406869e-08, 1.443178415, 14.05575009,
              0.7989285171, 1e-05, -4.554532729, 2.790947026e-09, 7.712475299e-06, 7.149632481e-06,
              7.23671077e-13, 0.9999999841, 0.9999993314, 0.9999997449, 0.999999616, 0.9942973554,
              0.09090909091, 1.0)
IONIC_DEP = (9.398867673, 3.085280159, 10.11221508, 0.1390336202, 1.99991224, 2.650283082, 13.31617996,
             1.27194623, 2.77243063e-05, -0.4879979785, 0.9993971778, 0.9998082956, 0.8462659894,
             0.9973559367, 1.204223034e-07, 0.1155875563, 0.8371923037, 0.003858656587, 0.9840238873,
             0.1453865038, 1.0)


def ionic_core(d: int, J: int, seed: int = 7, r0: float = 0.2, w: float = 0.02, amp: float = 0.02,
               s_core: float = 0.2):
    """Depolarised core in resting tissue: u = rest + (dep - rest) chi with
    chi = (1 - tanh((r - r0(angle)) / w)) / 2 about the domain centre, the
    radius perturbed by smooth seeded Fourier noise; the energy supply S is
    1 - (1 - s_core) chi (an ischaemic core).  Shape (21, 2^(dJ))."""
    xs = cell_centres(d, J)
    dx = [x - 0.5 for x in xs]
    r = np.sqrt(sum(v * v for v in dx))
    th = np.arctan2(dx[1], dx[0]) / (2.0 * np.pi)
    rr = r0 + _fourier(seed, th, amp=amp)
    if d == 3:
        ph = np.arccos(np.clip(dx[2] / np.maximum(r, 1e-300), -1.0, 1.0)) / np.pi
        rr = rr + _fourier(seed + 1, ph, amp=amp)
    chi = _profile(r - rr, w)
    rest, dep = np.asarray(IONIC_REST), np.asarray(IONIC_DEP)
    u = rest[:, None] + (dep - rest)[:, None] * chi[None, :]
    u[20] = 1.0 - (1.0 - s_core) * chi
    return u
