"""Python access to the C oracle (test infrastructure only).

The oracle is a plain single-threaded FP64 CPU restatement of the adaptive
multiresolution Strang step (see oracle.h for the paper passages it follows).
Only tests/, the smoke check and the CPU-baseline leg of bench.py import this
module; the product package never does.
"""
from __future__ import annotations

import ctypes as C
import os
import subprocess
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = ["radau5.c", "rock4.c", "mrtree.c", "parallel.c"]
_LIB_PATH = os.path.join(_HERE, "_build", "liboracle.so")
_lock = threading.Lock()
_lib = None

OK = 0
MODEL_BZ, MODEL_NAGUMO, MODEL_LINEAR, MODEL_NETWORK, MODEL_IONIC = 1, 2, 3, 4, 5
MAXM = 32
IONIC_M = 21
MAXR = 32


def build(force: bool = False) -> str:
    """Compile the oracle with gcc (plain -O2, no fast-math, no vector ISA flags)."""
    srcs = [os.path.join(_HERE, s) for s in _SRC] + [os.path.join(_HERE, "oracle.h")]
    newest = max(os.path.getmtime(s) for s in srcs)
    if not force and os.path.exists(_LIB_PATH) and os.path.getmtime(_LIB_PATH) >= newest:
        return _LIB_PATH
    os.makedirs(os.path.dirname(_LIB_PATH), exist_ok=True)
    tmp = _LIB_PATH + f".{os.getpid()}.tmp"
    cmd = ["gcc", "-O2", "-std=c11", "-D_DEFAULT_SOURCE", "-ffp-contract=off", "-fPIC", "-pthread",
           "-shared", "-o", tmp] + [os.path.join(_HERE, s) for s in _SRC] + ["-lm"]
    subprocess.run(cmd, check=True)
    os.replace(tmp, _LIB_PATH)
    return _LIB_PATH


class Model(C.Structure):
    _fields_ = [("kind", C.c_int), ("m", C.c_int), ("p", C.c_double * 8),
                ("K", C.c_double * (MAXM * MAXM)), ("nr", C.c_int),
                ("sp", (C.c_int * 4) * MAXR), ("kf", C.c_double * MAXR), ("kb", C.c_double * MAXR)]


class RadauStats(C.Structure):
    _fields_ = [(n, C.c_int64) for n in
                ("nfev", "njac", "nstep", "naccept", "nreject", "nnewton", "ndec")] + \
               [("status", C.c_int)]


class RockStats(C.Structure):
    _fields_ = [(n, C.c_int64) for n in ("nsteps", "naccept", "nreject", "nstages", "nmatvec")] + \
               [("smax", C.c_int), ("status", C.c_int)]


def lib():
    global _lib
    with _lock:
        if _lib is None:
            _lib = C.CDLL(build())
            _declare(_lib)
    return _lib


def _declare(L):
    dp = C.POINTER(C.c_double)
    ip = C.POINTER(C.c_int32)
    lp = C.POINTER(C.c_int64)
    up = C.POINTER(C.c_uint64)
    vp = C.c_void_p
    sig = {
        "orc_model_f": (None, [C.POINTER(Model), dp, dp]),
        "orc_model_jac": (None, [C.POINTER(Model), dp, dp]),
        "orc_radau_constants": (None, [dp, dp, dp, dp, dp, dp, dp]),
        "orc_radau5": (C.c_int, [C.POINTER(Model), dp, C.c_double, C.c_double, C.c_double,
                                 C.c_double, C.POINTER(RadauStats)]),
        "orc_rock4_ell": (C.c_double, [C.c_int]),
        "orc_rock4_coeffs": (C.c_int, [C.c_int, dp, dp, dp, dp, dp, dp]),
        "orc_rock4_choose": (C.c_int, [C.c_double, C.POINTER(C.c_int), dp]),
        "orc_rock4_linear": (C.c_int, [C.c_int64, lp, ip, dp, C.c_double, C.c_double, dp,
                                       C.c_double, C.c_double, C.c_double, C.POINTER(RockStats)]),
        "orc_tree_new": (vp, [C.c_int, C.c_int, C.c_int, C.c_int]),
        "orc_tree_free": (None, [vp]),
        "orc_tree_set_full": (C.c_int, [vp, dp]),
        "orc_tree_set_leaves": (C.c_int, [vp, C.c_int64, up, dp]),
        "orc_tree_num_leaves": (C.c_int64, [vp]),
        "orc_tree_get_leaves": (C.c_int, [vp, up, dp]),
        "orc_tree_num_nodes": (C.c_int, [vp, lp]),
        "orc_tree_is_graded": (C.c_int, [vp]),
        "orc_project": (None, [vp]),
        "orc_details": (C.c_int, [vp, C.c_int64, up, dp]),
        "orc_value": (C.c_double, [vp, C.c_int, ip, C.c_int]),
        "orc_adapt": (C.c_int, [vp, C.c_double]),
        "orc_operator": (C.c_int, [vp, C.c_int64, lp, ip, dp, dp]),
        "orc_apply_literal": (C.c_int, [vp, dp, dp]),
        "orc_react": (C.c_int, [vp, C.POINTER(Model), C.c_double, C.c_double, C.c_double,
                                C.POINTER(RadauStats), ip]),
        "orc_diffuse": (C.c_int, [vp, dp, C.c_double, C.c_double, C.POINTER(RockStats)]),
        "orc_strang": (C.c_int, [vp, C.POINTER(Model), dp, C.c_double, C.c_double, C.c_double,
                                 C.c_double, C.c_double]),
        "orc_mass": (None, [vp, dp]),
        "orc_key": (C.c_uint64, [C.c_int, C.c_int, ip]),
        "orc_key_decode": (None, [C.c_int, C.c_uint64, C.POINTER(C.c_int), ip]),
    }
    for name, (res, args) in sig.items():
        f = getattr(L, name)
        f.restype = res
        f.argtypes = args


def _d(a):
    return a.ctypes.data_as(C.POINTER(C.c_double))


def _i(a):
    return a.ctypes.data_as(C.POINTER(C.c_int32))


def _l(a):
    return a.ctypes.data_as(C.POINTER(C.c_int64))


def _u(a):
    return a.ctypes.data_as(C.POINTER(C.c_uint64))


def set_threads(n: int):
    """Threads of the oracle's parallel-for (reaction leaves, operator rows); 1 = the plain serial loops."""
    lib().orc_set_threads(int(n))


def make_model(kind: str, m: int | None = None, params=None, K=None) -> Model:
    md = Model()
    if kind == "bz":
        md.kind, md.m = MODEL_BZ, 3
        eps, mu, f, q = params if params is not None else (1e-2, 1e-5, 1.6, 2e-3)
        for i, v in enumerate((eps, mu, f, q)):
            md.p[i] = v
    elif kind == "nagumo":
        md.kind, md.m = MODEL_NAGUMO, 1
        md.p[0] = params[0] if params is not None else 10.0
    elif kind == "linear":
        K = np.asarray(K, dtype=np.float64)
        md.kind, md.m = MODEL_LINEAR, K.shape[0]
        for i, v in enumerate(K.ravel()):
            md.K[i] = v
    elif kind == "network":
        # params = (species (nr x 4 ints), kf (nr), kb (nr)); m species
        sp, kf, kb = params
        sp = np.asarray(sp, dtype=np.int64)
        md.kind, md.m, md.nr = MODEL_NETWORK, int(m), len(sp)
        assert md.nr <= MAXR and md.m <= MAXM
        for r in range(md.nr):
            for t in range(4):
                md.sp[r][t] = int(sp[r, t])
            md.kf[r] = float(kf[r])
            md.kb[r] = float(kb[r])
    elif kind == "ionic":
        md.kind, md.m = MODEL_IONIC, IONIC_M
    else:
        raise ValueError(kind)
    return md


def model_f(md: Model, y):
    y = np.ascontiguousarray(y, dtype=np.float64)
    out = np.zeros(md.m)
    lib().orc_model_f(C.byref(md), _d(y), _d(out))
    return out


def model_jac(md: Model, y):
    y = np.ascontiguousarray(y, dtype=np.float64)
    out = np.zeros(md.m * md.m)
    lib().orc_model_jac(C.byref(md), _d(y), _d(out))
    return out.reshape(md.m, md.m)


def radau_constants():
    c, A, T, Ti = np.zeros(3), np.zeros(9), np.zeros(9), np.zeros(9)
    lam, bhat, e = np.zeros(3), np.zeros(3), np.zeros(3)
    lib().orc_radau_constants(_d(c), _d(A), _d(T), _d(Ti), _d(lam), _d(bhat), _d(e))
    return dict(c=c, A=A.reshape(3, 3), T=T.reshape(3, 3), Tinv=Ti.reshape(3, 3),
                gam=lam[0], alp=lam[1], bet=lam[2], bhat=bhat, e=e)


def radau5(md: Model, y0, tend, rtol=1e-6, atol=1e-6, hfix=0.0):
    y = np.array(y0, dtype=np.float64)
    st = RadauStats()
    rc = lib().orc_radau5(C.byref(md), _d(y), tend, rtol, atol, hfix, C.byref(st))
    return y, rc, {n: getattr(st, n) for n, _ in RadauStats._fields_}


def rock4_ell(s):
    return lib().orc_rock4_ell(s)


def rock4_coeffs(s):
    n = s - 4
    mu, nu, kap = np.zeros(n + 1), np.zeros(n + 1), np.zeros(n + 1)
    w, ec, xc = np.zeros(5), np.zeros(4), np.zeros(5)
    rc = lib().orc_rock4_coeffs(s, _d(mu), _d(nu), _d(kap), _d(w), _d(ec), _d(xc))
    if rc:
        raise RuntimeError(f"rock4 coefficients for s={s} failed ({rc})")
    return dict(mu=mu, nu=nu, kap=kap, w=w, errc=ec, xc=xc, ell=rock4_ell(s))


def rock4_choose(rho_dt):
    s = C.c_int(0)
    ell = C.c_double(0)
    over = lib().orc_rock4_choose(rho_dt, C.byref(s), C.byref(ell))
    return s.value, ell.value, bool(over)


def rock4_linear(rowptr, col, val, D, rho, y0, dt, tol=1e-6, hfix=0.0):
    rowptr = np.ascontiguousarray(rowptr, dtype=np.int64)
    col = np.ascontiguousarray(col, dtype=np.int32)
    val = np.ascontiguousarray(val, dtype=np.float64)
    y = np.array(y0, dtype=np.float64)
    st = RockStats()
    rc = lib().orc_rock4_linear(len(y), _l(rowptr), _i(col), _d(val), D, rho, _d(y), dt, tol,
                                hfix, C.byref(st))
    return y, rc, {n: getattr(st, n) for n, _ in RockStats._fields_}


class Tree:
    """Dense-per-level oracle tree (d, J, jmin, m)."""

    def __init__(self, d, J, m, jmin=2):
        self.d, self.J, self.m, self.jmin = d, J, m, jmin
        self.h = lib().orc_tree_new(d, J, jmin, m)
        if not self.h:
            raise ValueError("invalid tree parameters")

    def __del__(self):
        h = getattr(self, "h", None)
        if h:
            lib().orc_tree_free(h)
            self.h = None

    def set_full(self, u0):
        u0 = np.ascontiguousarray(u0, dtype=np.float64).reshape(self.m, -1)
        assert u0.shape[1] == 1 << (self.d * self.J)
        return lib().orc_tree_set_full(self.h, _d(u0))

    def set_leaves(self, keys, vals):
        keys = np.ascontiguousarray(keys, dtype=np.uint64)
        vals = np.ascontiguousarray(vals, dtype=np.float64).reshape(self.m, len(keys))
        return lib().orc_tree_set_leaves(self.h, len(keys), _u(keys), _d(vals))

    def num_leaves(self):
        return lib().orc_tree_num_leaves(self.h)

    def leaves(self):
        n = self.num_leaves()
        keys = np.zeros(n, dtype=np.uint64)
        vals = np.zeros((self.m, n))
        lib().orc_tree_get_leaves(self.h, _u(keys), _d(vals))
        return keys, vals

    def nodes_per_level(self):
        out = np.zeros(self.J + 1, dtype=np.int64)
        lib().orc_tree_num_nodes(self.h, _l(out))
        return out

    def is_graded(self):
        return bool(lib().orc_tree_is_graded(self.h))

    def project(self):
        lib().orc_project(self.h)

    def details(self):
        cap = int(self.nodes_per_level().sum())
        keys = np.zeros(cap, dtype=np.uint64)
        delta = np.zeros(cap)
        lib().orc_details(self.h, cap, _u(keys), _d(delta))
        n = cap - int(self.nodes_per_level()[0])
        return keys[:n], delta[:n]

    def value(self, j, k, i):
        kk = np.zeros(3, dtype=np.int32)
        kk[: len(k)] = k
        return lib().orc_value(self.h, j, _i(kk), i)

    def adapt(self, eta):
        return lib().orc_adapt(self.h, eta)

    def operator(self):
        n = self.num_leaves()
        cap = 16 * n + 1024
        while True:
            rp = np.zeros(n + 1, dtype=np.int64)
            col = np.zeros(cap, dtype=np.int32)
            val = np.zeros(cap)
            rho = C.c_double(0)
            rc = lib().orc_operator(self.h, cap, _l(rp), _i(col), _d(val), C.byref(rho))
            if rc == 0:
                nnz = int(rp[-1])
                return rp, col[:nnz].copy(), val[:nnz].copy(), rho.value
            cap = int(rp[-1]) + 16

    def apply_literal(self, u):
        n = self.num_leaves()
        u = np.ascontiguousarray(u, dtype=np.float64).reshape(self.m, n)
        out = np.zeros_like(u)
        lib().orc_apply_literal(self.h, _d(u), _d(out))
        return out

    def react(self, md: Model, dt, rtol=1e-6, atol=1e-6, want_complexity=False):
        st = RadauStats()
        cx = np.zeros(self.num_leaves(), dtype=np.int32)
        rc = lib().orc_react(self.h, C.byref(md), dt, rtol, atol, C.byref(st), _i(cx))
        out = {n: getattr(st, n) for n, _ in RadauStats._fields_}
        return (rc, out, cx) if want_complexity else (rc, out)

    def diffuse(self, D, dt, tol=1e-6):
        D = np.ascontiguousarray(D, dtype=np.float64)
        st = RockStats()
        rc = lib().orc_diffuse(self.h, _d(D), dt, tol, C.byref(st))
        return rc, {n: getattr(st, n) for n, _ in RockStats._fields_}

    def strang(self, md: Model, D, dt, eta, rtol=1e-6, atol=1e-6, rock_tol=1e-6):
        D = np.ascontiguousarray(D, dtype=np.float64)
        return lib().orc_strang(self.h, C.byref(md), _d(D), dt, eta, rtol, atol, rock_tol)

    def mass(self):
        out = np.zeros(self.m)
        lib().orc_mass(self.h, _d(out))
        return out


def key(d, j, k):
    kk = np.zeros(3, dtype=np.int32)
    kk[: len(k)] = k
    return int(lib().orc_key(d, j, _i(kk)))


def key_decode(d, key_):
    j = C.c_int(0)
    kk = np.zeros(3, dtype=np.int32)
    lib().orc_key_decode(d, key_, C.byref(j), _i(kk))
    return j.value, kk[:d].copy()
