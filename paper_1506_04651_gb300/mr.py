"""Python binding of the C-ABI in include/mr.h (argument marshalling only).

Every computation happens in the sm_103a kernels of libmrgb300.so; this module
only converts NumPy arrays / torch tensors to pointers.  It raises if the
native library has not been built: there is no CPU fallback.
"""
from __future__ import annotations

import ctypes as C
import os

import numpy as np

from . import build as _build

MR_OK = 0
MR_MODEL_BZ, MR_MODEL_NAGUMO, MR_MODEL_NETWORK, MR_MODEL_IONIC = 1, 2, 3, 4
IONIC_SPECIES = 21
MR_FP64, MR_MIXED, MR_MIXED_F32_DETAILS = 0, 1, 2
MR_RADAU_THREAD, MR_RADAU_POOL = 0, 1
MAX_SPECIES, MAX_LEVEL = 32, 16
NOALLOC_MAX_CELLS = 2147483647  # MR_NOALLOC_MAX_CELLS of include/mr.h

STATUS = {0: "MR_OK", -1: "MR_EINVAL", -2: "MR_ENOMEM", -3: "MR_ECUDA", -4: "MR_ESTATE",
          -10: "MR_ERADAU_HMIN", -11: "MR_ERADAU_MAXSTEPS", -12: "MR_ERADAU_SINGULAR",
          -20: "MR_EROCK_STEP", -30: "MR_ENONFINITE", -40: "MR_ETIMEOUT", -50: "MR_EIO"}


class Problem(C.Structure):
    _fields_ = [("dim", C.c_int), ("J", C.c_int), ("jmin", C.c_int), ("m", C.c_int),
                ("model", C.c_int), ("nparams", C.c_int), ("precision", C.c_int),
                ("reserved", C.c_int), ("params", C.c_double * 8),
                ("D", C.c_double * MAX_SPECIES), ("max_leaves", C.c_int64)]


class Stats(C.Structure):
    _fields_ = [("leaves", C.c_int64), ("nodes", C.c_int64),
                ("leaves_per_level", C.c_int64 * (MAX_LEVEL + 1)),
                ("compression_ratio", C.c_double)] + \
               [(n, C.c_int64) for n in ("radau_fev", "radau_jac", "radau_steps", "radau_accept",
                                         "radau_reject", "radau_newton", "radau_dec",
                                         "rock_steps", "rock_reject", "rock_stages", "rock_matvec")] + \
               [("rock_smax", C.c_int32), ("reserved0", C.c_int32), ("rock_rho", C.c_double),
                ("irregular_rows", C.c_int64), ("irregular_nnz", C.c_int64),
                ("ms_adapt", C.c_double), ("ms_react", C.c_double), ("ms_diffuse", C.c_double),
                ("kernel_launches", C.c_int64),
                ("radau_kernel_ms", C.c_double), ("radau_alg_flops", C.c_double),
                ("radau_kernel_launches", C.c_int64),
                ("rock_kernel_ms", C.c_double), ("rock_alg_bytes", C.c_double),
                ("rock_kernel_launches", C.c_int64), ("radau_counters", C.c_int64 * 8),
                ("rock_alg_flops", C.c_double)]

    def as_dict(self):
        out = {}
        for name, _ in self._fields_:
            v = getattr(self, name)
            out[name] = list(v) if name in ("leaves_per_level", "radau_counters") else v
        return out


_lib = None


def lib():
    """Load the in-tree libmrgb300.so (built by __graft_entry__.build())."""
    global _lib
    if _lib is None:
        path = _build.LIB
        if not os.path.exists(path):
            raise RuntimeError(f"native library missing: {path}; run __graft_entry__.build()")
        L = C.CDLL(path)
        vp, dp, i64, i64p = C.c_void_p, C.c_void_p, C.c_int64, C.POINTER(C.c_int64)
        sig = {
            "mr_create": [C.POINTER(Problem), vp, C.POINTER(C.c_void_p)],
            "mr_build": [vp, dp, C.c_int, C.c_double],
            "mr_set_leaves": [vp, i64, vp, dp, C.c_int],
            "mr_num_leaves": [vp, i64p],
            "mr_get_leaves": [vp, vp, dp, i64, i64p, C.c_int],
            "mr_adapt": [vp, C.c_double],
            "react_radau5": [vp, C.c_double, C.c_double, C.c_double],
            "mr_set_radau_schedule": [vp, C.c_int],
            "diffuse_rock4": [vp, C.c_double, C.c_double],
            "strang_step": [vp, C.c_double, C.c_double, C.c_double, C.c_double, C.c_double],
            "mr_get_stats": [vp, C.POINTER(Stats)],
            "mr_get_complexity": [vp, vp, i64, C.c_int],
            "mr_mass": [vp, dp],
            "mr_apply_operator": [vp, dp, dp, C.c_int, C.POINTER(C.c_double)],
            "mr_operator_forms": [vp, C.c_int, C.POINTER(C.c_double), C.POINTER(C.c_double), i64p,
                                  C.POINTER(C.c_double)],
            "mr_rock4_coefficients": [C.c_int, dp, dp, dp, dp, dp, C.POINTER(C.c_double)],
            "mr_radau_work": [C.c_int, C.c_int, dp],
            "mr_last_error": [vp, C.c_char_p, C.c_size_t],
            "mr_fp64_fma_rate": [C.POINTER(C.c_double), C.POINTER(C.c_double)],
            "mr_save": [vp, C.c_char_p],
            "mr_set_network": [vp, C.c_int, vp, dp, dp],
            "mr_load": [vp, C.c_char_p],
            "mr_batch_create": [C.c_int, C.POINTER(Problem), C.c_int, C.POINTER(C.c_void_p)],
            "mr_batch_run": [vp, C.c_int, C.c_double, dp, C.c_double, C.c_double, C.c_double],
            "mr_batch_diffuse": [vp, C.c_double, C.c_double],
            "mr_batch_get_stats": [vp, C.POINTER(BatchStats)],
            "mr_batch_set_autotune": [vp, C.c_int],
            "mr_batch_tuning": [vp, vp, C.c_int, C.POINTER(C.c_int)],
        }
        for name, args in sig.items():
            f = getattr(L, name)
            f.argtypes = args
            f.restype = C.c_int
        L.mr_destroy.argtypes = [vp]
        L.mr_destroy.restype = None
        L.mr_batch_context.argtypes = [vp, C.c_int]
        L.mr_batch_context.restype = C.c_void_p
        L.mr_batch_destroy.argtypes = [vp]
        L.mr_batch_destroy.restype = None
        L.mr_status_str.argtypes = [C.c_int]
        L.mr_status_str.restype = C.c_char_p
        _lib = L
    return _lib


class TuneEntry(C.Structure):
    _fields_ = [("phase", C.c_int32), ("block", C.c_int32), ("per_sm", C.c_int32), ("order", C.c_int32),
                ("launches", C.c_int64), ("ms", C.c_double), ("work", C.c_double), ("rate", C.c_double),
                ("chosen", C.c_int32), ("schedule", C.c_int32)]


class BatchStats(C.Structure):
    _fields_ = [(n, C.c_int64) for n in ("instances", "threads", "steps", "leaf_updates")] + \
               [("ms_device", C.c_double), ("ms_react_kernel", C.c_double), ("react_launches", C.c_int64)] + \
               [(n, C.c_int64) for n in ("radau_fev", "radau_jac", "radau_steps", "radau_accept", "radau_reject",
                                         "radau_newton", "radau_dec")] + \
               [("radau_alg_flops", C.c_double), ("joint_reaction", C.c_int32), ("joint_diffusion", C.c_int32),
                ("ms_adapt_phase", C.c_double), ("ms_diffuse_phase", C.c_double),
                ("ms_diffuse_kernel", C.c_double), ("diffuse_launches", C.c_int64)]

    def as_dict(self):
        return {n: getattr(self, n) for n, _ in self._fields_}


class MRError(RuntimeError):
    def __init__(self, code, where, msg=""):
        super().__init__(f"{where}: {STATUS.get(code, code)} {msg}".strip())
        self.code = code


def _ptr(a):
    """(pointer, on_device) of a NumPy array or a torch tensor."""
    if isinstance(a, np.ndarray):
        return a.ctypes.data, 0
    return a.data_ptr(), int(a.is_cuda)


def problem(dim, J, model="bz", params=None, D=None, jmin=2, precision=MR_FP64, max_leaves=0):
    p = Problem()
    p.dim, p.J, p.jmin, p.precision, p.max_leaves = dim, J, jmin, precision, max_leaves
    if model == "bz":
        p.model, p.m = MR_MODEL_BZ, 3
        params = params if params is not None else (1e-2, 1e-5, 1.6, 2e-3)
        D = D if D is not None else (2.5e-3, 2.5e-3, 1.5e-3)
    elif model == "nagumo":
        p.model, p.m = MR_MODEL_NAGUMO, 1
        params = params if params is not None else (10.0,)
        D = D if D is not None else (0.1,)
    elif model == "network":
        # reactions are set on the context (Context.set_network); D has m entries
        p.model, p.m = MR_MODEL_NETWORK, len(D)
        params = ()
    elif model == "ionic":
        # the synthetic 21-species membrane model; D has 21 entries
        p.model, p.m = MR_MODEL_IONIC, IONIC_SPECIES
        params = ()
        assert D is not None and len(D) == IONIC_SPECIES
    else:
        raise ValueError(model)
    p.nparams = len(params)
    for i, v in enumerate(params):
        p.params[i] = v
    for i, v in enumerate(D):
        p.D[i] = v
    return p


class Context:
    """One problem on one GPU (owns the device memory of mr_create)."""

    def __init__(self, prob: Problem, stream=None):
        h = C.c_void_p()
        s = stream.cuda_stream if hasattr(stream, "cuda_stream") else (stream or 0)
        rc = lib().mr_create(C.byref(prob), C.c_void_p(s), C.byref(h))
        if rc:
            raise MRError(rc, "mr_create")
        self.h, self.prob, self.m = h, prob, prob.m

    @classmethod
    def _borrowed(cls, handle, prob):
        """A view of a context owned by something else (a Batch): not destroyed on close."""
        c = cls.__new__(cls)
        c.h, c.prob, c.m, c._owned = C.c_void_p(handle), prob, prob.m, False
        return c

    def close(self):
        if getattr(self, "h", None):
            if getattr(self, "_owned", True):
                lib().mr_destroy(self.h)
            self.h = None

    __del__ = close

    def _check(self, rc, where):
        if rc:
            buf = C.create_string_buffer(256)
            lib().mr_last_error(self.h, buf, 256)
            raise MRError(rc, where, buf.value.decode())
        return rc

    def build(self, u0, eta):
        p, dev = _ptr(u0)
        return self._check(lib().mr_build(self.h, C.c_void_p(p), dev, eta), "mr_build")

    def set_leaves(self, keys, values):
        kp, kd = _ptr(keys)
        vp, vd = _ptr(values)
        assert kd == vd
        return self._check(lib().mr_set_leaves(self.h, len(keys), C.c_void_p(kp), C.c_void_p(vp), kd),
                           "mr_set_leaves")

    def num_leaves(self):
        n = C.c_int64()
        self._check(lib().mr_num_leaves(self.h, C.byref(n)), "mr_num_leaves")
        return n.value

    def leaves(self, keys_out=None, values_out=None):
        n = self.num_leaves()
        keys = keys_out if keys_out is not None else np.zeros(n, dtype=np.uint64)
        vals = values_out if values_out is not None else np.zeros((self.m, n))
        kp, kd = _ptr(keys)
        vp, vd = _ptr(vals)
        cnt = C.c_int64()
        self._check(lib().mr_get_leaves(self.h, C.c_void_p(kp), C.c_void_p(vp), n, C.byref(cnt), vd),
                    "mr_get_leaves")
        return keys, vals

    def adapt(self, eta):
        return self._check(lib().mr_adapt(self.h, eta), "mr_adapt")

    def react(self, dt, rtol=1e-6, atol=1e-6):
        return self._check(lib().react_radau5(self.h, dt, rtol, atol), "react_radau5")

    def set_radau_schedule(self, schedule):
        """MR_RADAU_THREAD (the default) or MR_RADAU_POOL; bit-identical results."""
        return self._check(lib().mr_set_radau_schedule(self.h, schedule), "mr_set_radau_schedule")

    def diffuse(self, dt, tol=1e-6):
        return self._check(lib().diffuse_rock4(self.h, dt, tol), "diffuse_rock4")

    def strang(self, dt, eta, rtol=1e-6, atol=1e-6, rock_tol=1e-6):
        return self._check(lib().strang_step(self.h, dt, eta, rtol, atol, rock_tol), "strang_step")

    def stats(self):
        s = Stats()
        self._check(lib().mr_get_stats(self.h, C.byref(s)), "mr_get_stats")
        return s.as_dict()

    def complexity(self):
        out = np.zeros(self.num_leaves(), dtype=np.int32)
        self._check(lib().mr_get_complexity(self.h, C.c_void_p(out.ctypes.data), len(out), 0),
                    "mr_get_complexity")
        return out

    def set_network(self, species, kf, kb):
        """Reactions of a network-model context (mr_set_network)."""
        sp = np.ascontiguousarray(species, dtype=np.int32)
        kf = np.ascontiguousarray(kf, dtype=np.float64)
        kb = np.ascontiguousarray(kb, dtype=np.float64)
        self._check(lib().mr_set_network(self.h, len(sp), C.c_void_p(sp.ctypes.data), C.c_void_p(kf.ctypes.data),
                                         C.c_void_p(kb.ctypes.data)), "mr_set_network")

    def save(self, path):
        """Write a checkpoint of the current leaves (mr_save)."""
        self._check(lib().mr_save(self.h, os.fsencode(path)), "mr_save")

    def load(self, path):
        """Replace the tree by a checkpoint's leaves (mr_load)."""
        self._check(lib().mr_load(self.h, os.fsencode(path)), "mr_load")

    def mass(self):
        out = np.zeros(self.m)
        self._check(lib().mr_mass(self.h, C.c_void_p(out.ctypes.data)), "mr_mass")
        return out

    def operator_forms(self, reps=20):
        """Mean device time of one application of the leaf operator in its compact
        form and as a CSR matrix (mr_operator_forms)."""
        a, b, d = C.c_double(), C.c_double(), C.c_double()
        nnz = C.c_int64()
        self._check(lib().mr_operator_forms(self.h, reps, C.byref(a), C.byref(b), C.byref(nnz), C.byref(d)),
                    "mr_operator_forms")
        return {"ms_compact": a.value, "ms_csr": b.value, "csr_nnz": nnz.value, "max_rel_diff": d.value}

    def apply_operator(self, u):
        u = np.ascontiguousarray(u, dtype=np.float64)
        out = np.zeros_like(u)
        rho = C.c_double()
        self._check(lib().mr_apply_operator(self.h, C.c_void_p(u.ctypes.data), C.c_void_p(out.ctypes.data),
                                            0, C.byref(rho)), "mr_apply_operator")
        return out, rho.value


def rock4_coefficients(s):
    n = s - 4
    mu, nu, kap = np.zeros(n + 1), np.zeros(n + 1), np.zeros(n + 1)
    w, errc = np.zeros(5), np.zeros(4)
    ell = C.c_double()
    rc = lib().mr_rock4_coefficients(s, *(C.c_void_p(a.ctypes.data) for a in (mu, nu, kap, w, errc)),
                                     C.byref(ell))
    if rc:
        raise MRError(rc, "mr_rock4_coefficients")
    return dict(mu=mu, nu=nu, kap=kap, w=w, errc=errc, ell=ell.value)


def radau_work(model, m):
    """The library's per-event FP64 operation counts of the Radau5 kernel
    (rhs, jac, dec, newton, monitor, attempt, extrap, accept)."""
    out = np.zeros(8)
    rc = lib().mr_radau_work(model, m, C.c_void_p(out.ctypes.data))
    if rc:
        raise MRError(rc, "mr_radau_work")
    return dict(zip(("rhs", "jac", "dec", "newton", "monitor", "attempt", "extrap", "accept"), out.tolist()))


def status_str(code):
    return lib().mr_status_str(code).decode()


def fp64_fma_rate():
    """(TFLOP/s, SM MHz) of the device's FP64 FMA pipe, from the library's probe."""
    t, mhz = C.c_double(), C.c_double()
    rc = lib().mr_fp64_fma_rate(C.byref(t), C.byref(mhz))
    if rc:
        raise MRError(rc, "mr_fp64_fma_rate")
    return t.value, mhz.value


class Batch:
    """Batched serving (mr_batch_*): independent instances stepped together,
    the reaction half steps of all of them as one joint Radau5 launch and
    the diffusion sub-step as one joint ROCK4 launch."""

    def __init__(self, problems, threads=0):
        arr = (Problem * len(problems))(*problems)
        h = C.c_void_p()
        rc = lib().mr_batch_create(len(problems), arr, threads, C.byref(h))
        if rc:
            raise MRError(rc, "mr_batch_create")
        self.h, self.n = h, len(problems)
        self.contexts = [Context._borrowed(lib().mr_batch_context(h, i), problems[i]) for i in range(self.n)]

    def __getitem__(self, i):
        return self.contexts[i]

    def run(self, nsteps, dt, eta, rtol=1e-6, atol=1e-6, rock_tol=1e-6):
        eta = np.ascontiguousarray(eta, dtype=np.float64)
        assert len(eta) == self.n
        rc = lib().mr_batch_run(self.h, nsteps, dt, C.c_void_p(eta.ctypes.data), rtol, atol, rock_tol)
        if rc:
            msgs = []
            for i, c in enumerate(self.contexts):
                buf = C.create_string_buffer(256)
                lib().mr_last_error(c.h, buf, 256)
                if buf.value:
                    msgs.append(f"[{i}] {buf.value.decode()}")
            raise MRError(rc, "mr_batch_run", "; ".join(msgs))

    def diffuse(self, dt, tol=1e-6):
        rc = lib().mr_batch_diffuse(self.h, dt, tol)
        if rc:
            raise MRError(rc, "mr_batch_diffuse")

    def stats(self):
        s = BatchStats()
        lib().mr_batch_get_stats(self.h, C.byref(s))
        return s.as_dict()

    def set_autotune(self, on):
        rc = lib().mr_batch_set_autotune(self.h, int(bool(on)))
        if rc:
            raise MRError(rc, "mr_batch_set_autotune")

    def tuning(self):
        """The autotuner's trial table: one dict per candidate launch shape."""
        arr = (TuneEntry * 16)()
        n = C.c_int()
        rc = lib().mr_batch_tuning(self.h, C.addressof(arr), 16, C.byref(n))
        if rc:
            raise MRError(rc, "mr_batch_tuning")
        names = ("reaction", "diffusion")
        return [dict(phase=names[e.phase], block=e.block, per_sm=e.per_sm, order=e.order, launches=e.launches,
                     ms=e.ms, work=e.work, rate=e.rate, chosen=bool(e.chosen),
                     schedule="pool" if e.schedule == MR_RADAU_POOL else "thread") for e in arr[:n.value]]

    def close(self):
        if getattr(self, "h", None):
            for c in self.contexts:
                c.h = None
            lib().mr_batch_destroy(self.h)
            self.h = None

    __del__ = close
