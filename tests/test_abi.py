"""The C-ABI library builds for sm_103a, loads, and exports every symbol that
include/mr.h declares (no GPU needed).  The host-side ROCK4-type coefficient
construction of the library is compared with the oracle's independent one."""
import ctypes as C
import os
import re

import numpy as np
import pytest

from oracle import oracle as O

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.fixture(scope="module")
def native():
    from paper_1506_04651_gb300 import build as B
    B.build()
    from paper_1506_04651_gb300 import mr
    return mr


def declared_symbols():
    src = open(os.path.join(ROOT, "include", "mr.h")).read()
    src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
    names = re.findall(r"^\s*(?:const\s+)?[a-z_0-9]+\s*\*?\s*([a-z_0-9]+)\s*\(", src, flags=re.M)
    return sorted(set(names))


def test_header_declares_the_boundary():
    names = declared_symbols()
    for want in ("mr_create", "mr_destroy", "mr_build", "mr_adapt", "react_radau5", "diffuse_rock4",
                 "strang_step", "mr_get_leaves", "mr_set_leaves", "mr_get_stats", "mr_status_str"):
        assert want in names


def test_library_exports_every_declared_symbol(native):
    L = native.lib()
    for name in declared_symbols():
        assert hasattr(L, name), name


def test_status_strings(native):
    for code in native.STATUS:
        assert native.status_str(code)


def test_invalid_problem_rejected_before_gpu_work(native):
    p = native.problem(2, 10)
    p.dim = 4
    h = C.c_void_p()
    assert native.lib().mr_create(C.byref(p), None, C.byref(h)) == -1
    p = native.problem(3, 11)  # d*J > 30
    assert native.lib().mr_create(C.byref(p), None, C.byref(h)) == -1


@pytest.mark.parametrize("s", [5, 6, 9, 17, 40, 100, 152])
def test_rock4_coefficients_match_oracle(native, s):
    g = native.rock4_coefficients(s)
    o = O.rock4_coeffs(s)
    assert g["ell"] == o["ell"]
    for k in ("mu", "nu", "kap"):
        np.testing.assert_allclose(g[k], o[k], rtol=2e-12, atol=1e-15)
    np.testing.assert_allclose(g["w"], o["w"], rtol=2e-12)
    np.testing.assert_allclose(g["errc"], o["errc"], rtol=1e-10)


def test_noalloc_maximum_rejected_before_gpu_work(native):
    """The allocation-free reaction rejects one cell more than its documented
    maximum before touching the device (the buffer is a host array of four
    doubles, never read)."""
    src = open(os.path.join(ROOT, "include", "mr.h")).read()
    mx = int(re.search(r"#define MR_NOALLOC_MAX_CELLS (\d+)LL", src).group(1))
    assert mx == native.NOALLOC_MAX_CELLS
    f = native.lib().mr_react_radau5_noalloc
    f.argtypes = [C.c_int, C.POINTER(C.c_double), C.c_int, C.c_void_p, C.c_int64, C.c_int64,
                  C.c_double, C.c_double, C.c_double, C.c_void_p, C.c_void_p]
    f.restype = C.c_int
    params = (C.c_double * 4)(1e-2, 1e-5, 1.6, 2e-3)
    buf = (C.c_double * 4)()
    assert f(1, params, 4, C.addressof(buf), mx + 1, mx + 1, 5e-4, 1e-6, 1e-6, None, None) == -1
    assert f(1, params, 4, C.addressof(buf), -1, 4, 5e-4, 1e-6, 1e-6, None, None) == -1


def test_radau_schedule_setter_rejects_bad_arguments(native):
    """mr_set_radau_schedule accepts only MR_RADAU_THREAD and MR_RADAU_POOL,
    and a context; anything else is MR_EINVAL with no device work (no
    context is created here)."""
    src = open(os.path.join(ROOT, "include", "mr.h")).read()
    vals = dict(re.findall(r"(MR_RADAU_(?:THREAD|POOL)) = (\d+)", src))
    assert int(vals["MR_RADAU_THREAD"]) == native.MR_RADAU_THREAD == 0
    assert int(vals["MR_RADAU_POOL"]) == native.MR_RADAU_POOL == 1
    f = native.lib().mr_set_radau_schedule
    for sched in (0, 1, 2, -1):
        assert f(None, sched) == -1


@pytest.mark.parametrize("model,name,m", [(1, "bz", 3), (2, "nagumo", 1)])
def test_radau_work_table_matches_bench(native, model, name, m):
    """The per-event FP64 operation counts the library forms
    mr_stats.radau_alg_flops from, and the copy bench.py reports beside the
    counters (work_per_event), are the same numbers, so a reader can
    recompute the roofline's achieved rate from either."""
    import importlib.util
    spec = importlib.util.spec_from_file_location("bench", os.path.join(ROOT, "bench.py"))
    bench = importlib.util.module_from_spec(spec)
    spec.loader.exec_module(bench)
    lib_w = native.radau_work(model, m)
    bench_w = bench.radau_work(name, m)
    assert set(lib_w) == set(bench_w)
    for k in lib_w:
        assert lib_w[k] == bench_w[k], k
    with pytest.raises(native.MRError):
        native.radau_work(3, 16)  # the network model has team kernels, not this table
