"""Checkpoint and resume (mr_save / mr_load): a context restored from a file
continues bit-identically to the context that wrote it, and files written
for another problem are rejected."""
import numpy as np
import pytest

from paper_1506_04651_gb300 import inputs as I

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def mr():
    import __graft_entry__ as g
    g.build()
    from paper_1506_04651_gb300 import mr as M
    return M


def test_resume_is_bit_identical(mr, tmp_path):
    J, eta, dt = 8, 1e-3, 1e-3
    u0 = I.bz_cross_2d(J, 2, w=0.01, amp=0.1)
    a = mr.Context(mr.problem(2, J))
    a.build(u0, eta)
    for _ in range(2):
        a.strang(dt, eta)
    path = str(tmp_path / "ck.mrgb")
    a.save(path)
    b = mr.Context(mr.problem(2, J))
    b.build(I.bz_front_2d(J, 1), eta)  # some other state, replaced by the load
    b.load(path)
    ka, va = a.leaves()
    kb, vb = b.leaves()
    assert np.array_equal(ka, kb) and np.array_equal(va, vb)
    for _ in range(2):
        a.strang(dt, eta)
        b.strang(dt, eta)
    ka, va = a.leaves()
    kb, vb = b.leaves()
    assert np.array_equal(ka, kb) and np.array_equal(va, vb)


def test_load_rejects_other_problem_and_bad_files(mr, tmp_path):
    J = 7
    a = mr.Context(mr.problem(2, J))
    a.build(I.bz_front_2d(J, 1), 1e-3)
    path = str(tmp_path / "ck.mrgb")
    a.save(path)
    keys0, vals0 = a.leaves()
    other = mr.Context(mr.problem(2, J + 1))
    other.build(I.bz_front_2d(J + 1, 1), 1e-3)
    with pytest.raises(mr.MRError) as e:
        other.load(path)
    assert e.value.code == -1
    with pytest.raises(mr.MRError) as e:
        a.load(str(tmp_path / "missing.mrgb"))
    assert e.value.code == -50
    bad = tmp_path / "trunc.mrgb"
    bad.write_bytes(open(path, "rb").read()[:100])
    with pytest.raises(mr.MRError) as e:
        a.load(str(bad))
    assert e.value.code == -50
    keys1, vals1 = a.leaves()  # failed loads leave the context as it was
    assert np.array_equal(keys0, keys1) and np.array_equal(vals0, vals1)


def test_version_1_files_still_load(mr, tmp_path):
    """Format version 1 stored 16 diffusion coefficients after the 8
    parameters (version 2 stores MR_MAX_SPECIES = 32): a version-1 file,
    rebuilt here from a version-2 one, loads to the same leaves."""
    import struct
    J = 7
    a = mr.Context(mr.problem(2, J))
    a.build(I.bz_front_2d(J, 1), 1e-3)
    path = str(tmp_path / "v2.mrgb")
    a.save(path)
    raw = open(path, "rb").read()
    assert struct.unpack_from("<i", raw, 8)[0] == 2
    header = bytearray(raw[:64])
    struct.pack_into("<i", header, 8, 1)
    params = raw[64:64 + 8 * 8]
    d16 = raw[64 + 8 * 8:64 + 8 * 8 + 16 * 8]
    rest = raw[64 + 8 * 8 + 32 * 8:]
    v1 = tmp_path / "v1.mrgb"
    v1.write_bytes(bytes(header) + params + d16 + rest)
    b = mr.Context(mr.problem(2, J))
    b.build(I.bz_front_2d(J, 2), 1e-3)
    b.load(str(v1))
    ka, va = a.leaves()
    kb, vb = b.leaves()
    assert np.array_equal(ka, kb) and np.array_equal(va, vb)
