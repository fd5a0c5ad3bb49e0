"""The C-ABI library builds, loads without a GPU, exports every declared entry
point, and rejects invalid arguments on the host before touching CUDA."""
import ctypes
import os
import re

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.fixture(scope="module")
def lib():
    import __graft_entry__
    __graft_entry__.build()
    from paper_2501_10689_gb300 import kzprecode
    return kzprecode.load()


def declared_functions():
    names = []
    for fn in os.listdir(os.path.join(ROOT, "include")):
        if fn.endswith(".h"):
            text = open(os.path.join(ROOT, "include", fn)).read()
            text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
            names += re.findall(r"^\s*(?:[\w\s\*]+?)\b(kz_\w+)\s*\(", text, flags=re.M)
    return sorted(set(names))


def test_every_declared_symbol_is_exported(lib):
    names = declared_functions()
    assert len(names) >= 10
    for n in names:
        assert hasattr(lib, n), n
    from paper_2501_10689_gb300 import kzprecode
    assert sorted(kzprecode.EXPORTS) == names


def test_version(lib):
    assert lib.kz_version() >= 10000


FAKE = ctypes.c_void_p(0x10000)  # never dereferenced: validation fails first


def _create(lib, K, Nt, off, ln, H=FAKE, prec=0):
    import numpy as np
    o = np.asarray(off, dtype=np.int32)
    l = np.asarray(ln, dtype=np.int32)
    h = ctypes.c_void_p()
    rc = lib.kz_plan_create(ctypes.byref(h), K, Nt, o.ctypes.data_as(ctypes.c_void_p),
                            l.ctypes.data_as(ctypes.c_void_p), H, prec, None)
    return rc, lib.kz_last_error().decode()


def test_plan_create_rejects_bad_input(lib):
    from paper_2501_10689_gb300.kzprecode import KZ_ERR_INVALID_ARG
    assert _create(lib, 4, 4, [0] * 4, [1] * 4)[0] == KZ_ERR_INVALID_ARG  # K >= Nt
    assert _create(lib, 0, 8, [], [])[0] == KZ_ERR_INVALID_ARG
    rc, msg = _create(lib, 2, 8, [0, 5], [3, 4])  # VR past the array
    assert rc == KZ_ERR_INVALID_ARG and "outside" in msg
    assert _create(lib, 2, 8, [0, -1], [3, 2])[0] == KZ_ERR_INVALID_ARG
    assert _create(lib, 2, 8, [0, 1], [3, 0])[0] == KZ_ERR_INVALID_ARG  # empty VR
    assert _create(lib, 2, 8, [0, 1], [3, 2], H=ctypes.c_void_p(0x10004))[0] == KZ_ERR_INVALID_ARG  # misaligned
    assert _create(lib, 2, 8, [0, 1], [3, 2], H=None)[0] == KZ_ERR_INVALID_ARG
    assert _create(lib, 2, 8, [0, 1], [3, 2], prec=7)[0] == KZ_ERR_INVALID_ARG


def test_solve_calls_reject_null_and_bad_enums(lib):
    from paper_2501_10689_gb300.kzprecode import KZ_ERR_INVALID_ARG
    rc = lib.kz_precode(None, FAKE, 1, 1.0, 5, 0, 1e-6, 10, 0, FAKE, None, FAKE, FAKE, None, 0, 0, None)
    assert rc == KZ_ERR_INVALID_ARG and "plan" in lib.kz_last_error().decode()
    rc = lib.kz_precode_batched(None, 0, 1e-6, 10, 0, 0, None, None)
    assert rc == KZ_ERR_INVALID_ARG
    h = ctypes.c_void_p()
    rc = lib.kz_batch_prepare(ctypes.byref(h), None, 0, 1, 5, 0, 0, None)
    assert rc == KZ_ERR_INVALID_ARG
    rc = lib.kz_precode_adjoint(None, 1, 1.0, FAKE, FAKE, FAKE, FAKE, 1e-6, 10, FAKE, FAKE, FAKE, FAKE, FAKE, FAKE,
                                None, None)
    assert rc == KZ_ERR_INVALID_ARG


def test_binding_fails_loudly_without_library(monkeypatch, tmp_path):
    from paper_2501_10689_gb300 import kzprecode
    monkeypatch.setattr(kzprecode, "_lib", None)
    monkeypatch.setattr(kzprecode, "library_path", lambda: str(tmp_path / "missing.so"))
    with pytest.raises(RuntimeError, match="missing"):
        kzprecode.load()


def test_batch_query_and_launch_reject_null(lib):
    from paper_2501_10689_gb300.kzprecode import KZ_ERR_INVALID_ARG
    v = [ctypes.c_int32() for _ in range(4)]
    rc = lib.kz_batch_query(None, *[ctypes.byref(x) for x in v])
    assert rc == KZ_ERR_INVALID_ARG and "batch" in lib.kz_last_error().decode()
    assert lib.kz_batch_set_launch(None, 3, 8, 512, None) == KZ_ERR_INVALID_ARG
    assert lib.kz_batch_rebind(None, None, None) == KZ_ERR_INVALID_ARG


def test_plan_dense_rejects_bad_input(lib):
    """kz_plan_dense validates like kz_plan_create, on the host, before any CUDA call."""
    import numpy as np
    from paper_2501_10689_gb300.kzprecode import KZ_ERR_INVALID_ARG

    def dense(K, Nt, off, ln, H=FAKE):
        o = np.asarray(off, dtype=np.int32)
        l = np.asarray(ln, dtype=np.int32)
        h = ctypes.c_void_p()
        rc = lib.kz_plan_dense(ctypes.byref(h), K, Nt, o.ctypes.data_as(ctypes.c_void_p),
                               l.ctypes.data_as(ctypes.c_void_p), H, 0, None)
        return rc, lib.kz_last_error().decode()

    assert dense(4, 4, [0] * 4, [1] * 4)[0] == KZ_ERR_INVALID_ARG      # K >= Nt
    rc, msg = dense(2, 8, [0, 5], [3, 4])                               # VR past the array
    assert rc == KZ_ERR_INVALID_ARG and "kz_plan_dense" in msg
    rc, msg = dense(2, 8, [0, 1], [3, 4], H=None)
    assert rc == KZ_ERR_INVALID_ARG and "H_dense" in msg
    assert dense(2, 8, [0, 1], [3, 4], H=ctypes.c_void_p(0x10004))[0] == KZ_ERR_INVALID_ARG  # misaligned


def test_precoder_matrix_rejects_bad_input(lib):
    from paper_2501_10689_gb300.kzprecode import KZ_ERR_INVALID_ARG
    P = ctypes.c_void_p
    assert lib.kz_precoder_matrix(None, FAKE, 4, 2, 0, FAKE, None, None) == KZ_ERR_INVALID_ARG
    assert "kz_precoder_matrix" in lib.kz_last_error().decode()
