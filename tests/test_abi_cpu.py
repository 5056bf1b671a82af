"""CPU checks of the C ABI: the library loads, exports what the header declares,
and rejects invalid arguments before touching a GPU."""
import ctypes
import os
import re

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.fixture(scope="module")
def lib():
    from paper_1510_06689_gb300 import build, tucker

    build.build()
    return tucker.load()


def header_functions():
    text = open(os.path.join(ROOT, "include", "tucker.h")).read()
    return sorted(set(re.findall(r"TUCKER_API[^;(]*?\b(tucker_\w+)\s*\(", text)))


def test_header_declares_the_boundary():
    names = header_functions()
    for required in ("tucker_sthosvd", "tucker_reconstruct", "tucker_rel_error", "tucker_result_free"):
        assert required in names


def test_every_declared_symbol_is_exported(lib):
    from paper_1510_06689_gb300 import tucker

    names = header_functions()
    assert sorted(tucker.EXPORTS) == names
    for n in names:
        assert hasattr(lib, n), n


def test_status_strings(lib):
    assert lib.tucker_status_string(0) == b"ok"
    assert lib.tucker_status_string(-1) == b"invalid argument"
    assert lib.tucker_status_string(-4) == b"eigensolver did not converge"
    assert lib.tucker_status_string(12345) == b"unknown status"


def test_invalid_arguments_are_rejected_on_host(lib):
    from paper_1510_06689_gb300 import tucker

    dims = (ctypes.c_int64 * 3)(4, 5, 6)
    res = tucker._Result()
    fake = ctypes.c_void_p(0x1000)  # never dereferenced: validation fails first
    # NULL tensor
    assert lib.tucker_sthosvd(None, 0, dims, 3, 1e-3, None, 0, None, ctypes.byref(res)) == -1
    assert b"NULL" in lib.tucker_last_error()
    # bad N, bad dims, NaN eps, bad order, bad dtype, bad precision
    assert lib.tucker_sthosvd(fake, 0, dims, 0, 1e-3, None, 0, None, ctypes.byref(res)) == -1
    bad = (ctypes.c_int64 * 3)(4, 0, 6)
    assert lib.tucker_sthosvd(fake, 0, bad, 3, 1e-3, None, 0, None, ctypes.byref(res)) == -1
    big = (ctypes.c_int64 * 3)(4, 5000, 6)
    assert lib.tucker_sthosvd(fake, 0, big, 3, 1e-3, None, 0, None, ctypes.byref(res)) == -1
    assert lib.tucker_sthosvd(fake, 0, dims, 3, float("nan"), None, 0, None, ctypes.byref(res)) == -1
    order = (ctypes.c_int * 3)(0, 0, 2)
    assert lib.tucker_sthosvd(fake, 0, dims, 3, 1e-3, order, 0, None, ctypes.byref(res)) == -1
    assert b"permutation" in lib.tucker_last_error()
    assert lib.tucker_sthosvd(fake, 7, dims, 3, 1e-3, None, 0, None, ctypes.byref(res)) == -1
    assert lib.tucker_sthosvd(fake, 0, dims, 3, 1e-3, None, 9, None, ctypes.byref(res)) == -1
    assert lib.tucker_sthosvd(fake, 0, dims, 3, 1e-3, None, 0, None, None) == -1
    # step entry points
    out = ctypes.c_double()
    assert lib.tucker_norm2(None, 0, 10, ctypes.byref(out), None) == -1
    assert lib.tucker_gram(fake, 0, 1, 0, 1, fake, None) == -1
    assert lib.tucker_gram(fake, 0, 1, 2000, 1, fake, None) == -1
    assert lib.tucker_eig(fake, 0, fake, fake, None, None) == -1
    r, t = ctypes.c_int64(), ctypes.c_double()
    assert lib.tucker_rank_cut(fake, 4, float("nan"), 0, ctypes.byref(r), ctypes.byref(t), None) == -1
    assert lib.tucker_ttm(fake, 0, 1, 3, 1, fake, 0, 1, fake, None) == -1
    # results
    assert lib.tucker_reconstruct(ctypes.byref(res), fake, None) == -1
    rel = ctypes.c_double()
    assert lib.tucker_rel_error(fake, 0, ctypes.byref(res), ctypes.byref(rel), None) == -1
    lib.tucker_result_free(ctypes.byref(res))  # safe on an empty result
    lib.tucker_result_free(None)


def test_profile_counters_without_gpu(lib):
    from paper_1510_06689_gb300 import tucker

    tucker.profile_enable(True)
    p = tucker.profile_read()
    assert set(p) == set(tucker.PHASES)
    assert all(v["ms"] == 0 and v["launches"] == 0 for v in p.values())
    tucker.profile_enable(False)
    assert tucker.launch_count() >= 0


def test_binding_fails_loudly_without_library(tmp_path):
    from paper_1510_06689_gb300 import tucker

    saved = tucker._lib
    tucker._lib = None
    try:
        with pytest.raises(RuntimeError, match="not built"):
            tucker.load(str(tmp_path / "missing.so"))
    finally:
        tucker._lib = saved
